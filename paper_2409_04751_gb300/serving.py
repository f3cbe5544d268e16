"""Continuous-batching render server over device-resident scenes (forward rendering).

Requests (scene, camera) arrive over time. The server keeps a few slots, each a CUDA stream with
its own buffers; a free slot takes the oldest pending request plus every other pending request
of the same scene that fits (at most `max_batch_views` views and the HBM budget left), and
renders them in one call per stage. Slots run concurrently, so work of requests that arrive
while others are on the GPU overlaps on the device. Completion is detected with CUDA events;
latency = completion time - arrival time on the host clock.

A request's image does not depend on which other views share its batch: every kernel treats
views independently (tested).

The intersection count of a batch is not known before it runs. Each slot sizes its key buffers
from the intersections per pixel seen so far for that scene (times a margin); a batch whose
count overflows is detected on completion (status word) and re-run with room to spare.
"""
import collections
import time
from dataclasses import dataclass, field

import torch

from . import fgs
from .renderer import FisheyeRenderer


@dataclass
class Request:
    rid: int
    scene: int
    cam: dict
    t_arrival: float
    t_done: float = 0.0
    image: object = None
    retries: int = 0

    @property
    def pixels(self):
        return int(self.cam["width"]) * int(self.cam["height"])


@dataclass
class _Batch:
    reqs: list
    event: object
    frame: object
    bytes: int
    t_launch: float


@dataclass
class _Slot:
    stream: object
    renderer: FisheyeRenderer
    batch: object = None


@dataclass
class ServeStats:
    latencies_ms: list = field(default_factory=list)
    views: int = 0
    batches: int = 0
    retries: int = 0
    wall_s: float = 0.0

    def summary(self):
        import numpy as np
        lat = np.asarray(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return dict(views=self.views, batches=self.batches, retries=self.retries,
                    views_per_s=self.views / max(self.wall_s, 1e-9),
                    p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                    mean_ms=float(lat.mean()), wall_s=self.wall_s)


class Server:
    def __init__(self, scenes_gs, n_slots=3, max_batch_views=16, hbm_budget_bytes=48 << 30,
                 margin=1.6, keep_images=False, device="cuda"):
        self.scenes = scenes_gs
        self.device = torch.device(device)
        self.slots = [_Slot(torch.cuda.Stream(self.device), FisheyeRenderer(self.device))
                      for _ in range(n_slots)]
        self.max_batch_views = max_batch_views
        self.budget = int(hbm_budget_bytes)
        self.margin = margin
        self.keep_images = keep_images
        self.pending = collections.deque()
        self.in_flight_bytes = 0
        # intersections per (f / W)^2-weighted pixel, per scene (starts pessimistic)
        self.ipp = [80.0 * max(1.0, gs["means"].shape[0] / 5e5) for gs in scenes_gs]
        self.stats = ServeStats()

    # ---------------------------------------------------------------------------------------
    def _bytes(self, scene, reqs, capacity):
        n = int(self.scenes[scene]["means"].shape[0])
        R = n * len(reqs)
        P = sum(r.pixels for r in reqs)
        ws = fgs.fgs_workspace_size(n, fgs.cameras([r.cam for r in reqs]), capacity)
        return R * 52 + capacity * 12 + ws + P * 20

    @staticmethod
    def _weight(reqs):
        """Pixels weighted by (focal length / width)^2: a footprint's area in pixels grows with
        f^2, so intersections per pixel of an equidistant view scale as (f / W)^2."""
        return sum(r.pixels * (float(r.cam["fx"]) / float(r.cam["width"])) ** 2 for r in reqs)

    def _capacity(self, scene, reqs):
        return min(int(self.ipp[scene] * self._weight(reqs) * self.margin) + 65536, (1 << 31) - 1)

    def calibrate(self, cams_by_scene):
        """Render a view per scene to learn its intersections per weighted pixel."""
        for k, cams in enumerate(cams_by_scene):
            r = FisheyeRenderer(self.device, capacity=1 << 22)
            fr = r.forward(self.scenes[k], cams, check=True)
            w = self._weight([Request(0, k, c, 0.0) for c in cams])
            self.ipp[k] = int(fr.n_intersections.item()) / max(w, 1e-9)

    def _form_batch(self):
        first = self.pending[0]
        scene = first.scene
        picked = []
        for r in list(self.pending):
            if r.scene != scene:
                continue
            trial = picked + [r]
            cap = self._capacity(scene, trial)
            if picked and (len(trial) > self.max_batch_views or
                           self.in_flight_bytes + self._bytes(scene, trial, cap) > self.budget):
                break
            picked = trial
        cap = self._capacity(scene, picked)
        need = self._bytes(scene, picked, cap)
        if self.in_flight_bytes > 0 and self.in_flight_bytes + need > self.budget:
            return None  # wait for memory to free up
        for r in picked:
            self.pending.remove(r)
        return scene, picked, cap, need

    def _launch(self, slot, scene, reqs, cap, need):
        slot.renderer.capacity = cap
        with torch.cuda.stream(slot.stream):
            fr = slot.renderer.forward(self.scenes[scene], [r.cam for r in reqs], check=False)
            ev = torch.cuda.Event()
            ev.record(slot.stream)
        slot.batch = _Batch(reqs, ev, fr, need, time.perf_counter())
        self.in_flight_bytes += need

    def _complete(self, slot, now):
        b = slot.batch
        slot.batch = None
        self.in_flight_bytes -= b.bytes
        st = fgs.fgs_read_status(slot.renderer._bufs["ws"], slot.stream)
        n_int = int(b.frame.n_intersections.item())
        scene = b.reqs[0].scene
        w = max(self._weight(b.reqs), 1e-9)
        self.ipp[scene] = max(0.95 * self.ipp[scene], n_int / w)
        if st == fgs.FGS_ERR_CAPACITY:
            self.ipp[scene] = max(self.ipp[scene], 1.2 * n_int / w)
            for r in reversed(b.reqs):
                r.retries += 1
                self.pending.appendleft(r)
            self.stats.retries += 1
            return
        if st != fgs.FGS_OK:
            raise fgs.FgsError(st, "serving batch")
        imgs = b.frame.view_images([r.cam for r in b.reqs]) if self.keep_images else None
        for k, r in enumerate(b.reqs):
            r.t_done = now
            if imgs is not None:
                r.image = imgs[k].clone()
            self.stats.latencies_ms.append(1e3 * (r.t_done - r.t_arrival))
        self.stats.views += len(b.reqs)
        self.stats.batches += 1

    def poll(self):
        """Retire finished batches and start new ones on free slots. Returns True if any work is
        pending or in flight."""
        for slot in self.slots:
            if slot.batch is not None and slot.batch.event.query():
                self._complete(slot, time.perf_counter())
        for slot in self.slots:
            if slot.batch is None and self.pending:
                formed = self._form_batch()
                if formed is None:
                    break
                self._launch(slot, *formed)
        return bool(self.pending) or any(s.batch is not None for s in self.slots)

    def run(self, requests, t0=None):
        """Serve `requests` (sorted by t_arrival, seconds relative to the start) in real time.
        Returns ServeStats."""
        t0 = time.perf_counter() if t0 is None else t0
        for r in requests:
            r.t_arrival += t0
        i = 0
        while i < len(requests) or self.poll():
            now = time.perf_counter()
            while i < len(requests) and requests[i].t_arrival <= now:
                self.pending.append(requests[i])
                i += 1
            busy = self.poll()
            if not busy and i < len(requests):
                time.sleep(max(0.0, min(5e-4, requests[i].t_arrival - time.perf_counter())))
        self.stats.wall_s = time.perf_counter() - t0
        return self.stats


def serve_plain(scenes_gs, requests, device="cuda", keep_images=False):
    """One request at a time, one single-view call sequence each, in arrival order."""
    r = FisheyeRenderer(torch.device(device), capacity=1 << 22)
    stats = ServeStats()
    t0 = time.perf_counter()
    for q in requests:
        q.t_arrival += t0
    for q in requests:
        now = time.perf_counter()
        if q.t_arrival > now:
            time.sleep(q.t_arrival - now)
        fr = r.forward(scenes_gs[q.scene], [q.cam], check=True)  # syncs: the result is ready
        q.t_done = time.perf_counter()
        if keep_images:
            q.image = fr.view_images([q.cam])[0].clone()
        stats.latencies_ms.append(1e3 * (q.t_done - q.t_arrival))
        stats.views += 1
        stats.batches += 1
    stats.wall_s = time.perf_counter() - t0
    return stats


def poisson_requests(rate, duration_s, n_scenes, seed, sizes=None, fov=(150.0, 200.0)):
    """Poisson arrivals at `rate` per second for `duration_s`; each request picks a scene
    uniformly, a random pose, a square resolution from `sizes` and a FOV ~ U(fov)."""
    import numpy as np
    from . import scenes as sc
    rng = np.random.default_rng(seed)
    sizes = sizes or list(range(512, 2049, 256))
    t = 0.0
    out = []
    k = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration_s:
            break
        s = int(rng.integers(len(sizes)))
        cam = sc.pose_camera(sizes[s], sizes[s], float(rng.uniform(*fov)), seed=seed * 100000 + k)
        out.append(Request(k, int(rng.integers(n_scenes)), cam, t))
        k += 1
    return out
