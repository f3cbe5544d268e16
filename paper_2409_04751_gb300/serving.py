"""Continuous-batching render server over device-resident scenes (forward rendering).

Requests (scene, camera) arrive over time. The server keeps a few slots, each a CUDA stream with
its own buffers. A free slot takes the pending requests in arrival order - of any scene and
any size - while the batch stays within `max_batch_views` views and the HBM budget left, and
renders them with one call per stage for each scene of the batch (all views of a scene in one
multi-view call), on its stream. Slots run concurrently, so the work of requests that arrive
while others are on the GPU overlaps on the device. When the device is idle a free slot starts
at once; while other work is in flight it waits up to `window_ms` (or until a full batch is
pending) so that requests arriving meanwhile join the batch: the device is busy anyway, and one
call over several views costs less than one call per view. Completion is detected with CUDA
events; latency = completion time - arrival time on the host clock.

A request's image does not depend on which other views share its batch: every kernel treats
views independently (tested).

The intersection count of a batch is not known before it runs. Each slot sizes the key buffers
of a scene's views from the intersections per weighted pixel of that scene (calibrated on the
worst of several poses, times a margin, decaying slowly); a group that still overflows is
detected on completion (status word) and re-run with room to spare.
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

    @property
    def tiles(self):
        return ((int(self.cam["width"]) + 15) // 16) * ((int(self.cam["height"]) + 15) // 16)


@dataclass
class _Group:
    """The views of one scene inside a batch: one multi-view call per stage, and an event
    recorded after it, so that the group completes as soon as its own calls have run."""
    scene: int
    reqs: list
    cap: int
    bytes: int
    frame: object = None
    event: object = None
    done: bool = False


@dataclass
class _Batch:
    groups: list
    bytes: int
    t_launch: float
    views_done: int = 0


@dataclass
class _Slot:
    stream: object
    renderers: dict = field(default_factory=dict)  # scene -> FisheyeRenderer (its buffers)
    batch: object = None


@dataclass
class ServeStats:
    latencies_ms: list = field(default_factory=list)
    views: int = 0
    batches: int = 0
    retries: int = 0
    wall_s: float = 0.0
    batch_views: list = field(default_factory=list)   # views per completed batch
    batch_scenes: list = field(default_factory=list)  # scenes per completed batch

    def summary(self):
        import numpy as np
        lat = np.asarray(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        hist = collections.Counter(self.batch_views)
        return dict(views=self.views, batches=self.batches, retries=self.retries,
                    views_per_s=self.views / max(self.wall_s, 1e-9),
                    p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                    mean_ms=float(lat.mean()), wall_s=self.wall_s,
                    views_per_batch_mean=self.views / max(self.batches, 1),
                    views_per_batch_hist={int(k): int(v) for k, v in sorted(hist.items())},
                    multi_scene_batches=int(sum(1 for n in self.batch_scenes if n > 1)))


class Server:
    def __init__(self, scenes_gs, n_slots=2, max_batch_views=16, hbm_budget_bytes=48 << 30,
                 margin=2.0, window_ms=0.5, max_group_records=8 << 20, keep_images=False,
                 device="cuda"):
        self.scenes = scenes_gs
        self.device = torch.device(device)
        self.slots = [_Slot(torch.cuda.Stream(self.device)) for _ in range(n_slots)]
        self.max_batch_views = max_batch_views
        self.budget = int(hbm_budget_bytes)
        self.margin = margin
        self.window_s = window_ms * 1e-3
        # views of one scene per group: at most this many records (views x Gaussians)
        self.max_group_records = int(max_group_records)
        self.keep_images = keep_images
        self.pending = collections.deque()
        self.in_flight_bytes = 0
        # intersections per (f / W)^2-weighted pixel, per scene (starts pessimistic)
        self.ipp = [80.0 * max(1.0, gs["means"].shape[0] / 5e5) for gs in scenes_gs]
        self.stats = ServeStats()

    # ---------------------------------------------------------------------------------------
    def _bytes(self, scene, reqs, capacity):
        """Device bytes of one scene group: records and tiles_touched, keys and values, the
        workspace, images, final T and processed counts."""
        n = int(self.scenes[scene]["means"].shape[0])
        R = n * len(reqs)
        P = sum(r.pixels for r in reqs)
        ws = fgs.fgs_workspace_size(n, fgs.cameras([r.cam for r in reqs]), capacity)
        return R * 52 + capacity * 12 + ws + P * 20

    def _bytes_estimate(self, scene, reqs, capacity):
        """_bytes without the library call (the workspace from its dominant regions: 60 bytes
        per record, 8 per key slot, 16 per tile), for the budget checks while a batch is
        formed."""
        n = int(self.scenes[scene]["means"].shape[0])
        R = n * len(reqs)
        P = sum(r.pixels for r in reqs)
        T = sum(r.tiles for r in reqs)
        return R * (52 + 60) + capacity * (12 + 8) + T * 16 + P * 20 + 4096

    @staticmethod
    def _weight(reqs):
        """Pixels weighted by (focal length / width)^2: a footprint's area in pixels grows with
        f^2, so intersections per pixel of an equidistant view scale as (f / W)^2."""
        return sum(r.pixels * (float(r.cam["fx"]) / float(r.cam["width"])) ** 2 for r in reqs)

    def _capacity(self, scene, reqs):
        return min(int(self.ipp[scene] * self._weight(reqs) * self.margin) + 65536, (1 << 31) - 1)

    def calibrate(self, cams_by_scene):
        """Render the given views of each scene to learn its intersections per weighted pixel
        (the largest over the views)."""
        for k, cams in enumerate(cams_by_scene):
            r = FisheyeRenderer(self.device, capacity=1 << 22)
            ipp = 0.0
            for c in cams:
                fr = r.forward(self.scenes[k], [c], check=True)
                w = self._weight([Request(0, k, c, 0.0)])
                ipp = max(ipp, int(fr.n_intersections.item()) / max(w, 1e-9))
            self.ipp[k] = ipp

    def _form_batch(self):
        """The pending requests in arrival order, of any scene, while the batch holds at most
        max_batch_views views and (beside the work in flight) fits the HBM budget. Returns the
        batch's scene groups (in order of first appearance) and their bytes, or None if the
        oldest request does not fit beside the work in flight (an idle device always admits
        it)."""
        by = collections.OrderedDict()  # scene -> requests
        est = {}                        # scene -> estimated bytes of its group
        total, picked = 0, 0
        for r in self.pending:
            if picked + 1 > self.max_batch_views:
                break
            rs = by.get(r.scene, []) + [r]
            if picked and len(rs) * int(self.scenes[r.scene]["means"].shape[0]) > self.max_group_records:
                break
            b = self._bytes_estimate(r.scene, rs, self._capacity(r.scene, rs))
            t = total - est.get(r.scene, 0) + b
            if picked and self.in_flight_bytes + t > self.budget:
                break
            by[r.scene], est[r.scene], total, picked = rs, b, t, picked + 1
        groups = []
        for scene, rs in by.items():
            cap = self._capacity(scene, rs)
            groups.append(_Group(scene, rs, cap, self._bytes(scene, rs, cap)))
        need = sum(g.bytes for g in groups)
        if self.in_flight_bytes > 0 and self.in_flight_bytes + need > self.budget:
            return None  # wait for memory to free up
        taken = {id(r) for g in groups for r in g.reqs}
        self.pending = collections.deque(r for r in self.pending if id(r) not in taken)
        return groups, need

    def _ready(self, now):
        """Whether a free slot starts a batch now: at once on an idle device; while other
        batches are in flight, when a full batch is pending or the oldest request has waited
        the window."""
        if not self.pending:
            return False
        if not any(s.batch is not None for s in self.slots):
            return True
        if len(self.pending) >= self.max_batch_views:
            return True
        return now - self.pending[0].t_arrival >= self.window_s

    def warm(self, max_size=2048, fov=150.0):
        """Size every slot's buffers for the largest group each scene can form (its most views
        at max_size^2 and the narrowest FOV, whose longer focal length gives the largest key
        capacity), before serving: the serving loop then reuses them instead of allocating
        device memory between requests."""
        for k, gs in enumerate(self.scenes):
            n = int(gs["means"].shape[0])
            views = max(1, min(self.max_batch_views, self.max_group_records // max(n, 1)))
            reqs = [Request(0, k, _wide_camera(max_size, fov, j), 0.0) for j in range(views)]
            cap = self._capacity(k, reqs)
            for slot in self.slots:
                r = self._renderer(slot, k)
                r.capacity = cap
                with torch.cuda.stream(slot.stream):
                    r.forward(gs, [q.cam for q in reqs], check=False)
        torch.cuda.synchronize(self.device)

    def _renderer(self, slot, scene):
        r = slot.renderers.get(scene)
        if r is None:
            r = slot.renderers[scene] = FisheyeRenderer(self.device)
        return r

    def _launch(self, slot, groups, need):
        with torch.cuda.stream(slot.stream):
            for g in groups:
                r = self._renderer(slot, g.scene)
                r.capacity = g.cap
                g.frame = r.forward(self.scenes[g.scene], [q.cam for q in g.reqs], check=False)
                g.event = torch.cuda.Event()
                g.event.record(slot.stream)
        slot.batch = _Batch(groups, need, time.perf_counter())
        self.in_flight_bytes += need

    def _complete_group(self, slot, g, now):
        """Results of one scene group whose calls have run: latencies, or a re-queue of its
        requests if its key buffers overflowed."""
        g.done = True
        r = self._renderer(slot, g.scene)
        st = fgs.fgs_read_status(r._bufs["ws"], slot.stream)
        n_int = int(g.frame.n_intersections.item())
        w = max(self._weight(g.reqs), 1e-9)
        self.ipp[g.scene] = max(0.99 * self.ipp[g.scene], n_int / w)
        if st == fgs.FGS_ERR_CAPACITY:
            self.ipp[g.scene] = max(self.ipp[g.scene], 1.2 * n_int / w)
            for q in reversed(g.reqs):
                q.retries += 1
                self.pending.appendleft(q)
            self.stats.retries += 1
            return 0
        if st != fgs.FGS_OK:
            raise fgs.FgsError(st, "serving batch")
        imgs = g.frame.view_images([q.cam for q in g.reqs]) if self.keep_images else None
        for k, q in enumerate(g.reqs):
            q.t_done = now
            if imgs is not None:
                q.image = imgs[k].clone()
            self.stats.latencies_ms.append(1e3 * (q.t_done - q.t_arrival))
        return len(g.reqs)

    def _retire(self, slot):
        """Complete the finished groups of the slot's batch; free the slot when all are."""
        b = slot.batch
        for g in b.groups:
            if not g.done and g.event.query():
                b.views_done += self._complete_group(slot, g, time.perf_counter())
        if all(g.done for g in b.groups):
            slot.batch = None
            self.in_flight_bytes -= b.bytes
            done = b.views_done
            if done:
                self.stats.views += done
                self.stats.batches += 1
                self.stats.batch_views.append(done)
                self.stats.batch_scenes.append(len(b.groups))

    def poll(self):
        """Retire finished work and start new batches on free slots. Returns True if any work
        is pending or in flight."""
        for slot in self.slots:
            if slot.batch is not None:
                self._retire(slot)
        for slot in self.slots:
            if slot.batch is None and self._ready(time.perf_counter()):
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


def _wide_camera(size, fov, seed):
    from . import scenes as sc
    return sc.pose_camera(size, size, fov, seed=seed)


def serve_plain(scenes_gs, requests, device="cuda", keep_images=False, warm_size=0):
    """One request at a time, one single-view call sequence each, in arrival order. warm_size
    > 0 first renders one warm_size^2 view at 150 degrees of every scene (untimed), so that the
    buffers are sized before the requests arrive."""
    r = FisheyeRenderer(torch.device(device), capacity=1 << 22)
    for gs in (scenes_gs if warm_size else []):
        r.forward(gs, [_wide_camera(warm_size, 150.0, 0)], check=True)
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
