"""Rendering steps fed from and drained to host memory, with the copies overlapping the compute.

A HostPipeline owns n_sets device copies (two by default) of the inputs (Gaussian parameters
and dL/dimage) and of the outputs (images and parameter gradients), a copy-in stream, a compute
stream and a copy-out stream. Step i copies its inputs into set i % n_sets while step i - 1
computes on another set, and its outputs leave set i % n_sets while step i + 1 computes: the
host link and the GPU work overlap, so a stream of steps runs at about the slower of the two
instead of their sum. A set is reused n_sets steps later; on the bench workload the host link
(about 160 GB/s each way with both directions busy) bounds the stream, and a third set gains
nothing. Each step is the
plain call sequence fgs_preprocess -> fgs_bin_sort -> fgs_rasterize -> fgs_backward on its own
inputs, with the scratch buffers (records, keys, workspace) shared on the compute stream; events
order the three streams, so every step's results equal those of the plain path. With
use_graph=True (the default) that call sequence is captured once per input set in a CUDA graph
when the pipeline is sized, and each step replays the graph of its set.
"""
import torch

from . import fgs
from .renderer import FisheyeRenderer, gaussians_of

_KEYS = ("means", "scales", "quats", "opacities", "sh")


class HostPipeline:
    def __init__(self, n, sh_degree, cams_py, device="cuda", capacity=1 << 22, bg=None,
                 backward=True, use_graph=True, shape=(0, 0), n_sets=2):
        self.device = torch.device(device)
        dev = self.device
        self.n, self.sh_degree = int(n), int(sh_degree)
        self.cams_py = list(cams_py)
        self.cams = fgs.cameras(self.cams_py)
        self.P = fgs.fgs_total_pixels(self.cams)
        self.bg = None if bg is None else tuple(float(v) for v in bg)
        self.backward = bool(backward)
        self.n_sets = int(n_sets)
        if self.n_sets < 2:
            raise ValueError("n_sets >= 2")
        K = (self.sh_degree + 1) ** 2
        shapes = dict(means=(n, 3), scales=(n, 3), quats=(n, 4), opacities=(n,), sh=(n, K, 3))
        z = lambda s: torch.zeros(s, dtype=torch.float32, device=dev)
        S = self.n_sets
        self.inp = [{k: z(shapes[k]) for k in _KEYS} for _ in range(S)]
        self.dL = [z((3 * self.P,)) for _ in range(S)]
        self.img = [z((3 * self.P,)) for _ in range(S)]
        self.grad = [{k: z(shapes[k]) for k in _KEYS} for _ in range(S)]
        self.renderer = FisheyeRenderer(dev, capacity=capacity, fwd_ppt=shape[0], bwd_ppt=shape[1])
        self.s_in = torch.cuda.Stream(dev)
        self.s_run = torch.cuda.Stream(dev)
        self.s_out = torch.cuda.Stream(dev)
        E = lambda: torch.cuda.Event()
        self.ev_in = [E() for _ in range(S)]    # inputs of set k landed
        self.ev_run = [E() for _ in range(S)]   # compute on set k done
        self.ev_out = [E() for _ in range(S)]   # outputs of set k left
        self.step = 0
        self.use_graph = bool(use_graph)
        self.graphs = None

    def size(self, host_inputs):
        """Size the key buffers with one checked forward on these inputs (synchronises)."""
        for k in _KEYS:
            self.inp[0][k].copy_(host_inputs[k])
        gs = dict(self.inp[0], sh_degree=self.sh_degree)
        self.renderer.forward(gs, self.cams_py, bg=self.bg, check=True)
        r = self.renderer
        r.capacity = int(int(r._bufs["nint"].item()) * 1.1) + 4096
        r.forward(gs, self.cams_py, bg=self.bg, check=True)
        torch.cuda.synchronize(self.device)
        if self.use_graph:
            # one warm pass of the full call sequence, then one capture per input set
            self.s_run.wait_stream(torch.cuda.current_stream(self.device))
            with torch.cuda.stream(self.s_run):
                self._compute(0)
            self.s_run.synchronize()
            self.graphs = []
            for k in range(self.n_sets):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=self.s_run):
                    self._compute(k)
                self.graphs.append(g)
            torch.cuda.synchronize(self.device)

    def _compute(self, k):
        """The step's calls on input/output set k, on the current stream."""
        inp, dL, img, grad = self.inp[k], self.dL[k], self.img[k], self.grad[k]
        r = self.renderer
        gs = dict(inp, sh_degree=self.sh_degree)
        g = gaussians_of(gs)
        ws = r._bufs["ws"]
        cap = r.capacity
        wsb = fgs.fgs_workspace_size(self.n, self.cams, cap)
        rec, tt = r._bufs["records"], r._bufs["tt"]
        keys, vals, rg, nint = r._bufs["keys"], r._bufs["vals"], r._bufs["ranges"], r._bufs["nint"]
        fT, npr = r._bufs["final_T"], r._bufs["nproc"]
        fgs.fgs_preprocess(g, self.cams, rec, tt)
        fgs.fgs_bin_sort(rec, tt, self.n, self.cams, keys, vals, cap, rg, nint, ws, wsb)
        fgs.fgs_rasterize(rec, vals, rg, self.cams, self.bg, img, fT, npr, ws, wsb, opts=r.opts)
        if self.backward:
            fgs.fgs_backward(g, self.cams, rec, tt, vals, rg, self.bg, fT, npr, dL,
                             grad["means"], grad["scales"], grad["quats"],
                             grad["opacities"], grad["sh"], ws, wsb, opts=r.opts)

    def submit(self, host_inputs, host_dL, host_img, host_grads):
        """Queue one step: host_inputs (dict of pinned tensors) and host_dL in, host_img and
        host_grads (pinned) out. Asynchronous; the host buffers must stay untouched until
        `wait(handle)` returns. Returns a handle."""
        k = self.step % self.n_sets
        inp, dL, img, grad = self.inp[k], self.dL[k], self.img[k], self.grad[k]
        # copy in once the compute that last read set k is done
        self.s_in.wait_event(self.ev_run[k])
        with torch.cuda.stream(self.s_in):
            for key in _KEYS:
                inp[key].copy_(host_inputs[key], non_blocking=True)
            dL.copy_(host_dL, non_blocking=True)
            self.ev_in[k].record(self.s_in)
        # compute once the inputs landed and the outputs of set k have left
        self.s_run.wait_event(self.ev_in[k])
        self.s_run.wait_event(self.ev_out[k])
        with torch.cuda.stream(self.s_run):
            if self.graphs is not None:
                self.graphs[k].replay()
            else:
                self._compute(k)
            self.ev_run[k].record(self.s_run)
        # copy out after the compute
        self.s_out.wait_event(self.ev_run[k])
        with torch.cuda.stream(self.s_out):
            host_img.copy_(img, non_blocking=True)
            if self.backward:
                for key in _KEYS:
                    host_grads[key].copy_(grad[key], non_blocking=True)
            done = torch.cuda.Event()
            done.record(self.s_out)
            self.ev_out[k].record(self.s_out)
        self.step += 1
        return done

    def wait(self, handle):
        """Block until the step of `handle` has its outputs in host memory; returns the device
        status of the shared workspace (FGS_OK unless a step overflowed the key capacity)."""
        handle.synchronize()
        return fgs.fgs_read_status(self.renderer._bufs["ws"], self.s_run)
