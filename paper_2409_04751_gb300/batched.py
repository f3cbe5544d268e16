"""Batched multi-view rendering captured in a CUDA graph.

All views of a batch go through each stage in one launch (the kernels take up to 128 views per
call; global tile id = the view's tile offset + its local tile), and the whole forward (and
optionally backward) sequence of C-ABI calls is captured once in a CUDA graph and replayed. A
replay re-reads the Gaussian parameters and dL/dimage from their (fixed) device buffers, so a
caller updates them in place between replays. The cameras and the key capacity are fixed at
capture time: a new camera set needs a new capture.
"""
import torch

from . import fgs
from .renderer import FisheyeRenderer, gaussians_of


class GraphBatch:
    """One captured forward (+ backward) over a fixed set of views.

    gs: dict of device tensors (means, scales, quats, opacities, sh, sh_degree), updated in place
    by the caller between replays. cams_py: list of camera dicts (at most 128).
    """

    def __init__(self, gs, cams_py, bg=None, backward=True, capacity_margin=1.15,
                 device="cuda", stream=None, shape=(0, 0)):
        if len(cams_py) > fgs.MAX_VIEWS:
            raise ValueError(f"at most {fgs.MAX_VIEWS} views per batch")
        self.gs = gs
        self.cams_py = list(cams_py)
        self.bg = None if bg is None else tuple(float(v) for v in bg)
        self.backward_enabled = backward
        self.device = torch.device(device)
        self.renderer = FisheyeRenderer(self.device, capacity=1 << 20, fwd_ppt=shape[0],
                                        bwd_ppt=shape[1])
        # size the key buffers with one checked eager forward, then fix them for the capture
        fr = self.renderer.forward(gs, self.cams_py, bg=self.bg, check=True)
        need = int(fr.n_intersections.item())
        self.renderer.capacity = max(int(need * capacity_margin) + 4096,
                                     self.renderer.capacity)
        fr = self.renderer.forward(gs, self.cams_py, bg=self.bg, check=True)
        self.frame = fr
        n = int(gs["means"].shape[0])
        self.n = n
        self.cams = fr.cams
        self.ws = self.renderer._bufs["ws"]
        self.ws_bytes = fgs.fgs_workspace_size(n, self.cams, self.renderer.capacity)
        P = fgs.fgs_total_pixels(self.cams)
        self.dL_dimages = torch.zeros(3 * P, dtype=torch.float32, device=self.device)
        self.grads = {k: torch.empty_like(gs[k])
                      for k in ("means", "scales", "quats", "opacities", "sh")}
        self.g = gaussians_of(gs)
        self.stream = stream or torch.cuda.Stream(self.device)
        self.graph = torch.cuda.CUDAGraph()
        # warm the launch paths on the capture stream once, then capture
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(self.stream):
            self._calls()
        self.stream.synchronize()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._calls()
        torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def _calls(self):
        fr, cam, n, ws, wb = self.frame, self.cams, self.n, self.ws, self.ws_bytes
        cap = self.renderer.capacity
        fgs.fgs_preprocess(self.g, cam, fr.records, fr.tiles_touched)
        fgs.fgs_bin_sort(fr.records, fr.tiles_touched, n, cam, fr.keys, fr.vals, cap,
                         fr.tile_ranges, fr.n_intersections, ws, wb)
        opts = self.renderer.opts
        fgs.fgs_rasterize(fr.records, fr.vals, fr.tile_ranges, cam, self.bg, fr.images,
                          fr.final_T, fr.n_processed, ws, wb, opts=opts)
        if self.backward_enabled:
            g = self.grads
            fgs.fgs_backward(self.g, cam, fr.records, fr.tiles_touched, fr.vals, fr.tile_ranges,
                             self.bg, fr.final_T, fr.n_processed, self.dL_dimages, g["means"],
                             g["scales"], g["quats"], g["opacities"], g["sh"], ws, wb,
                             opts=opts)

    def replay(self):
        """Launch the captured graph on the current stream's device (asynchronous)."""
        self.graph.replay()

    def status(self):
        """Synchronise and return the device status word (0 = ok). FGS_ERR_CAPACITY means the
        scene now produces more intersections than the capture was sized for: recapture."""
        torch.cuda.synchronize(self.device)
        return fgs.fgs_read_status(self.ws)

    def images(self):
        return self.frame.view_images(self.cams_py)
