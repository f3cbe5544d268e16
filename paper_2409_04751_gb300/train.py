"""Fitting Gaussians to target views (Sec. 5.1 "Optimization": the method is trained with the
loss, optimiser and hyperparameters of the renderer it plugs into - an L1 photometric loss and
Adam on the per-Gaussian parameters).

A Trainer holds the raw parameters (means, log-scales, quaternions, logit-opacities, SH), their
activated copies (exp of the log-scales, sigmoid of the logits) that the C ABI renders, Adam's
moments and a device step counter. One training step over all views is

    fgs_preprocess -> fgs_bin_sort -> fgs_rasterize -> fgs_loss_l1 -> fgs_backward
    -> fgs_adam_step

with every view of the batch in one launch per stage, captured once in a CUDA graph and
replayed: the cameras, the targets and the key capacity are fixed at capture time. When the
Gaussians grow beyond the captured key capacity, the binning reports FGS_ERR_CAPACITY, that
step's images and gradients are left out (background and zero), and `check()` recaptures with
room to spare.

The learning rates default to those of the 3DGS renderer (positions 1.6e-4, scales 5e-3,
rotations 1e-3, opacities 5e-2, colours 2.5e-3), without its position-rate decay and scene-extent
scaling; one rate serves all SH coefficients.
"""
import torch

from . import fgs
from .renderer import FisheyeRenderer, gaussians_of

DEFAULT_LR = dict(means=1.6e-4, log_scales=5e-3, quats=1e-3, logit_opacities=5e-2, sh=2.5e-3)


def raw_from_scene(scene):
    """Raw parameters (numpy) of a scene given with activated scales and opacities."""
    import numpy as np
    op = np.clip(np.asarray(scene["opacities"], np.float64), 1e-6, 1 - 1e-6)
    return dict(means=scene["means"], log_scales=np.log(scene["scales"]), quats=scene["quats"],
                logit_opacities=np.log(op / (1 - op)), sh=scene["sh"],
                sh_degree=int(scene["sh_degree"]))


class Trainer:
    def __init__(self, raw, cams_py, targets, lr=None, bg=None, device="cuda",
                 capacity_margin=1.5, beta1=0.9, beta2=0.999, eps=1e-15, graph=True):
        self.device = torch.device(device)
        dev = self.device
        f32 = lambda a: torch.as_tensor(a, dtype=torch.float32).to(dev).contiguous()
        self.raw = {k: f32(raw[k]) for k in ("means", "log_scales", "quats", "logit_opacities", "sh")}
        self.sh_degree = int(raw["sh_degree"])
        self.gs = dict(means=self.raw["means"], scales=torch.exp(self.raw["log_scales"]),
                       quats=self.raw["quats"], opacities=torch.sigmoid(self.raw["logit_opacities"]),
                       sh=self.raw["sh"], sh_degree=self.sh_degree)
        self.cams_py = list(cams_py)
        self.bg = None if bg is None else tuple(float(v) for v in bg)
        self.targets = targets.to(dev).contiguous()
        self.lr = dict(DEFAULT_LR, **(lr or {}))
        self.betas = (float(beta1), float(beta2))
        self.eps = float(eps)
        self.margin = float(capacity_margin)
        self.grads = {k: torch.zeros_like(self.gs[k])
                      for k in ("means", "scales", "quats", "opacities", "sh")}
        self.m = {k: torch.zeros_like(v) for k, v in self.raw.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.raw.items()}
        self.step_count = torch.zeros(1, dtype=torch.int64, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        A = fgs
        spec = [("means", None, "means", A.FGS_ACT_NONE),
                ("log_scales", self.gs["scales"], "scales", A.FGS_ACT_EXP),
                ("quats", None, "quats", A.FGS_ACT_NONE),
                ("logit_opacities", self.gs["opacities"], "opacities", A.FGS_ACT_SIGMOID),
                ("sh", None, "sh", A.FGS_ACT_NONE)]
        self.groups = fgs.adam_groups([dict(raw=self.raw[k], act=act, grad=self.grads[gk],
                                            m=self.m[k], v=self.v[k], activation=a, lr=self.lr[k])
                                       for k, act, gk, a in spec])
        self.use_graph = bool(graph)
        self._setup(capacity=1 << 20)

    # ------------------------------------------------------------------------------------
    def _setup(self, capacity):
        r = FisheyeRenderer(self.device, capacity=capacity)
        fr = r.forward(self.gs, self.cams_py, bg=self.bg, check=True)
        need = int(fr.n_intersections.item())
        r.capacity = max(int(need * self.margin) + 4096, r.capacity)
        self.frame = r.forward(self.gs, self.cams_py, bg=self.bg, check=True)
        self.renderer = r
        self.n = int(self.gs["means"].shape[0])
        self.cams = self.frame.cams
        self.ws = r._bufs["ws"]
        self.ws_bytes = fgs.fgs_workspace_size(self.n, self.cams, r.capacity)
        self.P = fgs.fgs_total_pixels(self.cams)
        assert self.targets.numel() == 3 * self.P, "targets: packed [3, H, W] of every view"
        self.dL = torch.zeros(3 * self.P, dtype=torch.float32, device=self.device)
        self.g = gaussians_of(self.gs)
        self.graph = None
        if self.use_graph:
            self.stream = torch.cuda.Stream(self.device)
            self.graph = torch.cuda.CUDAGraph()
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
            with torch.cuda.stream(self.stream):
                # the loss and the backward once, eagerly, so that their launch set-up happens
                # outside the capture (they change no parameter)
                self._calls(adam=False)
            self.stream.synchronize()
            # capturing launches nothing: the parameters are untouched until the first replay
            with torch.cuda.graph(self.graph, stream=self.stream):
                self._calls()
            torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def _calls(self, adam=True):
        fr, cam, n, ws, wb = self.frame, self.cams, self.n, self.ws, self.ws_bytes
        cap = self.renderer.capacity
        fgs.fgs_preprocess(self.g, cam, fr.records, fr.tiles_touched)
        fgs.fgs_bin_sort(fr.records, fr.tiles_touched, n, cam, fr.keys, fr.vals, cap,
                         fr.tile_ranges, fr.n_intersections, ws, wb)
        opts = self.renderer.opts
        fgs.fgs_rasterize(fr.records, fr.vals, fr.tile_ranges, cam, self.bg, fr.images,
                          fr.final_T, fr.n_processed, ws, wb, opts=opts)
        fgs.fgs_loss_l1(fr.images, self.targets, self.dL, 3 * self.P, 1.0 / (3 * self.P), self.loss)
        g = self.grads
        fgs.fgs_backward(self.g, cam, fr.records, fr.tiles_touched, fr.vals, fr.tile_ranges,
                         self.bg, fr.final_T, fr.n_processed, self.dL, g["means"], g["scales"],
                         g["quats"], g["opacities"], g["sh"], ws, wb, opts=opts)
        if adam:
            fgs.fgs_adam_step(self.groups, self.betas[0], self.betas[1], self.eps,
                              self.step_count)

    def step(self):
        """One training step (asynchronous)."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._calls()

    def check(self):
        """Synchronise; if the last step overflowed the key capacity, recapture with more room.
        Returns the L1 loss of the last step."""
        torch.cuda.synchronize(self.device)
        st = fgs.fgs_read_status(self.ws)
        if st == fgs.FGS_ERR_CAPACITY:
            self._setup(int(int(self.frame.n_intersections.item()) * self.margin) + 4096)
        elif st != fgs.FGS_OK:
            raise fgs.FgsError(st, "training step")
        return float(self.loss.item())

    def images(self):
        return self.frame.view_images(self.cams_py)
