"""torch.autograd.Function around the C ABI: differentiable fisheye rendering.

render(means, scales, quats, opacities, sh, cams, ...) returns one [3, H, W] image per camera;
backpropagating through them runs fgs_backward (the hand-written backward kernels). The
gradients are those of the ABI inputs as passed (activated scales and opacities, raw
quaternions); callers compose exp / sigmoid / any parameterisation with ordinary torch ops
before the call and autograd chains through them.

Renderers (their device buffers and key capacity) are kept in a per-device pool: a render takes
one, its backward gives it back, so a training loop reuses the same buffers step after step.
check=True (the default) reads the binning's status after the forward - one host
synchronisation - and re-runs the binning with larger key buffers if they overflowed. With
check=False nothing synchronises; the pool's capacity is the largest seen so far, and an
overflow is reported by last_status() (FGS_ERR_CAPACITY; that frame's image is the background
and its gradients zero) after which the next checked call grows the buffers.
"""
import threading

import torch

from . import fgs
from .renderer import FisheyeRenderer

_lock = threading.Lock()
_pool = {}       # device -> list of idle renderers
_capacity = {}   # device -> largest key capacity seen
_last = {}       # device -> (renderer, frame) of the latest unchecked forward


def _take(device):
    with _lock:
        free = _pool.setdefault(device, [])
        r = free.pop() if free else FisheyeRenderer(device, capacity=_capacity.get(device, 1 << 20))
        r.capacity = max(r.capacity, _capacity.get(device, 0))
        return r


def _give(device, r):
    with _lock:
        _capacity[device] = max(_capacity.get(device, 0), r.capacity)
        _pool.setdefault(device, []).append(r)


def last_status(device=None):
    """Synchronises and returns the binning status of the latest render(check=False) on the
    device (fgs.FGS_OK, or FGS_ERR_CAPACITY when its key buffers overflowed)."""
    device = torch.device(device or "cuda")
    entry = _last.get(device)
    if entry is None:
        return fgs.FGS_OK
    r, _ = entry
    ws = r._bufs.get("ws")
    if ws is None:
        return fgs.FGS_OK
    st = fgs.fgs_read_status(ws)
    if st == fgs.FGS_ERR_CAPACITY:
        with _lock:
            need = int(r._bufs["nint"].item())
            _capacity[device] = max(_capacity.get(device, 0), int(need * r.growth) + 1024)
    return st


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, opacities, sh, cams, sh_degree, bg, check):
        gs = dict(means=means.detach().contiguous(), scales=scales.detach().contiguous(),
                  quats=quats.detach().contiguous(), opacities=opacities.detach().contiguous(),
                  sh=sh.detach().contiguous(), sh_degree=int(sh_degree))
        dev = means.device
        r = _take(dev)  # its buffers stay with this frame until the backward gives them back
        frame = r.forward(gs, cams, bg=bg, check=check)
        if not check:
            _last[dev] = (r, frame)
        ctx.state = (r, gs, frame, dev)
        ctx.sh_shape = sh.shape
        return frame.images[:3 * frame.final_T.numel()].clone()

    @staticmethod
    def backward(ctx, dL_dimages):
        r, gs, frame, dev = ctx.state
        grads = r.backward(gs, frame, dL_dimages.contiguous(), check=False)
        ctx.state = None
        _give(dev, r)
        return (grads["means"], grads["scales"], grads["quats"], grads["opacities"],
                grads["sh"].view(ctx.sh_shape), None, None, None, None)


def render(means, scales, quats, opacities, sh, cams, sh_degree, bg=None, check=True):
    """Differentiable render of `cams` (list of camera dicts). Returns a list of [3, H, W]."""
    packed = _Render.apply(means, scales, quats, opacities, sh, list(cams), int(sh_degree),
                           None if bg is None else tuple(float(v) for v in bg), bool(check))
    out, off = [], 0
    for c in cams:
        w, h = int(c["width"]), int(c["height"])
        out.append(packed[3 * off:3 * (off + w * h)].view(3, h, w))
        off += w * h
    return out
