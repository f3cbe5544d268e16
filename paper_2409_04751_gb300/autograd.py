"""torch.autograd.Function around the C ABI: differentiable fisheye rendering.

render(means, scales, quats, opacities, sh, cams, ...) returns one [3, H, W] image per camera;
backpropagating through them runs fgs_backward (the hand-written backward kernels). The
gradients are those of the ABI inputs as passed (activated scales and opacities, raw
quaternions); callers compose exp / sigmoid / any parameterisation with ordinary torch ops
before the call and autograd chains through them.
"""
import torch

from .renderer import FisheyeRenderer

_capacity_hint = {"cap": 1 << 20}


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, opacities, sh, cams, sh_degree, bg):
        gs = dict(means=means.detach().contiguous(), scales=scales.detach().contiguous(),
                  quats=quats.detach().contiguous(), opacities=opacities.detach().contiguous(),
                  sh=sh.detach().contiguous(), sh_degree=int(sh_degree))
        # buffers owned by this call, kept alive until the backward
        r = FisheyeRenderer(means.device, capacity=_capacity_hint["cap"])
        frame = r.forward(gs, cams, bg=bg, check=True)
        _capacity_hint["cap"] = max(_capacity_hint["cap"], r.capacity)
        ctx.state = (r, gs, frame)
        ctx.sh_shape = sh.shape
        return frame.images[:3 * frame.final_T.numel()].clone()

    @staticmethod
    def backward(ctx, dL_dimages):
        r, gs, frame = ctx.state
        grads = r.backward(gs, frame, dL_dimages.contiguous())
        ctx.state = None
        return (grads["means"], grads["scales"], grads["quats"], grads["opacities"],
                grads["sh"].view(ctx.sh_shape), None, None, None)


def render(means, scales, quats, opacities, sh, cams, sh_degree, bg=None):
    """Differentiable render of `cams` (list of camera dicts). Returns a list of [3, H, W]."""
    packed = _Render.apply(means, scales, quats, opacities, sh, list(cams), int(sh_degree),
                           None if bg is None else tuple(float(v) for v in bg))
    out, off = [], 0
    for c in cams:
        w, h = int(c["width"]), int(c["height"])
        out.append(packed[3 * off:3 * (off + w * h)].view(3, h, w))
        off += w * h
    return out
