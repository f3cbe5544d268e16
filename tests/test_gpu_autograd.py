"""torch.autograd through the hand-written backward: a parameterised loss (log-scales through
exp, opacity logits through sigmoid, raw quaternions, two views) against the FP64 oracle's
gradient chained through the same parameterisation."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_04751_gb300 import scenes
from paper_2409_04751_gb300.autograd import render
from tests import parity

pytestmark = pytest.mark.gpu


def test_autograd_matches_oracle_chain(cuda_device):
    sc = scenes.shell_scene(5000, seed=95, sh_degree=2)
    cams = [scenes.pose_camera(128, 96, 180.0, seed=951), scenes.pose_camera(96, 96, 200.0, seed=952)]
    dev = cuda_device
    means = torch.tensor(sc["means"], device=dev, requires_grad=True)
    log_s = torch.log(torch.tensor(sc["scales"], device=dev)).requires_grad_()
    quats = torch.tensor(sc["quats"] * np.float32(1.3), device=dev, requires_grad=True)
    logit = torch.logit(torch.tensor(sc["opacities"], device=dev)).requires_grad_()
    sh = torch.tensor(sc["sh"], device=dev, requires_grad=True)
    s, o = log_s.exp(), torch.sigmoid(logit)
    imgs = render(means, s, quats, o, sh, cams, 2, bg=(0.1, 0.1, 0.1))
    rng = np.random.default_rng(96)
    Gs = [rng.normal(0, 1, tuple(im.shape)) for im in imgs]
    loss = sum((im * torch.tensor(g, device=dev, dtype=torch.float32)).sum() for im, g in zip(imgs, Gs))
    loss.backward()
    used = dict(means=sc["means"], scales=s.detach().cpu().numpy(), quats=quats.detach().cpu().numpy(),
                opacities=o.detach().cpu().numpy(), sh=sc["sh"], sh_degree=2)
    ref = None
    for c, g in zip(cams, Gs):
        G = oracle.project(used, c)
        rv = oracle.backward(G, used, c, oracle.all_pixels(c), g.transpose(1, 2, 0).reshape(-1, 3),
                             (0.1, 0.1, 0.1))
        ref = rv if ref is None else {k: ref[k] + rv[k] for k in ref}
    sv, ov = used["scales"].astype(np.float64), used["opacities"].astype(np.float64)
    want = dict(means=ref["means"], log_s=ref["scales"] * sv, quats=ref["quats"],
                logit=ref["opacities"] * ov * (1 - ov), sh=ref["sh"])
    got = dict(means=means.grad, log_s=log_s.grad, quats=quats.grad, logit=logit.grad, sh=sh.grad)
    for k in want:
        r = parity.rel_l2(got[k].cpu().numpy(), want[k])
        assert r < parity.GRAD_REL, (k, r)
    # the images themselves match the oracle
    for im, c in zip(imgs, cams):
        refi = oracle.render_image(oracle.project(used, c), c, bg=(0.1, 0.1, 0.1),
                                   impact_min=parity.IMPACT_MIN)
        parity.check_image(im.detach().cpu().numpy(), refi, "autograd")
