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


def test_renders_reuse_pooled_buffers_and_unchecked_renders_agree(cuda_device):
    """A training loop's renders take their buffers from the pool and give them back in the
    backward, so steps reuse the same device buffers; frames alive at the same time get
    separate buffers; a render without the host-synchronising check gives the checked result."""
    from paper_2409_04751_gb300 import autograd as ag, fgs
    sc = scenes.shell_scene(4000, seed=97, sh_degree=1)
    cam = [scenes.pose_camera(96, 80, 180.0, seed=971)]
    dev = cuda_device
    p = [torch.tensor(sc[k], device=dev, requires_grad=True)
         for k in ("means", "scales", "quats", "opacities", "sh")]
    ag._pool.pop(dev, None)
    grads = []
    for step in range(3):
        for t in p:
            t.grad = None
        img = ag.render(*p, cam, 1, check=(step == 0))[0]
        img.sum().backward()
        grads.append([t.grad.clone() for t in p])
    assert ag.last_status(dev) == fgs.FGS_OK
    assert len(ag._pool[dev]) == 1  # one renderer, reused by every step
    for g in grads[1:]:
        for a, b in zip(g, grads[0]):
            assert parity.rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-5
    # two frames alive together hold two renderers
    a = ag.render(*p, cam, 1)[0]
    b = ag.render(*p, cam, 1)[0]
    assert torch.equal(a, b)
    (a.sum() + b.sum()).backward()
    assert len(ag._pool[dev]) == 2
