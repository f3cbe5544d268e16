"""Training pieces on the GPU (fgs_loss_l1, fgs_adam_step) against the oracle's NumPy
statements, and the graph-captured training loop: it fits perturbed Gaussians back towards
target views, and a graph replay does what the eager call sequence does."""
import numpy as np
import pytest
import torch

from oracle import optim
from paper_2409_04751_gb300 import fgs, scenes
from paper_2409_04751_gb300.renderer import FisheyeRenderer, scene_to_device
from paper_2409_04751_gb300.train import Trainer, raw_from_scene

pytestmark = pytest.mark.gpu


def test_adam_step_matches_oracle(cuda_device):
    rng = np.random.default_rng(0)
    acts = [optim.ACT_NONE, optim.ACT_EXP, optim.ACT_SIGMOID]
    sizes = [1, 1000, 12345]
    lrs = [1e-2, 5e-3, 5e-2]
    raw = [rng.normal(size=s) for s in sizes]
    ref = [dict(raw=r.copy(), m=np.zeros_like(r), v=np.zeros_like(r)) for r in raw]
    dev = torch.device("cuda:0")
    T = lambda a: torch.as_tensor(np.asarray(a, np.float32)).to(dev)
    st = [dict(raw=T(r), act=T(np.zeros_like(r)), grad=T(np.zeros_like(r)), m=T(np.zeros_like(r)),
               v=T(np.zeros_like(r))) for r in raw]
    groups = fgs.adam_groups([dict(st[k], activation=acts[k], lr=lrs[k]) for k in range(3)])
    step = torch.zeros(1, dtype=torch.int64, device=dev)
    for t in range(1, 5):
        for k in range(3):
            g = rng.normal(size=sizes[k])
            st[k]["grad"].copy_(T(g))
            # the oracle takes the FP32 raw values the GPU holds
            rr = st[k]["raw"].cpu().numpy().astype(np.float64)
            ref[k]["raw"], act, ref[k]["m"], ref[k]["v"] = optim.adam_step(
                rr, g.astype(np.float32).astype(np.float64), ref[k]["m"], ref[k]["v"], acts[k],
                lrs[k], 0.9, 0.999, 1e-8, t)
            ref[k]["act"] = act
        fgs.fgs_adam_step(groups, 0.9, 0.999, 1e-8, step)
        torch.cuda.synchronize()
        assert int(step.item()) == t
        for k in range(3):
            got = {n: st[k][n].cpu().numpy().astype(np.float64) for n in ("raw", "m", "v", "act")}
            assert np.allclose(got["m"], ref[k]["m"], rtol=1e-5, atol=1e-7)
            assert np.allclose(got["v"], ref[k]["v"], rtol=1e-5, atol=1e-9)
            assert np.allclose(got["raw"], ref[k]["raw"], rtol=1e-6, atol=2e-6 * lrs[k])
            if acts[k] != optim.ACT_NONE:
                assert np.allclose(got["act"], ref[k]["act"], rtol=2e-6, atol=1e-7)


def test_loss_l1_matches_oracle(cuda_device):
    rng = np.random.default_rng(1)
    n = 3 * 333 * 211
    img = rng.uniform(0, 1, n).astype(np.float32)
    tgt = rng.uniform(0, 1, n).astype(np.float32)
    tgt[:1000] = img[:1000]  # ties: zero gradient
    dev = torch.device("cuda:0")
    dL = torch.empty(n, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    fgs.fgs_loss_l1(torch.as_tensor(img).to(dev), torch.as_tensor(tgt).to(dev), dL, n, 1.0 / n, loss)
    L, g = optim.loss_l1(img.astype(np.float64), tgt.astype(np.float64), 1.0 / n)
    assert abs(float(loss.item()) - L) < 1e-5 * L
    assert np.array_equal(dL.cpu().numpy(), g.astype(np.float32))


def _fit_setup(seed=5, n=3000):
    scene = scenes.shell_scene(n, seed=seed, sh_degree=1)
    cams = [scenes.pose_camera(128, 96, 180.0, seed=50 + k) for k in range(4)]
    dev = torch.device("cuda:0")
    r = FisheyeRenderer(dev, capacity=1 << 20)
    targets = r.forward(scene_to_device(scene, dev), cams).images.clone()
    rng = np.random.default_rng(seed + 1)
    raw = raw_from_scene(scene)
    raw["means"] = raw["means"] + rng.normal(0, 0.01, raw["means"].shape)
    raw["log_scales"] = raw["log_scales"] + 0.3
    raw["logit_opacities"] = raw["logit_opacities"] - 0.5
    raw["sh"] = raw["sh"] + rng.normal(0, 0.1, raw["sh"].shape)
    return raw, cams, targets


def test_trainer_reduces_the_loss(cuda_device):
    raw, cams, targets = _fit_setup()
    tr = Trainer(raw, cams, targets)
    tr.step()
    first = tr.check()
    for k in range(200):
        tr.step()
        if k % 50 == 49:
            tr.check()
    last = tr.check()
    assert last < 0.5 * first, (first, last)
    assert int(tr.step_count.item()) == 201


def test_trainer_graph_equals_eager(cuda_device):
    raw, cams, targets = _fit_setup(seed=7, n=1500)
    a = Trainer(raw, cams, targets, graph=True)
    b = Trainer(raw, cams, targets, graph=False)
    for _ in range(3):
        a.step()
        b.step()
    la, lb = a.check(), b.check()
    assert abs(la - lb) <= 1e-5 * max(la, 1e-6)
    for k in a.raw:
        x, y = a.raw[k].cpu().numpy(), b.raw[k].cpu().numpy()
        assert np.allclose(x, y, rtol=1e-4, atol=1e-5), k
