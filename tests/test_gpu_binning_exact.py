"""The exact (ellipse) binning of fgs_bin_sort_ex on the GPU: the kept pairs against the
oracle's exact binning on the same records (bit for bit away from the margin, and within the
rect pairs everywhere), sorted order and tile ranges; images, transmittances and gradients equal
to those of the rect binning; the capacity contract."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_04751_gb300 import fgs, scenes
from paper_2409_04751_gb300.renderer import FisheyeRenderer, scene_to_device
from tests import parity

pytestmark = pytest.mark.gpu


def _frame(scene, cam, binning, capacity=1 << 21):
    dev = torch.device("cuda:0")
    gs = scene_to_device(scene, dev)
    r = FisheyeRenderer(dev, capacity=capacity, binning=binning)
    fr = r.forward(gs, [cam], bg=(0.1, 0.2, 0.3))
    return r, gs, fr


@pytest.mark.parametrize("model,fov,seed", [(fgs.FGS_CAM_EQUIDISTANT, 180.0, 1),
                                            (fgs.FGS_CAM_EQUIDISTANT, 200.0, 2),
                                            (fgs.FGS_CAM_PINHOLE, 90.0, 3)])
def test_exact_pairs_match_oracle(cuda_device, model, fov, seed):
    scene = scenes.shell_scene(40_000, seed=seed, sh_degree=1)
    cam = scenes.pose_camera(416, 304, fov, seed=100 + seed, model=model)
    r, gs, fr = _frame(scene, cam, "ellipse")
    n = scene["means"].shape[0]
    rec = parity.records_np(fr.records, n)
    tt = fr.tiles_touched.cpu().numpy()
    m = int(fr.n_intersections.item())
    keys = parity.u64(fr.keys)[:m]
    vals = parity.u32(fr.vals)[:m]
    ranges = parity.u32(fr.tile_ranges).reshape(-1, 2)
    vis = tt > 0
    rect = np.where(vis[:, None], rec["rect"], -1).astype(np.int32)
    opac = rec["opacity"].astype(np.float64)
    qs = np.maximum(2.0 * np.log(255.0 * np.maximum(opac, 1e-30)), 0.0)
    ell = np.concatenate([rec["xy"].astype(np.float64), rec["conic"].astype(np.float64),
                          qs[:, None]], 1)
    tx, ty = (cam["width"] + 15) // 16, (cam["height"] + 15) // 16
    view = np.zeros(n, np.int32)
    db = rec["depth"].astype(np.float32).view(np.uint32)
    k_o, v_o, _ = oracle.build_keys(view, rect, db, [0], [tx], tx * ty, ellipse=ell)
    k_r, v_r, _ = oracle.build_keys(view, rect, db, [0], [tx], tx * ty)
    assert len(k_o) < 0.9 * len(k_r)
    # sorted by key, equal keys by record
    assert np.all(np.diff(keys.astype(np.float64)) >= 0)
    same = keys[1:] == keys[:-1]
    assert np.all(vals[1:][same] > vals[:-1][same])
    # every GPU pair is a rect pair; pairs on which the two sides disagree sit at the margin
    gpu = set(zip(keys.tolist(), vals.tolist()))
    orc = set(zip(k_o.tolist(), v_o.tolist()))
    assert gpu <= set(zip(k_r.tolist(), v_r.tolist()))
    for (k, v) in gpu ^ orc:
        t = k >> 32
        x0, y0 = (t % tx) * 16 + 0.5, (t // tx) * 16 + 0.5
        q = oracle.rect_min_q(ell[v, :2], ell[v, 2:5], x0, x0 + 15, y0, y0 + 15)
        thr = ell[v, 5] * 1.001 + 1e-2
        assert abs(q - thr) <= 1e-4 * thr, (k, v, q, thr)
    assert len(gpu ^ orc) <= 1e-3 * len(orc) + 2
    # tile ranges
    t_of = (keys >> np.uint64(32)).astype(np.int64)
    for t in np.unique(t_of):
        s, e = ranges[t]
        assert np.all(t_of[s:e] == t) and (s == 0 or t_of[s - 1] != t)


def test_exact_binning_renders_the_same(cuda_device):
    scene = scenes.shell_scene(60_000, seed=7, sh_degree=3)
    cam = scenes.pose_camera(480, 352, 190.0, seed=70)
    r1, gs1, f1 = _frame(scene, cam, "rect")
    r2, gs2, f2 = _frame(scene, cam, "ellipse")
    n1, n2 = int(f1.n_intersections.item()), int(f2.n_intersections.item())
    assert n2 < 0.9 * n1
    assert torch.equal(f1.images, f2.images)
    assert torch.equal(f1.final_T, f2.final_T)
    P = cam["width"] * cam["height"]
    dL = torch.as_tensor(scenes.upstream_grad((3 * P,), 1.0, 71)).cuda()
    g1 = r1.backward(gs1, f1, dL)
    g2 = r2.backward(gs2, f2, dL)
    for k in g1:
        assert parity.rel_l2(g2[k].cpu().numpy(), g1[k].cpu().numpy()) < 1e-5, k


def test_exact_binning_capacity_contract(cuda_device):
    scene = scenes.shell_scene(20_000, seed=8, sh_degree=0)
    cam = scenes.pose_camera(256, 256, 180.0, seed=80)
    dev = torch.device("cuda:0")
    gs = scene_to_device(scene, dev)
    r = FisheyeRenderer(dev, capacity=1 << 21, binning="ellipse")
    fr = r.forward(gs, [cam])
    kept = int(fr.n_intersections.item())
    cand = int(fr.tiles_touched.to(torch.int64).sum().item())
    assert kept < cand
    # capacity between the kept and the candidate counts: the candidates must fit
    r2 = FisheyeRenderer(dev, capacity=(kept + cand) // 2, binning="ellipse")
    fr2 = r2.forward(gs, [cam], check=False)
    assert fgs.fgs_read_status(r2._bufs["ws"]) == fgs.FGS_ERR_CAPACITY
    assert int(fr2.n_intersections.item()) == cand
    # the renderer grows the buffers and gets the same frame
    fr3 = r2.forward(gs, [cam], check=True)
    assert int(fr3.n_intersections.item()) == kept
    assert torch.equal(fr3.images, fr.images)
