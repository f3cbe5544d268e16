"""Parity at the full benchmark workload (500k Gaussians, SH degree 3, one 1752x1168 view at
180 degrees, random pose), in the launch configuration the benchmark times (its rasterizer work
shapes are 4 pixels per thread forward and 8 backward, the library's defaults, which its tuner
confirms; every other shape is covered too): sampled pixels rendered one by one by the oracle,
the gradient of the loss restricted to those pixels, and properties of the sorted keys that hold
at any size."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_04751_gb300 import scenes
from paper_2409_04751_gb300.renderer import FisheyeRenderer, scene_to_device
from tests import parity

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def cfg1():
    scene, cams = scenes.config1()
    dev = torch.device("cuda:0")
    gs = scene_to_device(scene, dev)
    r = FisheyeRenderer(dev, capacity=24_000_000, fwd_ppt=BENCH_SHAPE[0], bwd_ppt=BENCH_SHAPE[1])
    fr = r.forward(gs, cams)
    G = oracle.project(scene, cams[0])
    return scene, cams, gs, r, fr, G


BENCH_SHAPE = (4, 8)  # pixels per thread of the forward and backward rasterizers


def test_config1_sampled_pixels(cfg1):
    scene, cams, gs, r, fr, G = cfg1
    cam = cams[0]
    w, h = cam["width"], cam["height"]
    rng = np.random.default_rng(123)
    pix = np.stack([rng.integers(0, w, 3000), rng.integers(0, h, 3000)], 1).astype(np.int32)
    ref = oracle.render(G, pix, impact_min=parity.IMPACT_MIN)
    img = fr.view_images(cams)[0].cpu().numpy()
    got = img[:, pix[:, 1], pix[:, 0]].T
    d = np.abs(got - ref["color"])
    fl = parity.flagged(ref["margins"])
    assert fl.mean() < 0.08, (fl.mean(), d[~fl].max(), d.mean(0))
    assert d[~fl].max() <= parity.IMG_MAX
    assert np.all(d.mean(0) <= parity.IMG_MEAN)


def test_config1_keys_properties(cfg1):
    """Sorted keys are non-decreasing, each tile's range holds exactly its keys, and the
    (key, value) multiset is the one the records define (count per record = rect area, tile
    ids inside the rect, low word = the record's depth bits)."""
    scene, cams, gs, r, fr, G = cfg1
    n = scene["means"].shape[0]
    m = int(fr.n_intersections.item())
    keys = parity.u64(fr.keys)[:m]
    vals = parity.u32(fr.vals)[:m]
    assert m > 5_000_000
    assert np.all(keys[1:] >= keys[:-1])
    same = keys[1:] == keys[:-1]
    assert np.all(vals[1:][same] > vals[:-1][same])  # stable: equal keys in record order
    rec = parity.records_np(fr.records, n)
    tt = fr.tiles_touched.cpu().numpy().astype(np.int64)
    assert np.array_equal(np.bincount(vals, minlength=n), tt)
    assert np.array_equal((keys & np.uint64(0xFFFFFFFF)).astype(np.uint32), rec["depth_bits"][vals])
    tile = (keys >> np.uint64(32)).astype(np.int64)
    tx, ty = tile % 110, tile // 110
    rc = rec["rect"][vals]
    assert np.all((tx >= rc[:, 0]) & (tx <= rc[:, 2]) & (ty >= rc[:, 1]) & (ty <= rc[:, 3]))
    ranges = parity.u32(fr.tile_ranges).reshape(-1, 2).astype(np.int64)
    cnt = np.bincount(tile, minlength=ranges.shape[0])
    assert np.array_equal(ranges[:, 1] - ranges[:, 0], cnt)
    # GPU rects against the oracle's FP64 rects, except rounding-near boundaries
    F = oracle.F
    vis = G[:, F["vis"]] > 0
    near = G[:, F["rmargin"]] < 1e-4
    ok = vis & (tt > 0) & ~near
    assert np.array_equal(rec["rect"][ok], G[ok][:, F["rect"]:F["rect"] + 4].astype(np.int32))
    assert np.array_equal(vis[~near], (tt > 0)[~near])


@pytest.fixture(scope="module")
def cfg1_grad(cfg1):
    """dL/dimage nonzero only on 1500 sampled pixels, and the oracle's gradient of that
    restricted loss (computed once)."""
    scene, cams, gs, r, fr, G = cfg1
    cam = cams[0]
    w, h = cam["width"], cam["height"]
    rng = np.random.default_rng(321)
    idx = rng.choice(w * h, 1500, replace=False)
    pix = np.stack([idx % w, idx // w], 1).astype(np.int32)
    gvals = rng.normal(0, 1e-2, (1500, 3))
    dL = np.zeros((3, h * w), np.float32)
    dL[:, idx] = gvals.T.astype(np.float32)
    ref = oracle.backward(G, scene, cam, pix, dL[:, idx].T.astype(np.float64))
    return torch.as_tensor(dL.reshape(-1)).cuda(), ref


@pytest.mark.parametrize("bwd", [8, 1, 2, 4])
def test_config1_sampled_gradient(cfg1, cfg1_grad, bwd):
    """Every gradient tensor against the oracle's gradient of the restricted loss, for the
    benchmark's backward shape (8 pixels per thread) and every other one."""
    scene, cams, gs, r, fr, G = cfg1
    dL, ref = cfg1_grad
    r2 = FisheyeRenderer(r.device, capacity=r.capacity, fwd_ppt=BENCH_SHAPE[0], bwd_ppt=bwd)
    r2._bufs = r._bufs  # the same frame and workspace
    g = r2.backward(gs, fr, dL)
    parity.check_grads(g, ref, f"config1 sampled, backward shape {bwd}")


@pytest.mark.parametrize("fwd", [1, 2])
def test_config1_forward_shapes_identical(cfg1, fwd):
    """The other forward work shapes give the benchmark shape's image, final T and processed
    counts bit for bit at full size."""
    scene, cams, gs, r, fr, G = cfg1
    img0, T0, n0 = fr.images.clone(), fr.final_T.clone(), fr.n_processed.clone()
    r2 = FisheyeRenderer(r.device, capacity=r.capacity, fwd_ppt=fwd, bwd_ppt=BENCH_SHAPE[1])
    f2 = r2.forward(gs, cams)
    assert torch.equal(f2.images, img0) and torch.equal(f2.final_T, T0)
    assert torch.equal(f2.n_processed, n0)


# ------------------------------------------------------------------------------------------
# Large scene: 3M Gaussians in a 20 x 20 x 5 box, SH degree 3, 2048 x 2048 at 190 degrees
# (theta up to 95 degrees), poses inside the box; single-view forward, as its throughput
# benchmark launches it.

@pytest.fixture(scope="module")
def cfg2():
    scene, cams = scenes.config2(n_poses=3)
    dev = torch.device("cuda:0")
    gs = scene_to_device(scene, dev)
    r = FisheyeRenderer(dev, capacity=32_000_000)
    return scene, cams, gs, r


@pytest.mark.parametrize("pose", [0, 2])
def test_config2_sampled_pixels_and_keys(cfg2, pose):
    scene, cams, gs, r = cfg2
    cam = cams[pose]
    n = scene["means"].shape[0]
    fr = r.forward(gs, [cam])
    w, h = cam["width"], cam["height"]
    rng = np.random.default_rng(77 + pose)
    pix = np.stack([rng.integers(0, w, 2500), rng.integers(0, h, 2500)], 1).astype(np.int32)
    G = oracle.project(scene, cam)
    rows = parity.rows_near_pixels(G, pix, w, h)
    ref = oracle.render(G[rows], pix, impact_min=parity.IMPACT_MIN)
    img = fr.view_images([cam])[0].cpu().numpy()
    got = img[:, pix[:, 1], pix[:, 0]].T
    d = np.abs(got - ref["color"])
    fl = parity.flagged(ref["margins"])
    assert (ref["n_contrib"] > 0).mean() > 0.5  # the sample sees the scene
    assert fl.mean() < 0.08, (fl.mean(), d[~fl].max(), d.mean(0))
    assert d[~fl].max() <= parity.IMG_MAX
    assert np.all(d.mean(0) <= parity.IMG_MEAN)
    Tg = fr.final_T.view(h, w).cpu().numpy()[pix[:, 1], pix[:, 0]]
    assert np.abs(Tg - ref["T_final"])[~fl].max() <= parity.IMG_MAX

    # keys: sorted, stable, each record's pair count = its rect area, ranges consistent
    m = int(fr.n_intersections.item())
    keys = parity.u64(fr.keys)[:m]
    vals = parity.u32(fr.vals)[:m]
    assert m > 1_000_000
    assert np.all(keys[1:] >= keys[:-1])
    same = keys[1:] == keys[:-1]
    assert np.all(vals[1:][same] > vals[:-1][same])
    rec = parity.records_np(fr.records, n)
    tt = fr.tiles_touched.cpu().numpy().astype(np.int64)
    assert np.array_equal(np.bincount(vals, minlength=n), tt)
    rc = rec["rect"]
    area = np.where(tt > 0, (rc[:, 2] - rc[:, 0] + 1) * (rc[:, 3] - rc[:, 1] + 1), 0)
    assert np.array_equal(area, tt)
    assert np.array_equal((keys & np.uint64(0xFFFFFFFF)).astype(np.uint32), rec["depth_bits"][vals])
    tile = (keys >> np.uint64(32)).astype(np.int64)
    ranges = parity.u32(fr.tile_ranges).reshape(-1, 2).astype(np.int64)
    assert ranges.shape[0] == 128 * 128
    assert np.array_equal(ranges[:, 1] - ranges[:, 0], np.bincount(tile, minlength=128 * 128))
    # visibility and rects against the oracle's FP64 decisions away from rounding boundaries
    F = oracle.F
    vis = G[:, F["vis"]] > 0
    near = G[:, F["rmargin"]] < 1e-4
    ok = vis & (tt > 0) & ~near
    assert np.array_equal(rc[ok], G[ok][:, F["rect"]:F["rect"] + 4].astype(np.int32))
    assert np.array_equal(vis[~near], (tt > 0)[~near])
