"""GPU forward (fgs_preprocess -> fgs_bin_sort -> fgs_rasterize) and backward (fgs_backward)
against the FP64 oracle on seeded synthetic scenes small enough for the oracle to render every
pixel in seconds: per-record projection, whole images, and every gradient."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2409_04751_gb300 import fgs, scenes
from paper_2409_04751_gb300.renderer import FisheyeRenderer, scene_to_device
from tests import parity

pytestmark = pytest.mark.gpu


def _render(scene, cams, bg=None, capacity=1 << 16, shape=(0, 0)):
    dev = torch.device("cuda:0")
    gs = scene_to_device(scene, dev)
    r = FisheyeRenderer(dev, capacity=capacity, fwd_ppt=shape[0], bwd_ppt=shape[1])
    fr = r.forward(gs, cams, bg=bg)
    return r, gs, fr


def _mid_scene(seed=11, n=20_000):
    return scenes.shell_scene(n, seed=seed, sh_degree=3)


def test_preprocess_matches_oracle(cuda_device):
    scene = _mid_scene()
    cam = scenes.pose_camera(640, 480, 190.0, seed=12)
    r, gs, fr = _render(scene, [cam])
    n = scene["means"].shape[0]
    rec = parity.records_np(fr.records, n)
    tt = fr.tiles_touched.cpu().numpy()
    G = oracle.project(scene, cam)
    F = oracle.F
    vis_o = G[:, F["vis"]] > 0
    vis_g = tt > 0
    # decisions on the rect / culling within rounding of their threshold may differ
    near = G[:, F["rmargin"]] < 1e-4
    assert np.array_equal(vis_o[~near], vis_g[~near])
    both = vis_o & vis_g
    xy = G[both][:, F["xy"]:F["xy"] + 2]
    assert np.abs(rec["xy"][both] - xy).max() < 2e-3
    con = G[both][:, F["conic"]:F["conic"] + 3]
    scale = np.abs(con).max(1)
    # FP32 inversion of Sigma_p loses about cond(Sigma_p) ulps
    a, b, c = (G[both][:, F["cov"] + k] for k in range(3))
    tr, det = a + c, a * c - b * b
    disc = np.sqrt(np.maximum(tr * tr - 4 * det, 0))
    cond = (tr + disc) / (tr - disc)
    err = np.abs(rec["conic"][both] - con).max(1) / scale
    assert np.all(err <= 1e-6 * cond + 1e-5), (err / (1e-6 * cond + 1e-5)).max()
    assert np.array_equal(rec["opacity"][both], scene["opacities"][both])
    assert np.abs(rec["rgb"][both] - G[both][:, F["rgb"]:F["rgb"] + 3]).max() < 2e-5
    assert (np.abs(rec["depth"][both] - G[both][:, F["depth"]]) / G[both][:, F["depth"]]).max() < 2e-6
    ok = both & ~near
    assert np.array_equal(rec["rect"][ok], G[ok][:, F["rect"]:F["rect"] + 4].astype(np.int32))
    area = (rec["rect"][:, 2] - rec["rect"][:, 0] + 1) * (rec["rect"][:, 3] - rec["rect"][:, 1] + 1)
    assert np.array_equal(tt[vis_g], area[vis_g])
    assert int(fr.n_intersections.item()) == int(tt.astype(np.int64).sum())


def test_config0_image_matches_oracle(cuda_device):
    scene, cams = scenes.config0()
    r, gs, fr = _render(scene, cams)
    img = fr.view_images(cams)[0].cpu().numpy()
    ref = oracle.render_image(oracle.project(scene, cams[0]), cams[0], impact_min=parity.IMPACT_MIN)
    st = parity.check_image(img, ref, "config0")
    assert st["flagged"] < 0.02 * st["pixels"]
    # the stop and contributor bookkeeping: final T and the last blended Gaussian
    T = fr.final_T.cpu().numpy().reshape(256, 256)
    ok = ~parity.flagged(ref["margins"])
    assert np.abs(T - ref["T_final"])[ok].max() < 1e-4
    nproc = parity.u32(fr.n_processed).reshape(256, 256)
    vals = parity.u32(fr.vals)
    ranges = parity.u32(fr.tile_ranges).reshape(-1, 2)
    jj, ii = np.nonzero(nproc > 0)
    tile = (jj // 16) * 16 + ii // 16
    last_g = vals[ranges[tile, 0] + nproc[jj, ii] - 1]
    assert np.array_equal(last_g[ok[jj, ii]], ref["last_g"][jj, ii][ok[jj, ii]])
    assert np.all(ref["last_g"][ok & (nproc == 0)] == -1)


@pytest.mark.parametrize("w,h,fov,deg,seed,bg", [
    (320, 224, 180.0, 3, 21, (0.0, 0.0, 0.0)),
    (333, 201, 200.0, 1, 22, (0.25, 0.5, 0.75)),   # ragged tiles, behind-camera Gaussians
    (200, 200, 150.0, 2, 23, (1.0, 1.0, 1.0)),
])
def test_images_match_oracle(cuda_device, w, h, fov, deg, seed, bg):
    scene = scenes.shell_scene(30_000, seed=seed, sh_degree=deg)
    cam = scenes.pose_camera(w, h, fov, seed=seed + 100)
    r, gs, fr = _render(scene, [cam], bg=bg)
    img = fr.view_images([cam])[0].cpu().numpy()
    ref = oracle.render_image(oracle.project(scene, cam), cam, bg=bg, impact_min=parity.IMPACT_MIN)
    parity.check_image(img, ref, f"{w}x{h}@{fov}")


def test_dense_scene_exercises_stop(cuda_device):
    """Many large opaque Gaussians: most pixels reach the 1e-4 stop."""
    scene = scenes.shell_scene(20_000, seed=31, log_scale=(-1.8, 0.3), sh_degree=0)
    scene["opacities"] = np.full_like(scene["opacities"], 0.97)
    cam = scenes.fisheye_camera(160, 128, 180.0)
    r, gs, fr = _render(scene, [cam], capacity=1 << 20)
    ref = oracle.render_image(oracle.project(scene, cam), cam, impact_min=parity.IMPACT_MIN)
    assert (ref["T_final"] < 1e-3).mean() > 0.5
    parity.check_image(fr.view_images([cam])[0].cpu().numpy(), ref, "dense")


def test_empty_and_culled(cuda_device):
    cam = scenes.fisheye_camera(48, 40, 180.0)
    bg = (0.1, 0.2, 0.3)
    empty = dict(means=np.zeros((0, 3)), scales=np.zeros((0, 3)), quats=np.zeros((0, 4)),
                 opacities=np.zeros(0), sh=np.zeros((0, 1, 3)), sh_degree=0)
    # near, on the singular cone, inside the cone, below the opacity cut, and visible but
    # projected 45 px outside the image (theta = 170 deg)
    culled = dict(means=np.array([[0, 0, 0.1], [0, 0, -3.0], [0.01, 0, -2.0], [0, 0, 2.0],
                                  [0.5, 0, -3.0]]),
                  scales=np.full((5, 3), 0.1), quats=np.tile([1.0, 0, 0, 0], (5, 1)),
                  opacities=np.array([0.9, 0.9, 0.9, 1.0 / 256, 0.9]), sh=np.zeros((5, 1, 3)),
                  sh_degree=0)
    for sc in (empty, culled):
        r, gs, fr = _render(sc, [cam], bg=bg)
        img = fr.view_images([cam])[0].cpu().numpy()
        for ch in range(3):
            assert np.all(img[ch] == np.float32(bg[ch]))
        assert np.all(fr.final_T.cpu().numpy() == 1.0)
        assert int(fr.n_intersections.item()) == 0
        if sc["means"].shape[0]:
            g = r.backward(gs, fr, torch.ones(3 * 48 * 40, device="cuda"))
            for k in g:
                assert torch.all(g[k] == 0)


def test_multiview_call_equals_single_view_calls(cuda_device):
    """One call over several views of uneven size gives each view's image bit for bit."""
    scene = scenes.shell_scene(15_000, seed=41, sh_degree=3)
    cams = [scenes.pose_camera(w, h, f, seed=410 + k)
            for k, (w, h, f) in enumerate([(128, 96, 180.0), (200, 200, 150.0), (64, 300, 200.0),
                                           (96, 96, 190.0)])]
    r, gs, fr = _render(scene, cams, capacity=1 << 20)
    multi = [x.cpu().numpy().copy() for x in fr.view_images(cams)]
    for k, c in enumerate(cams):
        r1, gs1, f1 = _render(scene, [c])
        assert np.array_equal(f1.view_images([c])[0].cpu().numpy(), multi[k])


def _grad_case(scene, cams, seed, bg=None, mask=None, shape=(0, 0)):
    dev = torch.device("cuda:0")
    r, gs, fr = _render(scene, cams, bg=bg, capacity=1 << 20, shape=shape)
    P = sum(c["width"] * c["height"] for c in cams)
    dL = scenes.upstream_grad((3 * P,), 1.0, seed)
    g = r.backward(gs, fr, torch.as_tensor(dL).to(dev))
    ref = None
    off = 0
    for c in cams:
        w, h = c["width"], c["height"]
        dv = dL[3 * off:3 * (off + w * h)].reshape(3, h * w).T
        G = oracle.project(scene, c)
        rv = oracle.backward(G, scene, c, oracle.all_pixels(c), dv, bg or (0, 0, 0))
        ref = rv if ref is None else {k: ref[k] + rv[k] for k in ref}
        off += w * h
    return g, ref


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_gradients_match_oracle(cuda_device, deg):
    scene = scenes.shell_scene(6000, seed=50 + deg, sh_degree=deg)
    scene["quats"] = scene["quats"] * np.float32(1.7)  # non-unit quaternions
    cam = scenes.pose_camera(160, 120, 190.0, seed=500 + deg)
    g, ref = _grad_case(scene, [cam], seed=5 + deg, bg=(0.2, 0.3, 0.4))
    parity.check_grads(g, ref, f"deg {deg}")


def test_gradients_multiview_sum(cuda_device):
    scene = scenes.shell_scene(5000, seed=60, sh_degree=3)
    cams = [scenes.pose_camera(w, h, 180.0, seed=600 + k) for k, (w, h) in enumerate([(96, 80), (128, 64), (50, 70)])]
    g, ref = _grad_case(scene, cams, seed=61)
    parity.check_grads(g, ref, "multiview")


def test_gradients_near_axis_series_region(cuda_device):
    """Gaussians within t = l_z / z < 0.3 of the optical axis (the near-axis series of h and
    dh/dl_z) and on it."""
    rng = np.random.default_rng(70)
    n = 400
    z = rng.uniform(1.0, 3.0, n)
    t = np.concatenate([rng.uniform(0, 0.3, n - 4), [0.0, 1e-7, 0.299, 0.301]])
    a = rng.uniform(0, 2 * math.pi, n)
    means = np.stack([t * z * np.cos(a), t * z * np.sin(a), z], 1).astype(np.float32)
    scene = scenes.shell_scene(n, seed=71, sh_degree=1)
    scene["means"] = means
    cam = scenes.fisheye_camera(128, 128, 180.0)
    g, ref = _grad_case(scene, [cam], seed=72)
    parity.check_grads(g, ref, "near-axis")


FWD_SHAPES = (1, 2, 4)
BWD_SHAPES = (1, 2, 4, 8)


def test_work_shapes_agree(cuda_device):
    """Every rasterizer work shape (forward 1, 2, 4 and backward 1, 2, 4, 8 pixels per thread)
    gives the same image, final T and processed counts bit for bit, and the same gradients up to
    summation order. The shapes are passed per call (each renderer its own)."""
    scene = scenes.shell_scene(20_000, seed=80, sh_degree=3)
    cam = scenes.pose_camera(300, 200, 190.0, seed=81)
    dL = torch.as_tensor(scenes.upstream_grad((3 * 300 * 200,), 1.0, 82)).cuda()
    outs = []
    for f, b in zip(FWD_SHAPES + (1,), BWD_SHAPES):
        r, gs, fr = _render(scene, [cam], capacity=1 << 20, shape=(f, b))
        g = r.backward(gs, fr, dL)
        outs.append((fr.images.cpu().numpy().copy(), fr.final_T.cpu().numpy().copy(),
                     fr.n_processed.cpu().numpy().copy(),
                     {k: v.cpu().numpy().copy() for k, v in g.items()}))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0])
        assert np.array_equal(o[1], outs[0][1])
        assert np.array_equal(o[2], outs[0][2])
        for k in o[3]:
            assert parity.rel_l2(o[3][k], outs[0][3][k]) < 1e-5, k


@pytest.fixture(scope="module")
def deg3_case():
    """The SH-degree-3 gradient case (6000 Gaussians, 160 x 120 at 190 degrees, non-unit
    quaternions, a background) with the oracle's gradient, computed once."""
    scene = scenes.shell_scene(6000, seed=53, sh_degree=3)
    scene["quats"] = scene["quats"] * np.float32(1.7)
    cam = scenes.pose_camera(160, 120, 190.0, seed=503)
    bg = (0.2, 0.3, 0.4)
    dL = scenes.upstream_grad((3 * 160 * 120,), 1.0, 8)
    G = oracle.project(scene, cam)
    ref = oracle.backward(G, scene, cam, oracle.all_pixels(cam), dL.reshape(3, -1).T, bg)
    return scene, cam, bg, dL, ref


@pytest.mark.parametrize("bwd", BWD_SHAPES)
def test_gradients_every_backward_shape_match_oracle(cuda_device, deg3_case, bwd):
    """Whole-image gradients of every backward work shape, including the one-warp-per-tile
    shape (8 pixels per thread) the benchmark's tuner picks, against the FP64 oracle."""
    scene, cam, bg, dL, ref = deg3_case
    r, gs, fr = _render(scene, [cam], bg=bg, capacity=1 << 20, shape=(1, bwd))
    g = r.backward(gs, fr, torch.as_tensor(dL).cuda())
    parity.check_grads(g, ref, f"backward shape {bwd}")


def test_calls_with_different_shapes_run_side_by_side(cuda_device):
    """The library keeps no process-wide setting: two renderers with different work shapes and
    their own workspaces, running fwd + bwd on two streams at the same time, each give exactly
    what they give alone (images bit for bit, gradients up to the order of their sums)."""
    scene = scenes.shell_scene(20_000, seed=84, sh_degree=3)
    cam = scenes.pose_camera(320, 240, 180.0, seed=85)
    dev = torch.device("cuda:0")
    gs = scene_to_device(scene, dev)
    dL = torch.as_tensor(scenes.upstream_grad((3 * 320 * 240,), 1.0, 86)).to(dev)
    shapes = [(1, 8), (4, 2)]
    rs = [FisheyeRenderer(dev, capacity=1 << 20, fwd_ppt=f, bwd_ppt=b) for f, b in shapes]
    alone = []
    for r in rs:
        fr = r.forward(gs, [cam])
        g = r.backward(gs, fr, dL)
        alone.append((fr.images.clone(), {k: v.clone() for k, v in g.items()}))
    streams = [torch.cuda.Stream(dev) for _ in rs]
    torch.cuda.synchronize()
    together = []
    for rep in range(3):
        frs = []
        for r, st in zip(rs, streams):
            with torch.cuda.stream(st):
                fr = r.forward(gs, [cam], check=False)
                frs.append((fr, r.backward(gs, fr, dL, check=False)))
        torch.cuda.synchronize()
        together.append([(fr.images.clone(), {k: v.clone() for k, v in g.items()})
                         for fr, g in frs])
        for r in rs:
            assert fgs.fgs_read_status(r._bufs["ws"]) == fgs.FGS_OK
    for run in together:
        for (img, g), (img0, g0) in zip(run, alone):
            assert torch.equal(img, img0)
            for k in g:
                assert parity.rel_l2(g[k].cpu().numpy(), g0[k].cpu().numpy()) < 1e-5, k


@pytest.mark.parametrize("shape", [(1, 1), (2, 2), (4, 8)])
def test_instrumented_launches_count_what_they_do(cuda_device, shape):
    """The measurement launches (FGS_OPT_INSTRUMENT) render the same image and count their work
    consistently: the backward's contributions are exactly the forward's blends (both passes
    take the same alpha decisions), every evaluation count bounds its blend count and every
    forward shape counts the same evaluations and blends, the backward
    stages exactly the entries up to each tile's furthest processed one, and the forward stages
    at least those and at most the tile's whole list."""
    scene, cams = scenes.config0()
    dev = cuda_device
    gs = scene_to_device(scene, dev)
    r = FisheyeRenderer(dev, capacity=1 << 16, fwd_ppt=shape[0], bwd_ppt=shape[1])
    plain = r.forward(gs, cams).images.clone()
    r.opts = fgs.options(fwd=shape[0], bwd=shape[1], instrument=True)
    fr = r.forward(gs, cams)
    assert torch.equal(fr.images, plain)
    dL = torch.as_tensor(scenes.upstream_grad((3 * 256 * 256,), 1e-2, seed=3)).to(dev)
    r.backward(gs, fr, dL)
    c = fgs.fgs_read_counters(r._bufs["ws"])
    m = int(fr.n_intersections.item())
    assert c[1] == c[3] > 0
    assert c[1] <= c[0] and c[3] <= c[2]
    # per tile: the furthest list entry any of its pixels processed (clamped to the list)
    rg = fr.tile_ranges.view(-1, 2).cpu().numpy().astype(np.int64)
    npr = fr.n_processed.view(256, 256).cpu().numpy().astype(np.int64)
    furthest = np.zeros(rg.shape[0], np.int64)
    for t in range(rg.shape[0]):
        ty, tx = divmod(t, 16)
        furthest[t] = min(npr[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16].max(), rg[t, 1] - rg[t, 0])
    assert c[5] == furthest.sum()
    assert furthest.sum() <= c[4] <= m
    # every work shape evaluates the same (pixel, entry) pairs: a live pixel, an entry kept at
    # staging, and no entry after the one that stopped the pixel
    r1 = FisheyeRenderer(dev, capacity=1 << 16, fwd_ppt=1, bwd_ppt=shape[1])
    r1.opts = fgs.options(fwd=1, bwd=shape[1], instrument=True)
    r1.forward(gs, cams)
    c1 = fgs.fgs_read_counters(r1._bufs["ws"])
    assert c[0] == c1[0] and c[1] == c1[1]
