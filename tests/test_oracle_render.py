"""Pins of the oracle's per-pixel blending (Sec. 3.1 "Rendering") and its backward.

Against: closed forms (one isotropic Gaussian on the axis), special cases (empty scene,
everything culled), invariants (transmittance bounds, colour bound, rotation symmetry), the
exact equality of the bounding-box candidate search with the all-Gaussian brute force, an
independent float64 torch autograd renderer on tiny scenes, and central finite differences.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_04751_gb300 import scenes

torch = pytest.importorskip("torch")
from tests import torch_brute  # noqa: E402

Y00 = 1.0 / (2.0 * math.sqrt(math.pi))


def _cam(w, h, fov, W=None, centre=(0, 0, 0)):
    return scenes.fisheye_camera(w, h, fov, W, centre)


def _one(mu, s, opac, dc):
    return dict(means=np.array([mu], np.float64), scales=np.array([[s, s, s]], np.float64),
                quats=np.array([[1.0, 0, 0, 0]]), opacities=np.array([opac]),
                sh=np.array([[[dc, dc * 0.5, -dc]]]), sh_degree=0)


def test_single_gaussian_closed_form():
    """One isotropic Gaussian on the axis: C(p) = alpha(p) rgb, T = 1 - alpha(p), with
    alpha(p) = min(0.99, o exp(-|p - c|^2 / (2 v))) kept iff >= 1/255,
    v = (f s / z)^2 + 0.3, rgb = 0.5 + Y00 sh (degree 0)."""
    cam = _cam(64, 48, 180.0)
    f, z, s = cam["fx"], 3.0, 0.08
    for opac in (0.5, 0.995):
        sc = _one([0, 0, z], s, opac, 0.9)
        G = oracle.project(sc, cam)
        im = oracle.render_image(G, cam, use_bbox=False)
        v = (f * s / z) ** 2 + 0.3
        jj, ii = np.meshgrid(np.arange(48) + 0.5, np.arange(64) + 0.5, indexing="ij")
        araw = opac * np.exp(-((ii - cam["cx"]) ** 2 + (jj - cam["cy"]) ** 2) / (2 * v))
        a = np.minimum(0.99, araw)
        a[a < 1 / 255] = 0
        rgb = 0.5 + Y00 * np.array([0.9, 0.45, -0.9])
        rgb = np.maximum(rgb, 0)
        for ch in range(3):
            assert np.allclose(im["color"][ch], a * rgb[ch], atol=1e-12)
        assert np.allclose(im["T_final"], 1 - a, atol=1e-12)
        assert np.array_equal(im["n_contrib"], (a > 0).astype(np.int32))


def test_empty_and_culled_scenes():
    cam = _cam(32, 32, 180.0)
    bg = (0.2, 0.4, 0.6)
    empty = dict(means=np.zeros((0, 3)), scales=np.zeros((0, 3)), quats=np.zeros((0, 4)),
                 opacities=np.zeros(0), sh=np.zeros((0, 1, 3)), sh_degree=0)
    culled = dict(means=np.array([[0, 0, 0.1], [0, 0, -3.0], [0.01, 0, -2.0], [0, 0, 2.0]]),
                  scales=np.full((4, 3), 0.1), quats=np.tile([1.0, 0, 0, 0], (4, 1)),
                  opacities=np.array([0.9, 0.9, 0.9, 1.0 / 256]), sh=np.zeros((4, 1, 3)),
                  sh_degree=0)
    for sc in (empty, culled):
        G = oracle.project(sc, cam)
        assert np.all(G[:, 0] == 0)
        im = oracle.render_image(G, cam, bg=bg)
        for ch in range(3):
            assert np.all(im["color"][ch] == bg[ch])
        assert np.all(im["T_final"] == 1.0) and np.all(im["last_g"] == -1)
        gr = oracle.backward(G, sc, cam, oracle.all_pixels(cam), np.ones((32 * 32, 3)), bg)
        for k in ("means", "scales", "quats", "opacities", "sh"):
            assert np.all(gr[k] == 0)


def test_config0_invariants_and_bbox_equals_brute_force():
    scene, cams = scenes.config0()
    cam = cams[0]
    G = oracle.project(scene, cam)
    bg = (0.1, 0.2, 0.3)
    a = oracle.render_image(G, cam, bg=bg, use_bbox=True)
    b = oracle.render_image(G, cam, bg=bg, use_bbox=False)
    assert np.array_equal(a["color"], b["color"]) and np.array_equal(a["last_g"], b["last_g"])
    T = a["T_final"]
    assert np.all(T >= 1e-4) and np.all(T <= 1.0)
    rgbmax = G[G[:, 0] > 0][:, oracle.F["rgb"]:oracle.F["rgb"] + 3].max()
    for ch in range(3):
        assert np.all(a["color"][ch] <= rgbmax * (1 - T) + T * bg[ch] + 1e-12)
        assert np.all(a["color"][ch] >= T * bg[ch] - 1e-12)
    assert np.all((a["n_contrib"] == 0) == (a["last_g"] == -1))


def _rotz_quat(ang):
    return np.array([math.cos(ang / 2), 0, 0, math.sin(ang / 2)])


def _qmul(a, b):
    aw, ax, ay, az = a.T
    bw, bx, by, bz = b.T
    return np.stack([aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw], -1)


def test_rotation_about_optical_axis_rotates_image():
    """Identity camera, square image, centred principal point: rotating the scene by 90 deg
    about z maps image offsets (u, v) from c to (-v, u)."""
    scene = scenes.shell_scene(3000, seed=5, sh_degree=0)
    cam = _cam(96, 96, 180.0)
    Rz = np.array([[0.0, -1, 0], [1, 0, 0], [0, 0, 1]])
    rot = dict(scene)
    rot["means"] = scene["means"].astype(np.float64) @ Rz.T
    rot["quats"] = _qmul(np.tile(_rotz_quat(math.pi / 2), (3000, 1)), scene["quats"].astype(np.float64))
    a = oracle.render_image(oracle.project(scene, cam), cam)
    b = oracle.render_image(oracle.project(rot, cam), cam)
    # b at offset (u', v') equals a at (v', -u'): b[j', i'] = a[95 - i', j']
    want = np.transpose(a["color"], (0, 2, 1))[:, :, ::-1]
    ok = (np.transpose(a["margins"], (1, 0, 2))[:, ::-1, :].min(-1) > 1e-6)
    ok &= b["margins"].min(-1) > 1e-6
    assert ok.mean() > 0.98
    assert np.abs(b["color"] - want)[:, ok].max() < 1e-9


def _tiny_scene(seed, n=6, degree=3):
    rng = np.random.default_rng(seed)
    means = np.zeros((n, 3))
    means[:, 0] = rng.uniform(-1.2, 1.2, n)
    means[:, 1] = rng.uniform(-0.9, 0.9, n)
    means[:, 2] = rng.uniform(0.8, 2.5, n)
    means[-1] = [rng.uniform(1.5, 2.5), 0.3, -0.5]  # behind the camera plane, inside 200 deg
    means[0] = [0.02, -0.03, 1.4]                   # three stacked near the axis -> T stop
    means[1] = [0.03, -0.02, 1.6]
    means[2] = [0.01, -0.01, 1.8]
    scales = np.exp(rng.normal(-1.6, 0.3, (n, 3)))
    quats = rng.normal(size=(n, 4)) * rng.uniform(0.5, 2.0, (n, 1))
    opac = rng.uniform(0.3, 0.95, n)
    opac[:3] = [0.999, 0.999, 0.97]
    K = (degree + 1) ** 2
    sh = rng.normal(0, 0.3, (n, K, 3))
    sh[:, 0, :] = rng.uniform(-1, 1, (n, 3))
    return dict(means=means, scales=scales, quats=quats, opacities=opac, sh=sh, sh_degree=degree)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_scene_matches_torch_autograd(seed):
    scene = _tiny_scene(seed)
    cam = _cam(24, 20, 200.0)
    rng = np.random.default_rng(100 + seed)
    g = rng.normal(0, 1, (3, 20, 24))
    bg = (0.05, 0.1, 0.2)
    img_t, gr_t = torch_brute.render_and_grad(scene, cam, g, bg)
    G = oracle.project(scene, cam)
    im = oracle.render_image(G, cam, bg=bg)
    assert np.abs(im["color"] - img_t).max() < 1e-12
    assert (im["T_final"] < 0.02).any()  # the stop rule is exercised
    pix = oracle.all_pixels(cam)
    dLdC = g.transpose(1, 2, 0).reshape(-1, 3)
    gr = oracle.backward(G, scene, cam, pix, dLdC, bg)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        a, b = gr[k], gr_t[k]
        assert np.abs(a - b).max() <= 1e-9 * max(1.0, np.abs(b).max()), (k, a, b)


def test_finite_differences_sampled_parameters():
    """Central differences of L = <G, C> of the oracle's own forward on 64 sampled parameters;
    samples whose contributing sets change between +-h are skipped."""
    scene = scenes.shell_scene(400, seed=9, sh_degree=3)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        scene[k] = scene[k].astype(np.float64)
    cam = scenes.pose_camera(64, 48, 180.0, seed=77)
    rng = np.random.default_rng(3)
    g = rng.normal(0, 1, (48 * 64, 3))
    pix = oracle.all_pixels(cam)
    G = oracle.project(scene, cam)
    gr = oracle.backward(G, scene, cam, pix, g)
    vis = np.nonzero(G[:, 0] > 0)[0]

    def loss(sc):
        Gs = oracle.project(sc, cam)
        r = oracle.render(Gs, pix)
        return float(np.sum(r["color"] * g)), r["n_contrib"], r["last_g"]

    checked = 0
    for t in range(64):
        key = ["means", "scales", "quats", "opacities", "sh"][t % 5]
        i = int(rng.choice(vis))
        idx = (i,) + tuple(int(rng.integers(d)) for d in scene[key].shape[1:])
        h = 1e-6 * max(1e-3, abs(scene[key][idx]))
        sp, sm = dict(scene), dict(scene)
        sp[key] = scene[key].copy()
        sm[key] = scene[key].copy()
        sp[key][idx] += h
        sm[key][idx] -= h
        lp, ncp, lgp = loss(sp)
        lm, ncm, lgm = loss(sm)
        if not (np.array_equal(ncp, ncm) and np.array_equal(lgp, lgm)):
            continue
        fd = (lp - lm) / (2 * h)
        an = gr[key][idx]
        assert abs(fd - an) <= 2e-5 * max(abs(an), 1e-2), (key, idx, fd, an)
        checked += 1
    assert checked >= 48


def test_row_prefilter_renders_the_same_pixels():
    """The sampled-pixel row prefilter of the full-size parity tests: rendering only the rows
    it keeps gives the same colour, transmittance and last index as rendering every row, on
    a box scene seen at 190 degrees (Gaussians behind the camera included)."""
    from tests import parity
    scene = scenes.box_scene(4000, seed=11, half=(3.0, 3.0, 1.0), log_scale=(-2.5, 0.6),
                             sh_degree=1)
    cam = scenes.pose_camera(192, 160, 190.0, seed=5, centre_box=(1.0, 1.0, 0.3))
    G = oracle.project(scene, cam)
    rng = np.random.default_rng(2)
    pix = np.stack([rng.integers(0, 192, 400), rng.integers(0, 160, 400)], 1).astype(np.int32)
    full = oracle.render(G, pix)
    rows = parity.rows_near_pixels(G, pix, 192, 160)
    assert 0 < rows.size < int((G[:, oracle.F["vis"]] > 0).sum())
    sub = oracle.render(G[rows], pix)
    assert np.array_equal(full["color"], sub["color"])
    assert np.array_equal(full["T_final"], sub["T_final"])
    last = np.where(sub["last_g"] >= 0, rows[np.maximum(sub["last_g"], 0)], -1)
    assert np.array_equal(full["last_g"], last)
    assert (full["n_contrib"] > 0).mean() > 0.3
