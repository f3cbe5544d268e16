"""GPU path for the other camera models (equisolid, stereographic and orthographic fisheye,
Sec. 3.2; equirectangular panorama, Sec. 6) against the FP64 oracle: per-record projection,
whole images and every gradient, including the near-axis region (where the closed forms of
these models have no series) and the panorama's seam and poles."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2409_04751_gb300 import fgs, scenes
from tests import parity
from tests.test_gpu_render import _grad_case, _render

pytestmark = pytest.mark.gpu

MODELS = [fgs.FGS_CAM_EQUISOLID, fgs.FGS_CAM_STEREOGRAPHIC, fgs.FGS_CAM_ORTHOGRAPHIC,
          fgs.FGS_CAM_EQUIRECTANGULAR, fgs.FGS_CAM_PINHOLE]


def _cam(model, w, h, seed, fov=None):
    if model == fgs.FGS_CAM_EQUIRECTANGULAR:
        return scenes.pose_camera(2 * h, h, 0.0, seed=seed, model=model)
    # the pinhole at 90 deg (its guard band keeps Gaussians whose mean projects within 1.3
    # times the half image)
    fov = fov or {fgs.FGS_CAM_ORTHOGRAPHIC: 170.0, fgs.FGS_CAM_PINHOLE: 90.0}.get(model, 190.0)
    return scenes.pose_camera(w, h, fov, seed=seed, model=model)


@pytest.mark.parametrize("model", MODELS)
def test_preprocess_matches_oracle(cuda_device, model):
    scene = scenes.shell_scene(20_000, seed=11 + model, sh_degree=3)
    cam = _cam(model, 640, 480, 12 + model)
    r, gs, fr = _render(scene, [cam])
    n = scene["means"].shape[0]
    rec = parity.records_np(fr.records, n)
    tt = fr.tiles_touched.cpu().numpy()
    G = oracle.project(scene, cam)
    F = oracle.F
    vis_o, vis_g = G[:, F["vis"]] > 0, tt > 0
    near = G[:, F["rmargin"]] < 1e-4
    assert np.array_equal(vis_o[~near], vis_g[~near])
    both = vis_o & vis_g
    assert both.sum() > 1000
    # FP32 positions: 2e-3 px plus a few ulps of the coordinate (records whose footprint
    # reaches the image from far outside it sit thousands of pixels from the centre)
    xy_o = G[both][:, F["xy"]:F["xy"] + 2]
    tol = 2e-3 + 5e-7 * np.abs(xy_o).max(1, keepdims=True)
    assert np.all(np.abs(rec["xy"][both] - xy_o) <= tol)
    con = G[both][:, F["conic"]:F["conic"] + 3]
    a, b, c = (G[both][:, F["cov"] + k] for k in range(3))
    tr, det = a + c, a * c - b * b
    disc = np.sqrt(np.maximum(tr * tr - 4 * det, 0))
    cond = (tr + disc) / (tr - disc)
    err = np.abs(rec["conic"][both] - con).max(1) / np.abs(con).max(1)
    assert np.all(err <= 1e-6 * cond + 1e-5), (err / (1e-6 * cond + 1e-5)).max()
    ok = both & ~near
    assert np.array_equal(rec["rect"][ok], G[ok][:, F["rect"]:F["rect"] + 4].astype(np.int32))


@pytest.mark.parametrize("model", MODELS)
def test_images_match_oracle(cuda_device, model):
    scene = scenes.shell_scene(30_000, seed=21 + model, sh_degree=3)
    cam = _cam(model, 288, 224, 121 + model)
    r, gs, fr = _render(scene, [cam], bg=(0.1, 0.2, 0.3))
    img = fr.view_images([cam])[0].cpu().numpy()
    ref = oracle.render_image(oracle.project(scene, cam), cam, bg=(0.1, 0.2, 0.3),
                              impact_min=parity.IMPACT_MIN)
    st = parity.check_image(img, ref, f"model {model}")
    assert st["flagged"] < 0.05 * st["pixels"]


@pytest.mark.parametrize("model", MODELS)
def test_gradients_match_oracle(cuda_device, model):
    scene = scenes.shell_scene(6000, seed=51 + model, sh_degree=3)
    scene["quats"] = scene["quats"] * np.float32(1.3)
    cam = _cam(model, 160, 120, 510 + model)
    g, ref = _grad_case(scene, [cam], seed=15 + model, bg=(0.2, 0.3, 0.4))
    parity.check_grads(g, ref, f"model {model}")


@pytest.mark.parametrize("model", MODELS[:3] + MODELS[4:])
def test_gradients_near_axis(cuda_device, model):
    """Gaussians within t = l_z / z < 0.3 of the optical axis and on it."""
    rng = np.random.default_rng(80 + model)
    n = 400
    z = rng.uniform(1.0, 3.0, n)
    t = np.concatenate([rng.uniform(0, 0.3, n - 3), [0.0, 1e-7, 0.299]])
    a = rng.uniform(0, 2 * math.pi, n)
    scene = scenes.shell_scene(n, seed=81 + model, sh_degree=1)
    scene["means"] = np.stack([t * z * np.cos(a), t * z * np.sin(a), z], 1).astype(np.float32)
    cam = scenes.fisheye_camera(128, 128, 120.0 if model == fgs.FGS_CAM_PINHOLE else 170.0,
                                model=model)
    g, ref = _grad_case(scene, [cam], seed=82 + model)
    parity.check_grads(g, ref, f"near-axis model {model}")


def test_panorama_seam_and_poles(cuda_device):
    """Gaussians on both sides of the longitude seam (behind the camera) and near the poles:
    the image and the gradients follow the oracle (no wrap-around, poles culled)."""
    rng = np.random.default_rng(90)
    n = 600
    lon = np.concatenate([rng.uniform(math.pi - 0.25, math.pi, n // 3),
                          rng.uniform(-math.pi, -math.pi + 0.25, n // 3),
                          rng.uniform(-math.pi, math.pi, n - 2 * (n // 3))])
    lat = np.concatenate([rng.uniform(-1.2, 1.2, 2 * (n // 3)),
                          rng.uniform(1.4, 1.55, n - 2 * (n // 3)) * rng.choice([-1, 1], n - 2 * (n // 3))])
    d = rng.uniform(1.5, 4.0, n)
    means = np.stack([d * np.cos(lat) * np.sin(lon), d * np.sin(lat), d * np.cos(lat) * np.cos(lon)], 1)
    scene = scenes.shell_scene(n, seed=91, sh_degree=2)
    scene["means"] = means.astype(np.float32)
    cam = scenes.panorama_camera(256, 128)
    r, gs, fr = _render(scene, [cam], bg=(0.3, 0.3, 0.3))
    G = oracle.project(scene, cam)
    lat_o = np.arcsin(np.abs(means[:, 1]) / np.linalg.norm(means, axis=1))
    culled = (lat_o >= math.pi / 2 - 0.05) | (scene["opacities"] < 1 / 255)
    assert np.array_equal(G[:, 0] == 0, culled)  # poles culled, only them
    assert (lat_o >= math.pi / 2 - 0.05).sum() > 20
    ref = oracle.render_image(G, cam, bg=(0.3, 0.3, 0.3), impact_min=parity.IMPACT_MIN)
    parity.check_image(fr.view_images([cam])[0].cpu().numpy(), ref, "panorama seam")
    g, refg = _grad_case(scene, [cam], seed=92, bg=(0.3, 0.3, 0.3))
    parity.check_grads(g, refg, "panorama seam")


def test_mixed_models_in_one_call(cuda_device):
    """One call over views of every model gives each view's image bit for bit as its own call."""
    scene = scenes.shell_scene(12_000, seed=95, sh_degree=3)
    cams = [_cam(m, 128, 96, 950 + m) for m in [fgs.FGS_CAM_EQUIDISTANT] + MODELS]
    r, gs, fr = _render(scene, cams, capacity=1 << 20)
    multi = [x.cpu().numpy().copy() for x in fr.view_images(cams)]
    for k, c in enumerate(cams):
        r1, gs1, f1 = _render(scene, [c])
        assert np.array_equal(f1.view_images([c])[0].cpu().numpy(), multi[k])

