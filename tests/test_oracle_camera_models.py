"""Pins of the oracle's other camera models: the radial fisheye models Sec. 3.2 names
(equisolid, stereographic, orthographic; r_d = f r(theta)), the pinhole camera the method is
compared with (r = tan(theta)), and the equirectangular panorama of Sec. 6 ("Extension to
Other Camera Models").

What pins them, other than the oracle itself:
  * projections at special angles, against values of r(theta) known in closed form
    (sin 30 deg = 1/2, tan 45 deg = 1, sin 60 deg = sqrt(3)/2, ...);
  * the pinhole limit on the optical axis, shared by every radial model;
  * J against central finite differences of the projection and dJ/dmu_c against central
    finite differences of J (a dropped term, sign or index fails them);
  * whole images and every gradient against the independent torch autograd renderer, whose
    J is autograd's Jacobian of the model's projection.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_04751_gb300 import scenes

torch = pytest.importorskip("torch")
from tests import torch_brute  # noqa: E402

RADIAL = [oracle.CAM_EQUIDISTANT, oracle.CAM_EQUISOLID, oracle.CAM_STEREOGRAPHIC,
          oracle.CAM_ORTHOGRAPHIC, oracle.CAM_PINHOLE]
ALL = RADIAL + [oracle.CAM_EQUIRECT]

# r(theta) at 60 and 90 degrees, from the special values of sin and tan
R_SPECIAL = {
    oracle.CAM_EQUIDISTANT: {60: math.pi / 3, 90: math.pi / 2},
    oracle.CAM_EQUISOLID: {60: 1.0, 90: math.sqrt(2.0)},            # 2 sin 30, 2 sin 45
    oracle.CAM_STEREOGRAPHIC: {60: 2.0 / math.sqrt(3.0), 90: 2.0},  # 2 tan 30, 2 tan 45
    oracle.CAM_ORTHOGRAPHIC: {60: math.sqrt(3.0) / 2.0, 90: 1.0},   # sin 60, sin 90
    oracle.CAM_PINHOLE: {30: 1.0 / math.sqrt(3.0), 60: math.sqrt(3.0)},  # tan 30, tan 60
}


@pytest.mark.parametrize("model", RADIAL)
def test_radial_projection_at_special_angles(model):
    f, cx, cy = 310.0, 400.0, 300.0
    for deg, r in R_SPECIAL[model].items():
        th = math.radians(deg)
        for az in (0.0, math.radians(45.0), math.radians(200.0)):
            for d in (0.7, 3.1):
                muc = d * np.array([math.sin(th) * math.cos(az), math.sin(th) * math.sin(az),
                                    math.cos(th)])
                xy = oracle.project_point(muc, f, f, cx, cy, model)
                assert abs(xy[0] - (cx + f * r * math.cos(az))) < 1e-9 * f
                assert abs(xy[1] - (cy + f * r * math.sin(az))) < 1e-9 * f


def test_panorama_projection_at_special_points():
    w, h = 1024.0, 512.0
    fx, fy, cx, cy = w / (2 * math.pi), h / math.pi, w / 2, h / 2
    cases = [((0, 0, 2), (w / 2, h / 2)), ((1.5, 0, 0), (3 * w / 4, h / 2)),
             ((-1.5, 0, 0), (w / 4, h / 2)), ((0, -1, 1), (w / 2, h / 4)),
             ((0, 0, -1), (w, h / 2)), ((1, 1, 0), (3 * w / 4, 3 * h / 4)),
             ((0, 0.5, -math.sqrt(0.75)), (w, h / 2 + h / 6))]
    for muc, want in cases:
        xy = oracle.project_point(np.array(muc, np.float64), fx, fy, cx, cy, oracle.CAM_EQUIRECT)
        assert np.allclose(xy, want, atol=1e-9 * w), (muc, xy, want)


@pytest.mark.parametrize("model", RADIAL)
def test_radial_models_are_pinhole_on_the_axis(model):
    f = 250.0
    for z in (0.5, 4.0):
        J = oracle.jacobian([0.0, 0.0, z], f, f, model)
        assert np.allclose(J, [[f / z, 0, 0], [0, f / z, 0]], atol=1e-12 * f)
        # one step off the axis the pinhole Jacobian [[f/z, 0, -f x/z^2], [0, f/z, -f y/z^2]]
        # holds to second order in the angle
        x, y = 1e-3 * z, -2e-3 * z
        J = oracle.jacobian([x, y, z], f, f, model)
        Jp = np.array([[f / z, 0, -f * x / z ** 2], [0, f / z, -f * y / z ** 2]])
        assert np.abs(J - Jp).max() < 1e-4 * f / z


def _points(model, rng, n=40):
    out = []
    lim = math.radians(85.0) if model in (oracle.CAM_ORTHOGRAPHIC, oracle.CAM_PINHOLE) else math.radians(170.0)
    while len(out) < n:
        p = rng.normal(size=3) * rng.uniform(0.3, 5.0)
        l = np.linalg.norm(p)
        if model == oracle.CAM_EQUIRECT:
            ok = math.atan2(abs(p[1]), math.hypot(p[0], p[2])) < math.radians(80)
        else:
            ok = math.atan2(math.hypot(p[0], p[1]), p[2]) < lim
        if ok and l > 0.3:
            out.append(p)
    return out


@pytest.mark.parametrize("model", ALL)
def test_jacobian_matches_finite_differences(model):
    rng = np.random.default_rng(10 + model)
    fx, fy = 300.0, 270.0
    for p in _points(model, rng):
        J = oracle.jacobian(p, fx, fy, model)
        h = 1e-6 * np.linalg.norm(p)
        fd = np.zeros((2, 3))
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            fd[:, j] = (oracle.project_point(p + e, fx, fy, 0, 0, model)
                        - oracle.project_point(p - e, fx, fy, 0, 0, model)) / (2 * h)
        assert np.abs(J - fd).max() < 1e-6 * np.abs(J).max(), (model, p, J, fd)


@pytest.mark.parametrize("model", ALL)
def test_jacobian_grad_matches_finite_differences(model):
    rng = np.random.default_rng(20 + model)
    fx, fy = 300.0, 270.0
    for p in _points(model, rng):
        dJ = oracle.jacobian_grad(p, fx, fy, model)
        h = 1e-5 * np.linalg.norm(p)
        scale = max(np.abs(d).max() for d in dJ)
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            fd = (oracle.jacobian(p + e, fx, fy, model) - oracle.jacobian(p - e, fx, fy, model)) / (2 * h)
            assert np.abs(dJ[j] - fd).max() < 1e-6 * scale, (model, p, j, dJ[j], fd)


def test_field_limits():
    """Orthographic: visible below theta = 85 deg, not above 90 - 2.86 deg; panorama: culled
    near the poles only; equidistant at theta = 150 deg visible."""
    one = lambda mu: dict(means=np.array([mu], np.float64), scales=np.full((1, 3), 0.05),
                          quats=np.array([[1.0, 0, 0, 0]]), opacities=np.array([0.8]),
                          sh=np.zeros((1, 1, 3)), sh_degree=0)
    ang = lambda deg: [2 * math.sin(math.radians(deg)), 0.0, 2 * math.cos(math.radians(deg))]
    cam_o = scenes.fisheye_camera(64, 64, 170.0, model=oracle.CAM_ORTHOGRAPHIC)
    assert oracle.project(one(ang(80.0)), cam_o)[0, 0] == 1
    assert oracle.project(one(ang(89.0)), cam_o)[0, 0] == 0
    cam_e = scenes.fisheye_camera(64, 64, 320.0)
    assert oracle.project(one(ang(150.0)), cam_e)[0, 0] == 1
    cam_p = scenes.panorama_camera(128, 64)
    assert oracle.project(one([0.0, -2.0, 0.05]), cam_p)[0, 0] == 0   # latitude ~ 88.6 deg
    assert oracle.project(one([0.0, -2.0, 0.5]), cam_p)[0, 0] == 1    # latitude ~ 76 deg
    assert oracle.project(one([0.3, 0.2, -2.0]), cam_p)[0, 0] == 1    # behind: still seen


def test_pinhole_guard_band():
    """The pinhole culls a Gaussian whose projected mean lies beyond 1.3 times the half image
    from the principal point: at 90 deg and 160 x 120 (f = 80, c = (80, 60)) the band is
    |x_c / z_c| <= 1.3 and |y_c / z_c| <= 0.975, far inside its angular field (87.1 deg). The
    Gaussians are large enough (footprints of about 100 px) to reach the image from there."""
    one = lambda mu: dict(means=np.array([mu], np.float64), scales=np.full((1, 3), 0.5),
                          quats=np.array([[1.0, 0, 0, 0]]), opacities=np.array([0.8]),
                          sh=np.zeros((1, 1, 3)), sh_degree=0)
    cam = scenes.fisheye_camera(160, 120, 90.0, model=oracle.CAM_PINHOLE)
    assert abs(cam["fx"] - 80.0) < 1e-9 and cam["cx"] == 80.0 and cam["cy"] == 60.0
    z = 2.0
    for tx, ty, vis in [(1.299, 0.0, 1), (1.301, 0.0, 0), (-1.299, 0.5, 1), (-1.301, 0.5, 0),
                        (0.3, 0.974, 1), (0.3, 0.976, 0), (0.0, -0.976, 0), (1.29, -0.97, 1)]:
        G = oracle.project(one([tx * z, ty * z, z]), cam)
        assert G[0, 0] == vis, (tx, ty)
        if vis:
            # the distance to the band (in tiles) is one of the decision margins
            gap = min(104.0 - abs(G[0, oracle.F["xy"]] - 80.0),
                      78.0 - abs(G[0, oracle.F["xy"] + 1] - 60.0)) / 16.0
            assert G[0, oracle.F["rmargin"]] <= gap + 1e-12
    # an equidistant camera of the same size keeps the point the pinhole culls
    cam_e = scenes.fisheye_camera(160, 120, 90.0)
    assert oracle.project(one([1.301 * z, 0.0, z]), cam_e)[0, 0] == 1


def _tiny_scene(seed, n=7, degree=2):
    rng = np.random.default_rng(seed)
    means = rng.normal(size=(n, 3))
    means /= np.linalg.norm(means, axis=1, keepdims=True)
    means *= rng.uniform(1.0, 2.5, (n, 1))
    means[:, 2] = np.abs(means[:, 2]) + 0.4        # in front, off the axis
    means[0] = [0.05, -0.04, 1.3]                   # near the axis: stacked -> the stop rule
    means[1] = [0.06, -0.03, 1.5]
    means[2] = [0.04, -0.05, 1.7]
    scales = np.exp(rng.normal(-1.7, 0.3, (n, 3)))
    quats = rng.normal(size=(n, 4))
    opac = rng.uniform(0.3, 0.95, n)
    opac[:3] = [0.999, 0.999, 0.98]
    K = (degree + 1) ** 2
    sh = rng.normal(0, 0.3, (n, K, 3))
    sh[:, 0, :] = rng.uniform(-1, 1, (n, 3))
    return dict(means=means, scales=scales, quats=quats, opacities=opac, sh=sh, sh_degree=degree)


@pytest.mark.parametrize("model", [oracle.CAM_EQUISOLID, oracle.CAM_STEREOGRAPHIC,
                                   oracle.CAM_ORTHOGRAPHIC, oracle.CAM_EQUIRECT, oracle.CAM_PINHOLE])
def test_tiny_scene_matches_torch_autograd(model):
    scene = _tiny_scene(40 + model)
    if model == oracle.CAM_EQUIRECT:
        cam = scenes.panorama_camera(40, 20)
        cam["fx"], cam["fy"] = 4 * cam["fx"], 4 * cam["fy"]   # zoomed so the scene fills it
        h_, w_ = 20, 40
    else:
        fov = {oracle.CAM_ORTHOGRAPHIC: 170.0, oracle.CAM_PINHOLE: 120.0}.get(model, 190.0)
        cam = scenes.fisheye_camera(24, 20, fov, model=model)
        h_, w_ = 20, 24
    rng = np.random.default_rng(200 + model)
    g = rng.normal(0, 1, (3, h_, w_))
    bg = (0.05, 0.1, 0.2)
    img_t, gr_t = torch_brute.render_and_grad(scene, cam, g, bg)
    G = oracle.project(scene, cam)
    assert (G[:, 0] > 0).sum() >= 4
    im = oracle.render_image(G, cam, bg=bg)
    assert np.abs(im["color"] - img_t).max() < 1e-12
    assert (im["color"] != np.array(bg)[:, None, None]).any()
    pix = oracle.all_pixels(cam)
    dLdC = g.transpose(1, 2, 0).reshape(-1, 3)
    gr = oracle.backward(G, scene, cam, pix, dLdC, bg)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        a, b = gr[k], gr_t[k]
        assert np.abs(a - b).max() <= 1e-9 * max(1.0, np.abs(b).max()), (model, k, a, b)
