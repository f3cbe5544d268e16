"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 5.1 "Dataset", Tables 1-3).

This module draws random numbers and nothing else: it holds none of the renderer's
arithmetic and imports nothing from the rest of the package, so the CUDA path and the FP64
oracle both take their inputs from here. All arrays are numpy, FP32 (the precision the
render path takes); the oracle widens the same values to FP64.

Scene dict: means [n,3], scales [n,3] (activated, > 0), quats [n,4] (w, x, y, z),
opacities [n] (activated, in (0, 1)), sh [n, (d+1)^2, 3], sh_degree d.
Camera dict: W [3,3] (world -> camera rotation, row-major), b [3], fx, fy, cx, cy,
width, height. Camera axes: x right, y down, z forward.
"""
import math

import numpy as np


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _sh(rng, n, degree, dc_as_colour=True, hi_std=0.1):
    K = (degree + 1) ** 2
    sh = np.zeros((n, K, 3), np.float32)
    u = rng.random((n, 3))
    # the degree-0 term times its basis value 1 / (2 sqrt(pi)), plus the 0.5 offset, is U(0, 1)
    sh[:, 0, :] = (u - 0.5) * (2.0 * math.sqrt(math.pi)) if dc_as_colour else u
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, hi_std, (n, K - 1, 3))
    return sh


def _unit_quats(rng, n):
    q = rng.normal(size=(n, 4))
    return (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)


def shell_scene(n, seed=0, r_min=1.0, r_max=5.0, log_scale=(-3.0, 0.5), sh_degree=0):
    """Means uniform in volume in the shell r_min <= |x| <= r_max (full sphere)."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.cbrt(rng.uniform(r_min ** 3, r_max ** 3, n))
    means = (d * r[:, None]).astype(np.float32)
    scales = np.exp(rng.normal(log_scale[0], log_scale[1], (n, 3))).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.0, n)).astype(np.float32)
    sh = _sh(rng, n, sh_degree)
    return dict(means=means, scales=scales, quats=quats, opacities=opac, sh=sh,
                sh_degree=sh_degree)


def box_scene(n, seed=0, half=(10.0, 10.0, 2.5), log_scale=(-4.0, 0.7), sh_degree=3):
    """Means uniform in the box [-hx, hx] x [-hy, hy] x [-hz, hz]."""
    rng = np.random.default_rng(seed)
    h = np.asarray(half)
    means = rng.uniform(-h, h, (n, 3)).astype(np.float32)
    scales = np.exp(rng.normal(log_scale[0], log_scale[1], (n, 3))).astype(np.float32)
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.0, n)).astype(np.float32)
    sh = _sh(rng, n, sh_degree)
    return dict(means=means, scales=scales, quats=quats, opacities=opac, sh=sh,
                sh_degree=sh_degree)


def random_rotation(rng):
    """Haar-uniform rotation (QR of a Gaussian matrix with the sign fix, det = +1)."""
    a = rng.normal(size=(3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


# camera models (the C ABI's fgs_camera.model)
CAM_EQUIDISTANT, CAM_EQUISOLID, CAM_STEREOGRAPHIC, CAM_ORTHOGRAPHIC, CAM_EQUIRECT, CAM_PINHOLE = range(6)
RADIAL_R = {CAM_EQUIDISTANT: lambda t: t,
            CAM_EQUISOLID: lambda t: 2.0 * math.sin(0.5 * t),
            CAM_STEREOGRAPHIC: lambda t: 2.0 * math.tan(0.5 * t),
            CAM_ORTHOGRAPHIC: lambda t: math.sin(t),
            CAM_PINHOLE: lambda t: math.tan(t)}


def _pose(rotation, centre):
    W = np.eye(3) if rotation is None else np.asarray(rotation, np.float64)
    W32 = W.astype(np.float32)
    c = np.asarray(centre, np.float64)
    b = (-(W32.astype(np.float64) @ c)).astype(np.float32)
    return W32, b


def fisheye_camera(width, height, fov_deg, rotation=None, centre=(0.0, 0.0, 0.0),
                   model=CAM_EQUIDISTANT):
    """Radial fisheye (r_d = f r(theta)) with horizontal field of view fov_deg: the image's
    half width is f r(fov / 2), so f = (width / 2) / r(fov / 2) (= width / fov in radians for
    the equidistant model); principal point at the image centre. rotation = world -> camera
    (identity if None); the camera sits at `centre` in world space, so b = -W centre."""
    W32, b = _pose(rotation, centre)
    f = float(np.float32(0.5 * width / RADIAL_R[model](0.5 * math.radians(fov_deg))))
    return dict(W=W32, b=b, fx=f, fy=f, cx=float(width) / 2.0, cy=float(height) / 2.0,
                width=int(width), height=int(height), model=int(model))


def panorama_camera(width, height, rotation=None, centre=(0.0, 0.0, 0.0)):
    """Equirectangular panorama: x_p = w (lon + pi) / 2 pi, y_p = h (lat + pi/2) / pi, i.e.
    fx = w / 2 pi, cx = w / 2, fy = h / pi, cy = h / 2."""
    W32, b = _pose(rotation, centre)
    return dict(W=W32, b=b, fx=float(np.float32(width / (2 * math.pi))),
                fy=float(np.float32(height / math.pi)), cx=float(width) / 2.0,
                cy=float(height) / 2.0, width=int(width), height=int(height),
                model=CAM_EQUIRECT)


def pose_camera(width, height, fov_deg, seed, centre_box=None, model=CAM_EQUIDISTANT):
    """Random pose: Haar rotation; centre at the origin, or uniform in centre_box (half
    extents). model = CAM_EQUIRECT gives a panorama (fov_deg unused)."""
    rng = np.random.default_rng(seed)
    R = random_rotation(rng)
    centre = (0.0, 0.0, 0.0) if centre_box is None else rng.uniform(-np.asarray(centre_box),
                                                                    np.asarray(centre_box))
    if model == CAM_EQUIRECT:
        return panorama_camera(width, height, R, centre)
    return fisheye_camera(width, height, fov_deg, R, centre, model)


def upstream_grad(n_views_pixels_shape, std, seed):
    """dL/dimage ~ N(0, std^2), FP32."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, std, n_views_pixels_shape).astype(np.float32)


# ------------------------------------------------------------------------------------------
# The five workloads (sizes of the paper's scenes and resolutions; synthetic stand-ins for the
# ScanNet++ / Blender data, which are not available here).

def config0():
    """10k Gaussians, shell 1-5, log-scales N(-3, 0.5), SH degree 0, 256x256, 180 deg,
    identity pose, seed 0."""
    return shell_scene(10_000, seed=0, sh_degree=0), [fisheye_camera(256, 256, 180.0)]


def config1(seed=1):
    """500k Gaussians as config 0 with SH degree 3; 1752x1168 at 180 deg, random pose with
    the centre at the origin."""
    scene = shell_scene(500_000, seed=seed, sh_degree=3)
    return scene, [pose_camera(1752, 1168, 180.0, seed * 1000 + 1)]


def config2(n_poses=100, seed=2):
    """3M Gaussians in a 20x20x5 box, log-scales N(-4, 0.7), SH degree 3; 2048x2048 at
    190 deg; poses with centres uniform in the box shrunk by 1 m."""
    scene = box_scene(3_000_000, seed=seed)
    cams = [pose_camera(2048, 2048, 190.0, seed * 1000 + k + 1, centre_box=(9.0, 9.0, 1.5))
            for k in range(n_poses)]
    return scene, cams


CONFIG3_RES = [(512, 512), (1024, 1024), (1752, 1168), (2048, 1536)]
CONFIG3_FOV = [150.0, 180.0, 200.0]


def config3(n_views=64, seed=3, n=1_000_000):
    """1M Gaussians (shell, SH degree 3); n_views views of mixed resolution and FOV."""
    scene = shell_scene(n, seed=seed, sh_degree=3)
    rng = np.random.default_rng(seed * 7919)
    cams = []
    for k in range(n_views):
        w, h = CONFIG3_RES[rng.integers(len(CONFIG3_RES))]
        fov = CONFIG3_FOV[rng.integers(len(CONFIG3_FOV))]
        cams.append(pose_camera(w, h, fov, seed * 1000 + k + 1))
    return scene, cams
