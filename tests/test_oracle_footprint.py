"""The oracle's footprint, checked pixel by pixel (Sec. 3.1 "Rendering": each projected ellipse
determines an axis-aligned bounding box, and a Gaussian is blended only in the tiles that box
covers).

The reading used on both sides: the box is the exact AABB of the ellipse d^T Sigma_p^-1 d <= q*,
q* = 2 ln(255 opacity), padded by x(1 + 1e-5) + 1e-3 px, and the tile rect is
floor((x -+ e) / 16) clamped to the grid. Its claim is that every pixel where
alpha = min(0.99, opacity exp(-0.5 d^T conic d)) >= 1/255 lies inside the box and in a tile of
the rect, so that tiling never changes the image. Here alpha is evaluated by brute force at
every pixel centre of the image for every Gaussian the oracle projects (no box, no window), on
scenes built to stress the bound: opacities near 1, very anisotropic covariances, a 200-degree
fisheye whose field includes Gaussians behind the camera, ragged edge tiles, and the pinhole
and equisolid models. A Gaussian the oracle culls because its footprint misses the image must
have no such pixel. As a control, the radius 3 sqrt(lambda_max) of the renderer's pseudo-code
misses pixels in the same scenes (it is not conservative once opacity > 0.353).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_04751_gb300 import scenes

F = oracle.F
ALPHA_MIN = 1.0 / 255.0


def _stress_scene(seed, n):
    """Shell scene with opacities near 1 for half of the Gaussians and one short and two long
    axes (log-scales about -4.5, -1.6, -2.1, in random order per Gaussian)."""
    rng = np.random.default_rng(seed)
    sc = scenes.shell_scene(n, seed=seed, sh_degree=0)
    op = sc["opacities"].astype(np.float64)
    hi = rng.random(n) < 0.5
    op[hi] = rng.uniform(0.95, 0.999, int(hi.sum()))
    sc["opacities"] = op.astype(np.float32)
    ls = np.stack([rng.normal(-4.5, 0.3, n), rng.normal(-1.6, 0.3, n), rng.normal(-2.1, 0.3, n)], 1)
    ls = np.take_along_axis(ls, np.argsort(rng.random((n, 3)), axis=1), axis=1)
    sc["scales"] = np.exp(ls).astype(np.float32)
    return sc


def _alpha_pixels(G, rows, w, h):
    """For Gaussians `rows` of G: boolean [len(rows), h, w] of alpha >= 1/255 at every pixel
    centre (i + 0.5, j + 0.5), straight from the definition."""
    px = np.arange(w, dtype=np.float64) + 0.5
    py = np.arange(h, dtype=np.float64) + 0.5
    x, y = G[rows, F["xy"]], G[rows, F["xy"] + 1]
    A, B, C = (G[rows, F["conic"] + k] for k in range(3))
    op = G[rows, F["opacity"]]
    dx = px[None, None, :] - x[:, None, None]
    dy = py[None, :, None] - y[:, None, None]
    q = A[:, None, None] * dx * dx + 2 * B[:, None, None] * dx * dy + C[:, None, None] * dy * dy
    alpha = np.minimum(0.99, op[:, None, None] * np.exp(-0.5 * q))
    return alpha >= ALPHA_MIN


CASES = [
    # (seed, n, width, height, fov, model)
    (1, 1500, 333, 201, 200.0, oracle.CAM_EQUIDISTANT),
    (2, 1500, 250, 250, 180.0, oracle.CAM_EQUIDISTANT),
    (3, 1200, 203, 157, 120.0, oracle.CAM_PINHOLE),
    (4, 1200, 241, 113, 190.0, oracle.CAM_EQUISOLID),
]


@pytest.mark.parametrize("seed,n,w,h,fov,model", CASES)
def test_every_contributing_pixel_is_inside_the_box_and_the_rect(seed, n, w, h, fov, model):
    sc = _stress_scene(seed, n)
    cam = scenes.pose_camera(w, h, fov, seed=100 + seed, model=model)
    G = oracle.project(sc, cam)
    vis = np.nonzero(G[:, F["vis"]] > 0)[0]
    assert vis.size > 200
    tiles_x, tiles_y = (w + 15) // 16, (h + 15) // 16
    ty, tx = np.meshgrid(np.arange(h) // 16, np.arange(w) // 16, indexing="ij")
    pyc, pxc = np.meshgrid(np.arange(h) + 0.5, np.arange(w) + 0.5, indexing="ij")
    n_pairs = 0
    n_opaque = 0
    for lo in range(0, vis.size, 48):
        rows = vis[lo:lo + 48]
        hit = _alpha_pixels(G, rows, w, h)
        for k, i in enumerate(rows):
            m = hit[k]
            if not m.any():
                continue
            n_pairs += int(m.sum())
            n_opaque += int(m.sum()) if G[i, F["opacity"]] > 0.95 else 0
            x0, y0, x1, y1 = (G[i, F["rect"] + c] for c in range(4))
            assert 0 <= x0 <= x1 <= tiles_x - 1 and 0 <= y0 <= y1 <= tiles_y - 1
            assert np.all((tx[m] >= x0) & (tx[m] <= x1) & (ty[m] >= y0) & (ty[m] <= y1)), i
            ex, ey = G[i, F["ext"]], G[i, F["ext"] + 1]
            assert np.all(np.abs(pxc[m] - G[i, F["xy"]]) <= ex), i
            assert np.all(np.abs(pyc[m] - G[i, F["xy"] + 1]) <= ey), i
    assert n_pairs > 10_000 and n_opaque > 2_000


@pytest.mark.parametrize("seed,n,w,h,fov,model", CASES[:2])
def test_culled_footprints_reach_no_pixel(seed, n, w, h, fov, model):
    """Gaussians in the field whose box misses the image (the oracle projects them, computes
    their conic, then culls them) reach alpha >= 1/255 at no pixel of it."""
    sc = _stress_scene(seed, n)
    cam = scenes.pose_camera(w, h, fov, seed=100 + seed, model=model)
    G = oracle.project(sc, cam)
    off = np.nonzero((G[:, F["vis"]] == 0) & (np.abs(G[:, F["conic"]]) > 0))[0]
    assert off.size > 20
    for lo in range(0, off.size, 48):
        assert not _alpha_pixels(G, off[lo:lo + 48], w, h).any()


def test_three_sigma_radius_of_the_pseudo_code_is_not_conservative():
    """Control: a square of half side ceil(3 sqrt(lambda_max)) around the mean (the renderer's
    pseudo-code) misses pixels with alpha >= 1/255 in the same scene, while the padded ellipse
    box above misses none."""
    seed, n, w, h, fov, model = CASES[0]
    sc = _stress_scene(seed, n)
    cam = scenes.pose_camera(w, h, fov, seed=100 + seed, model=model)
    G = oracle.project(sc, cam)
    vis = np.nonzero(G[:, F["vis"]] > 0)[0]
    pyc, pxc = np.meshgrid(np.arange(h) + 0.5, np.arange(w) + 0.5, indexing="ij")
    missed = 0
    for lo in range(0, vis.size, 48):
        rows = vis[lo:lo + 48]
        hit = _alpha_pixels(G, rows, w, h)
        for k, i in enumerate(rows):
            a, b, c = (G[i, F["cov"] + q] for q in range(3))
            lam = 0.5 * (a + c) + math.sqrt(max(0.25 * (a - c) ** 2 + b * b, 0.0))
            r = math.ceil(3.0 * math.sqrt(lam))
            m = hit[k]
            out = (np.abs(pxc - G[i, F["xy"]]) > r) | (np.abs(pyc - G[i, F["xy"] + 1]) > r)
            missed += int((m & out).sum())
    assert missed > 0
