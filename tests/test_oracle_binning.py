"""Pins of the oracle's exact (ellipse) binning: the minimum of the quadratic form over a
tile's rectangle of pixel centres against dense sampling of the rectangle, and the kept pairs
against a brute-force check of every pixel centre of every rect tile (a pair with a pixel
whose alpha reaches 1/255 is always kept; a dropped pair never has one)."""
import math

import numpy as np

import oracle
from paper_2409_04751_gb300 import scenes


def _conic(rng):
    L = rng.normal(size=(2, 2)) * rng.uniform(0.5, 20.0)
    S = L @ L.T + 0.3 * np.eye(2)
    return np.linalg.inv(S)


def test_rect_min_matches_dense_sampling():
    rng = np.random.default_rng(0)
    u = np.linspace(0.0, 1.0, 401)
    for _ in range(200):
        M = _conic(rng)
        mu = rng.uniform(-40, 60, 2)
        xl, yl = rng.uniform(-10, 30, 2)
        xh, yh = xl + rng.uniform(0, 15), yl + rng.uniform(0, 15)
        got = oracle.rect_min_q(mu, [M[0, 0], M[0, 1], M[1, 1]], xl, xh, yl, yh)
        X, Y = np.meshgrid(xl + u * (xh - xl), yl + u * (yh - yl))
        dx, dy = X - mu[0], Y - mu[1]
        q = M[0, 0] * dx * dx + 2 * M[0, 1] * dx * dy + M[1, 1] * dy * dy
        # the analytic minimum is never above any sample and within the grid's resolution of them
        assert got <= q.min() + 1e-9 * max(1.0, q.min())
        step = max(xh - xl, yh - yl) / 400.0
        slope = 2.0 * np.abs(M).max() * (abs(dx).max() + abs(dy).max() + 1.0)
        assert q.min() - got <= slope * step + 1e-9


def test_exact_binning_keeps_every_contributing_pair():
    scene = scenes.shell_scene(3000, seed=3, sh_degree=0)
    cam = scenes.pose_camera(160, 128, 180.0, seed=4)
    G = oracle.project(scene, cam)
    F = oracle.F
    vis = G[:, F["vis"]] > 0
    rect = np.where(vis[:, None], G[:, F["rect"]:F["rect"] + 4], -1).astype(np.int32)
    ell = np.concatenate([G[:, F["xy"]:F["xy"] + 2], G[:, F["conic"]:F["conic"] + 3],
                          G[:, F["qstar"]:F["qstar"] + 1]], 1)
    tx, ty = oracle.tiles_of(cam)
    view = np.zeros(len(G), np.int32)
    db = G[:, F["depth"]].astype(np.float32).view(np.uint32)
    k_all, v_all, _ = oracle.build_keys(view, rect, db, [0], [tx], tx * ty)
    k_ex, v_ex, rg = oracle.build_keys(view, rect, db, [0], [tx], tx * ty, ellipse=ell)
    assert 0 < len(k_ex) < len(k_all)
    kept = set(zip((k_ex >> np.uint64(32)).tolist(), v_ex.tolist()))
    alls = set(zip((k_all >> np.uint64(32)).tolist(), v_all.tolist()))
    assert kept <= alls
    # brute force: a pair (tile, record) has a pixel centre with alpha >= 1/255 iff
    # q(p) <= q*; every such pair is kept
    jj, ii = np.meshgrid(np.arange(16) + 0.5, np.arange(16) + 0.5, indexing="ij")
    contributing = 0
    for (t, r) in alls:
        tyy, txx = divmod(t, tx)
        dx = ii + txx * 16 - G[r, F["xy"]]
        dy = jj + tyy * 16 - G[r, F["xy"] + 1]
        A, B, C = G[r, F["conic"]:F["conic"] + 3]
        q = A * dx * dx + 2 * B * dx * dy + C * dy * dy
        if (q <= G[r, F["qstar"]]).any():
            contributing += 1
            assert (t, r) in kept
    assert contributing > 0.5 * len(kept)
    # tile ranges are consistent with the kept keys
    for t in range(tx * ty):
        s, e = rg[t]
        assert np.all((k_ex[s:e] >> np.uint64(32)) == t)
