"""FP64 CPU oracle of the Fisheye-GS hot path (arXiv 2409.04751).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s
cpu_baseline / reference leg may import this package. The product path
(``paper_2409_04751_gb300``) never imports it, and the two share no code: this package
computes everything in plain C (``fgs_oracle.c``, FP64) from the paper's definitions.

Functions and the passage each follows:
  project        view transform, equidistant projection (Sec. 3.2), J_phi (Sec. 4.2),
                 Sigma = R S S^T R^T (Sec. 3.1), Sigma_p = T Sigma T^T, T = J W (Sec. 4.3)
  render         the blending sum of Sec. 3.1 "Rendering", per pixel, by brute force
  backward       gradients of <dL/dC, C> (Sec. 4.2 / 4.3 backward and the inherited blend
                 derivative)
  build_keys     tile binning + stable key sort (Sec. 3.1 "Rendering", Sec. 4.1)
  jacobian, jacobian_grad, project_point, sh_basis: the pieces, exposed for the pins.

Parity unpinned (conventions the paper does not fix): the 0.2 near distance, the
theta < pi - 0.05 cone, the 0.3 dilation, pixel centres at +0.5, depth = |mu_c|, the
index tie-break, the 0.99 alpha cap, the 1e-4 stop. The functions themselves are pinned by
the tests in tests/test_oracle_*.py.
"""
import ctypes
import numpy as np

from .build import build_oracle

_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_U64 = ctypes.POINTER(ctypes.c_uint64)

# field offsets of the per-Gaussian FP64 record written by project()
F = dict(vis=0, muc=1, xy=4, J=6, sig=12, cov=18, conic=21, opacity=24, rgb=25, rgbv=28,
         depth=31, qstar=32, ext=33, rect=35, theta=39, rmargin=40, dir=41, camd=44)
NF = 48
TILE = 16


def _lib_handle():
    global _lib
    if _lib is None:
        path = build_oracle()
        lib = ctypes.CDLL(path)
        lib.orc_project.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D, ctypes.c_int, _D, _D]
        lib.orc_render.argtypes = [ctypes.c_int64, _D, ctypes.c_int64, _I32, _D, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double, _D, _D, _I64, _I32, _D]
        lib.orc_backward.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D, _D, ctypes.c_int, _D,
                                     ctypes.c_int64, _I32, _D, _D, ctypes.c_int, _D, _D, _D, _D,
                                     _D, _D]
        lib.orc_rect_min_q.argtypes = [_D, _D, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double]
        lib.orc_rect_min_q.restype = ctypes.c_double
        lib.orc_build_keys.argtypes = [ctypes.c_int64, _I32, _I32, _U32, _I64, _I32,
                                       ctypes.c_int64, ctypes.c_int64, _U64, _U32, _U32, _D]
        lib.orc_build_keys.restype = ctypes.c_int64
        lib.orc_project_point.argtypes = [_D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _D]
        lib.orc_jacobian.argtypes = [_D, ctypes.c_double, ctypes.c_double, _D]
        lib.orc_jacobian_grad.argtypes = [_D, ctypes.c_double, ctypes.c_double, _D, _D, _D]
        lib.orc_sh_basis.argtypes = [ctypes.c_int, _D, _D, _D]
        lib.orc_cam_project.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, _D]
        lib.orc_cam_jacobian.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, _D]
        lib.orc_cam_jacobian_grad.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double,
                                              _D, _D, _D]
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a, t=_D):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_lib_handle().orc_num_threads())


# camera models (the C oracle's camera[18])
CAM_EQUIDISTANT, CAM_EQUISOLID, CAM_STEREOGRAPHIC, CAM_ORTHOGRAPHIC, CAM_EQUIRECT, CAM_PINHOLE = range(6)


def cam_array(cam) -> np.ndarray:
    """double[19] = W (row-major, world -> camera), b, fx, fy, cx, cy, width, height, model."""
    return _f64(np.concatenate([np.asarray(cam["W"], np.float64).reshape(9),
                                np.asarray(cam["b"], np.float64).reshape(3),
                                [cam["fx"], cam["fy"], cam["cx"], cam["cy"],
                                 cam["width"], cam["height"], cam.get("model", 0)]]))


def tiles_of(cam):
    return (int(cam["width"]) + TILE - 1) // TILE, (int(cam["height"]) + TILE - 1) // TILE


def project(scene, cam) -> np.ndarray:
    """Per-Gaussian FP64 record [n, NF] (fields F) for one camera."""
    lib = _lib_handle()
    n = int(scene["means"].shape[0])
    out = np.zeros((max(n, 1), NF), np.float64)
    means, scales, quats = _f64(scene["means"]), _f64(scene["scales"]), _f64(scene["quats"])
    opac, sh = _f64(scene["opacities"]), _f64(scene["sh"])
    ca = cam_array(cam)
    lib.orc_project(n, _p(means), _p(scales), _p(quats), _p(opac), _p(sh),
                    int(scene["sh_degree"]), _p(ca), _p(out))
    return out[:n]


def all_pixels(cam) -> np.ndarray:
    w, h = int(cam["width"]), int(cam["height"])
    jj, ii = np.meshgrid(np.arange(h, dtype=np.int32), np.arange(w, dtype=np.int32), indexing="ij")
    return np.ascontiguousarray(np.stack([ii.reshape(-1), jj.reshape(-1)], 1))


def render(G, pixels, bg=(0.0, 0.0, 0.0), use_bbox=True, band=2e-3, impact_min=0.0):
    """Render the given pixels [(col, row)]. band: log-alpha half width of the decision band
    whose Gaussians are kept only to measure the alpha-threshold margin. impact_min: decisions
    whose flip could not move the colour by that much are left out of the margins."""
    lib = _lib_handle()
    G = _f64(G)
    pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
    npx = pix.shape[0]
    bgv = _f64(bg)
    color = np.zeros((npx, 3))
    T = np.zeros(npx)
    last = np.zeros(npx, np.int64)
    nc = np.zeros(npx, np.int32)
    marg = np.zeros((npx, 3))
    lib.orc_render(G.shape[0], _p(G), npx, _p(pix, _I32), _p(bgv), int(use_bbox), float(band),
                   float(impact_min), _p(color), _p(T), _p(last, _I64), _p(nc, _I32), _p(marg))
    return dict(color=color, T_final=T, last_g=last, n_contrib=nc, margins=marg)


def render_image(G, cam, bg=(0.0, 0.0, 0.0), use_bbox=True, band=2e-3, impact_min=0.0):
    """Whole image: color [3, H, W] (planar), T_final [H, W], last_g, n_contrib, margins."""
    w, h = int(cam["width"]), int(cam["height"])
    r = render(G, all_pixels(cam), bg, use_bbox, band, impact_min)
    return dict(color=r["color"].reshape(h, w, 3).transpose(2, 0, 1).copy(),
                T_final=r["T_final"].reshape(h, w), last_g=r["last_g"].reshape(h, w),
                n_contrib=r["n_contrib"].reshape(h, w), margins=r["margins"].reshape(h, w, 3))


def backward(G, scene, cam, pixels, dLdC, bg=(0.0, 0.0, 0.0), use_bbox=True):
    """Gradients of sum_p <dLdC[p], C_p> over the given pixels w.r.t. the scene inputs.
    Returns dict(means, scales, quats, opacities, sh, g2d) in FP64."""
    lib = _lib_handle()
    n = int(scene["means"].shape[0])
    K = (int(scene["sh_degree"]) + 1) ** 2
    G = _f64(G)
    pix = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
    g = _f64(dLdC).reshape(-1, 3)
    assert g.shape[0] == pix.shape[0]
    means, scales, quats = _f64(scene["means"]), _f64(scene["scales"]), _f64(scene["quats"])
    opac, sh = _f64(scene["opacities"]), _f64(scene["sh"])
    ca, bgv = cam_array(cam), _f64(bg)
    m1 = max(n, 1)
    dm, ds, dq = np.zeros((m1, 3)), np.zeros((m1, 3)), np.zeros((m1, 4))
    do, dsh, g2d = np.zeros(m1), np.zeros((m1, K, 3)), np.zeros((m1, 9))
    lib.orc_backward(n, _p(G), _p(means), _p(scales), _p(quats), _p(opac), _p(sh),
                     int(scene["sh_degree"]), _p(ca), pix.shape[0], _p(pix, _I32), _p(g),
                     _p(bgv), int(use_bbox), _p(dm), _p(ds), _p(dq), _p(do), _p(dsh), _p(g2d))
    return dict(means=dm[:n], scales=ds[:n], quats=dq[:n], opacities=do[:n], sh=dsh[:n],
                g2d=g2d[:n])


def build_keys(view, rect, depth_bits, tile_offset, tiles_x, n_tiles_total, ellipse=None):
    """Sorted (keys u64, vals u32) and tile_ranges [n_tiles, 2] u32 from per-record
    (view, rect x0 y0 x1 y1 inclusive, FP32 depth bits). ellipse: None (rect binning) or
    [nrec, 6] = (mean x, y, conic A, B, C, q*) for the exact binning."""
    lib = _lib_handle()
    view = np.ascontiguousarray(view, np.int32)
    rect = np.ascontiguousarray(rect, np.int32).reshape(-1, 4)
    db = np.ascontiguousarray(depth_bits, np.uint32)
    to = np.ascontiguousarray(tile_offset, np.int64)
    tx = np.ascontiguousarray(tiles_x, np.int32)
    nrec = rect.shape[0]
    ok = (rect[:, 0] >= 0) & (rect[:, 2] >= rect[:, 0]) & (rect[:, 3] >= rect[:, 1])
    m = int(np.sum(((rect[:, 2] - rect[:, 0] + 1).astype(np.int64)
                    * (rect[:, 3] - rect[:, 1] + 1))[ok]))
    keys = np.zeros(max(m, 1), np.uint64)
    vals = np.zeros(max(m, 1), np.uint32)
    ranges = np.zeros((max(int(n_tiles_total), 1), 2), np.uint32)
    ell = None if ellipse is None else _f64(np.asarray(ellipse).reshape(-1, 6))
    r = lib.orc_build_keys(nrec, _p(view, _I32), _p(rect, _I32), _p(db, _U32), _p(to, _I64),
                           _p(tx, _I32), int(n_tiles_total), m, _p(keys, _U64), _p(vals, _U32),
                           _p(ranges, _U32), None if ell is None else _p(ell))
    assert 0 <= r <= m
    m = r
    return keys[:m], vals[:m], ranges[:int(n_tiles_total)]


def rect_min_q(mu, conic, xl, xh, yl, yh):
    """min over [xl, xh] x [yl, yh] of (p - mu)^T [[A, B], [B, C]] (p - mu)."""
    return float(_lib_handle().orc_rect_min_q(_p(_f64(mu)), _p(_f64(conic)), xl, xh, yl, yh))


def project_point(muc, fx, fy, cx=0.0, cy=0.0, model=CAM_EQUIDISTANT):
    lib = _lib_handle()
    m = _f64(muc)
    out = np.zeros(2)
    if model == CAM_EQUIDISTANT:
        lib.orc_project_point(_p(m), fx, fy, cx, cy, _p(out))
    else:
        lib.orc_cam_project(int(model), _p(m), fx, fy, cx, cy, _p(out))
    return out


def jacobian(muc, fx, fy, model=CAM_EQUIDISTANT):
    lib = _lib_handle()
    m = _f64(muc)
    J = np.zeros(6)
    lib.orc_cam_jacobian(int(model), _p(m), fx, fy, _p(J))
    return J.reshape(2, 3)


def jacobian_grad(muc, fx, fy, model=CAM_EQUIDISTANT):
    """(dJ/dx_c, dJ/dy_c, dJ/dz_c), each 2x3."""
    lib = _lib_handle()
    m = _f64(muc)
    a, b, c = np.zeros(6), np.zeros(6), np.zeros(6)
    lib.orc_cam_jacobian_grad(int(model), _p(m), fx, fy, _p(a), _p(b), _p(c))
    return a.reshape(2, 3), b.reshape(2, 3), c.reshape(2, 3)


def jacobian_grad_paper_form(muc, fx, fy):
    """The equidistant (dJ/dx_c, dJ/dy_c, dJ/dz_c) in the paper's S1..S8 form (Sec. 4.3)."""
    lib = _lib_handle()
    m = _f64(muc)
    a, b, c = np.zeros(6), np.zeros(6), np.zeros(6)
    lib.orc_jacobian_grad(_p(m), fx, fy, _p(a), _p(b), _p(c))
    return a.reshape(2, 3), b.reshape(2, 3), c.reshape(2, 3)


def sh_basis(degree, d):
    """Y [(degree+1)^2] and dY/d(dir) [(degree+1)^2, 3] at unit direction d."""
    lib = _lib_handle()
    dd = _f64(d)
    K = (degree + 1) ** 2
    Y, dY = np.zeros(16), np.zeros(48)
    lib.orc_sh_basis(int(degree), _p(dd), _p(Y), _p(dY))
    return Y[:K], dY.reshape(16, 3)[:K]
