"""Shared helpers of the GPU-vs-oracle parity tests.

Tolerances (FP32 GPU against the FP64 oracle):
  images: max |d| <= 1e-3 over pixels whose decisions are not within rounding of a threshold,
          mean |d| <= 1e-5 per channel over all pixels;
  gradients: relative L2 <= 1e-3 per parameter tensor;
  keys / values / tile ranges: bit-exact given the same records.
A pixel is "flagged" when one of its decisions sits within FP32 reach of its threshold:
|ln alpha - ln(1/255)| < 2e-3, |ln(T (1 - alpha) / 1e-4)| < 2e-3, or two consecutive blended
Gaussians with depths within 2e-6 (relative), and flipping that decision could move the
colour by at least IMPACT_MIN (a quarter of the max tolerance; flips below it cannot break the
max check on their own). The GPU may decide a flagged pixel either way.
"""
import numpy as np
import torch

import oracle

IMG_MAX = 1e-3
IMG_MEAN = 1e-5
GRAD_REL = 1e-3
MARGIN_ALPHA = 2e-3
MARGIN_T = 2e-3
MARGIN_DEPTH = 2e-6
IMPACT_MIN = 2.5e-4


def flagged(margins):
    m = np.asarray(margins)
    return (m[..., 0] < MARGIN_ALPHA) | (m[..., 1] < MARGIN_T) | (m[..., 2] < MARGIN_DEPTH)


def check_image(gpu_img, ref, what=""):
    """gpu_img [3,H,W]; ref = oracle.render_image(...) dict. Returns a stats dict."""
    gpu_img = np.asarray(gpu_img, np.float64)
    d = np.abs(gpu_img - ref["color"])
    fl = flagged(ref["margins"])
    ok = ~fl
    mx = float(d[:, ok].max()) if ok.any() else 0.0
    mean = d.reshape(3, -1).mean(1)
    stats = dict(max_unflagged=mx, mean=mean.tolist(), flagged=int(fl.sum()), pixels=int(fl.size))
    assert mx <= IMG_MAX, f"{what} max |d| {mx} > {IMG_MAX} ({stats})"
    assert np.all(mean <= IMG_MEAN), f"{what} mean |d| {mean} > {IMG_MEAN} ({stats})"
    return stats


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def check_grads(gpu, ref, what="", tol=GRAD_REL):
    out = {}
    for k in ("means", "scales", "quats", "opacities", "sh"):
        a = gpu[k].detach().cpu().numpy() if torch.is_tensor(gpu[k]) else gpu[k]
        r = rel_l2(a, ref[k])
        out[k] = r
    bad = {k: v for k, v in out.items() if not v <= tol}
    assert not bad, f"{what} gradient rel L2 above {tol}: {bad} (all: {out})"
    return out


def u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def u64(t):
    return t.detach().cpu().numpy().view(np.uint64)


def records_np(frame_records, R):
    """[R] structured view of the 48-byte records."""
    raw = frame_records.detach().cpu().numpy()[:R * 12].copy()
    f = raw.reshape(R, 12)
    rect = f[:, 10:12].copy().view(np.uint16).reshape(R, 4)
    return dict(xy=f[:, 0:2], conic=f[:, 2:5], opacity=f[:, 5], rgb=f[:, 6:9], depth=f[:, 9],
                depth_bits=f[:, 9].copy().view(np.uint32), rect=rect.astype(np.int32))


def rows_near_pixels(G, pixels, width, height):
    """Ascending indices of the visible oracle rows whose FP64 bounding box (the oracle's own
    prefilter: |p - xy| <= ext per axis, pixel centres at +0.5) contains at least one of the
    given pixels, widened by one pixel per side. Rendering those rows alone gives the same
    pixels: every other row is skipped by the oracle's box test anyway, and keeping the rows
    in ascending order keeps the index tie-break. Lets the oracle render sampled pixels of a
    multi-million-Gaussian scene without scanning every row per pixel."""
    F = oracle.F
    pix = np.asarray(pixels, np.int64).reshape(-1, 2)
    occ = np.zeros((height + 1, width + 1), np.int64)
    occ[pix[:, 1] + 1, pix[:, 0] + 1] = 1
    sat = occ.cumsum(0).cumsum(1)  # sat[j, i] = samples with row < j and column < i
    rows = np.nonzero(G[:, F["vis"]] > 0)[0]
    H = G[rows]
    x, y = H[:, F["xy"]], H[:, F["xy"] + 1]
    ex, ey = H[:, F["ext"]], H[:, F["ext"] + 1]
    i0 = np.clip(np.floor(x - ex - 0.5) - 1, 0, width).astype(np.int64)
    i1 = np.clip(np.ceil(x + ex - 0.5) + 2, 0, width).astype(np.int64)
    j0 = np.clip(np.floor(y - ey - 0.5) - 1, 0, height).astype(np.int64)
    j1 = np.clip(np.ceil(y + ey - 0.5) + 2, 0, height).astype(np.int64)
    cnt = sat[j1, i1] - sat[j0, i1] - sat[j1, i0] + sat[j0, i0]
    return rows[cnt > 0]
