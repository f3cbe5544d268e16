"""fgs_bin_sort_noalloc: the key sort for callers that cannot allocate device memory.

Plugins inside a host application that owns the GPU memory budget, and real-time loops that
must not call cudaMalloc / cudaFree, have no workspace to hand the library; this entry point
keeps its scratch in a fixed array inside the library. Here it is called twice in a row through
the C ABI, on different inputs, and each result must equal fgs_bin_sort's (which uses a
caller-provided workspace) bit for bit. Sizes beyond its fixed limits must be refused.

This file is named to be collected last, so a run that stops at the first failure has already
run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2409_04751_gb300 import fgs

pytestmark = pytest.mark.gpu


def _cams(sizes):
    return [dict(W=np.eye(3), b=np.zeros(3), fx=100.0, fy=100.0, cx=w / 2, cy=h / 2, width=w,
                 height=h) for (w, h) in sizes]


def _records(seed, n, cams_py):
    """Seeded 48-byte records: random tile rects per view (some empty), depths with ties."""
    rng = np.random.default_rng(seed)
    V = len(cams_py)
    R = n * V
    rec = np.zeros((R, 12), np.float32)
    rect = np.zeros((R, 4), np.int64)
    for v, c in enumerate(cams_py):
        tx, ty = (c["width"] + 15) // 16, (c["height"] + 15) // 16
        x0, y0 = rng.integers(0, tx, n), rng.integers(0, ty, n)
        ext = rng.integers(0, 4, (n, 2))
        rect[v * n:(v + 1) * n] = np.stack(
            [x0, y0, np.minimum(tx - 1, x0 + ext[:, 0]), np.minimum(ty - 1, y0 + ext[:, 1])], 1)
    tt = ((rect[:, 2] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 1] + 1)).astype(np.uint32)
    tt[rng.random(R) < 0.25] = 0
    depth = rng.uniform(0.2, 30.0, R).astype(np.float32)
    depth[rng.random(R) < 0.3] = np.float32(2.5)
    rec[:, 9] = depth
    rec[:, 10:12] = rect.astype(np.uint16).copy().view(np.float32).reshape(R, 2)
    return rec, tt


def _buffers(capacity, tiles, dev):
    return dict(keys=torch.zeros(capacity, dtype=torch.int64, device=dev),
                vals=torch.zeros(capacity + 4, dtype=torch.int32, device=dev),
                ranges=torch.zeros(2 * tiles, dtype=torch.int32, device=dev),
                nint=torch.zeros(1, dtype=torch.int64, device=dev))


def _outputs(b, m):
    return (b["keys"].cpu().numpy()[:m].copy(), b["vals"].cpu().numpy()[:m].copy(),
            b["ranges"].cpu().numpy().copy(), int(b["nint"].item()))


def test_noalloc_matches_workspace_version_twice(cuda_device):
    dev = cuda_device
    cases = [(6000, _cams([(640, 480), (256, 256)]), 1), (2500, _cams([(1752, 1168)]), 2)]
    for n, cams_py, seed in cases:  # two calls in a row, the second on smaller, other inputs
        rec, tt = _records(seed, n, cams_py)
        m = int(tt.astype(np.int64).sum())
        capacity = m + 100
        cams = fgs.cameras(cams_py)
        tiles = fgs.fgs_total_tiles(cams)
        records = torch.as_tensor(rec.reshape(-1)).to(dev)
        ttd = torch.as_tensor(tt.view(np.int32)).to(dev)

        ref = _buffers(capacity, tiles, dev)
        wsb = fgs.fgs_workspace_size(n, cams, capacity)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        fgs.fgs_bin_sort(records, ttd, n, cams, ref["keys"], ref["vals"], capacity,
                         ref["ranges"], ref["nint"], ws, wsb)
        assert fgs.fgs_read_status(ws) == fgs.FGS_OK

        got = _buffers(capacity, tiles, dev)
        status = torch.full((1,), -1, dtype=torch.int32, device=dev)
        fgs.fgs_bin_sort_noalloc(records, ttd, n, cams, got["keys"], got["vals"], capacity,
                                 got["ranges"], got["nint"], status)
        torch.cuda.synchronize()
        assert int(status.item()) == fgs.FGS_OK
        k0, v0, r0, n0 = _outputs(ref, m)
        k1, v1, r1, n1 = _outputs(got, m)
        assert n0 == n1 == m
        assert np.array_equal(k0, k1) and np.array_equal(v0, v1) and np.array_equal(r0, r1)


def test_noalloc_reports_capacity_overflow_like_the_workspace_version(cuda_device):
    """A device-side error reaches the caller's status buffer: with fewer key slots than pairs
    the call reports FGS_ERR_CAPACITY and the true pair count, as fgs_bin_sort does, and the
    next call with room is correct again."""
    dev = cuda_device
    cams_py = _cams([(640, 480)])
    n = 5000
    rec, tt = _records(3, n, cams_py)
    m = int(tt.astype(np.int64).sum())
    cams = fgs.cameras(cams_py)
    tiles = fgs.fgs_total_tiles(cams)
    records = torch.as_tensor(rec.reshape(-1)).to(dev)
    ttd = torch.as_tensor(tt.view(np.int32)).to(dev)
    small = m // 2
    ref = _buffers(small, tiles, dev)
    wsb = fgs.fgs_workspace_size(n, cams, small)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    fgs.fgs_bin_sort(records, ttd, n, cams, ref["keys"], ref["vals"], small, ref["ranges"],
                     ref["nint"], ws, wsb)
    assert fgs.fgs_read_status(ws) == fgs.FGS_ERR_CAPACITY
    got = _buffers(small, tiles, dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    fgs.fgs_bin_sort_noalloc(records, ttd, n, cams, got["keys"], got["vals"], small,
                             got["ranges"], got["nint"], status)
    torch.cuda.synchronize()
    assert int(status.item()) == fgs.FGS_ERR_CAPACITY
    assert int(got["nint"].item()) == int(ref["nint"].item()) == m
    big = _buffers(m + 8, tiles, dev)
    fgs.fgs_bin_sort_noalloc(records, ttd, n, cams, big["keys"], big["vals"], m + 8,
                             big["ranges"], big["nint"], status)
    torch.cuda.synchronize()
    assert int(status.item()) == fgs.FGS_OK and int(big["nint"].item()) == m


def test_noalloc_refuses_sizes_beyond_its_limits(cuda_device):
    L = fgs.lib()
    cams = fgs.cameras(_cams([(256, 256)]))
    dummy = torch.zeros(64, dtype=torch.int64, device=cuda_device)
    p = dummy.data_ptr()
    # more key slots than the fixed scratch holds
    assert L.fgs_bin_sort_noalloc(p, p, 10, cams, 1, p, p, (1 << 19) + 1, p, p, p, None) == \
        fgs.FGS_ERR_INVALID_ARG
    # more records than the fixed scratch holds
    assert L.fgs_bin_sort_noalloc(p, p, (1 << 19) + 1, cams, 1, p, p, 1024, p, p, p, None) == \
        fgs.FGS_ERR_INVALID_ARG
    # a missing status buffer
    assert L.fgs_bin_sort_noalloc(p, p, 10, cams, 1, p, p, 1024, p, p, None, None) == \
        fgs.FGS_ERR_INVALID_ARG
    # more tiles over all views than the fixed scratch holds (2^17): two views of 512 x 256
    # tiles each
    big = fgs.cameras(_cams([(8192, 4096), (8192, 4096)]))
    assert L.fgs_bin_sort_noalloc(p, p, 10, big, 2, p, p, 1024, p, p, p, None) == \
        fgs.FGS_ERR_INVALID_ARG
    # a Gaussian count so large that it would overflow when multiplied by the view count
    assert L.fgs_bin_sort_noalloc(p, p, 1 << 62, big, 2, p, p, 1024, p, p, p, None) == \
        fgs.FGS_ERR_INVALID_ARG
