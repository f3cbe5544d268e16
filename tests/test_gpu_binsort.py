"""GPU bin/sort (fgs_bin_sort: cell count, cell scan, cell scatter, per-cell sort with tile
masks, tile scan, per-tile emission; and fgs_bin_sort_ex with FGS_BIN_ONESWEEP: key emission and
device-wide onesweep radix sort) against the oracle's key builder, bit for bit, on the same
seeded synthetic records. The cases reach every size class of the per-cell sort (cells sorted
in shared memory at both word counts of the smaller class and in the larger class, and cells
longer than the largest shared-memory class, sorted in chunks through global memory), the
bucket sort and its radix fallback, and both ways the cell walks count (in shared memory, and
with more cells than a CTA holds, in global memory)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2409_04751_gb300 import fgs

pytestmark = pytest.mark.gpu


def _cams(sizes):
    return [dict(W=np.eye(3), b=np.zeros(3), fx=100.0, fy=100.0, cx=w / 2, cy=h / 2, width=w,
                 height=h) for (w, h) in sizes]


def _records(rng, n, cams_py, p_empty=0.2, max_ext=3, tie_frac=0.3, big_frac=0.0):
    """Seeded records for n Gaussians x V views: random rects inside each view's tile grid
    (some empty, a few very large), depths with many exact ties."""
    V = len(cams_py)
    R = n * V
    rec = np.zeros((R, 12), np.float32)
    rect = np.full((R, 4), -1, np.int32)
    for v, c in enumerate(cams_py):
        tx, ty = (c["width"] + 15) // 16, (c["height"] + 15) // 16
        sl = slice(v * n, (v + 1) * n)
        x0 = rng.integers(0, tx, n)
        y0 = rng.integers(0, ty, n)
        ext = rng.integers(0, max_ext + 1, (n, 2))
        big = rng.random(n) < big_frac
        ext[big] = rng.integers(max_ext, max(tx, ty) + 1, (int(big.sum()), 2))
        x1 = np.minimum(tx - 1, x0 + ext[:, 0])
        y1 = np.minimum(ty - 1, y0 + ext[:, 1])
        rect[sl] = np.stack([x0, y0, x1, y1], 1)
    empty = rng.random(R) < p_empty
    rect[empty] = -1
    depth = rng.uniform(0.2, 60.0, R).astype(np.float32)
    ties = rng.random(R) < tie_frac
    depth[ties] = rng.choice(np.float32([0.5, 1.0, 2.5, 7.75]), int(ties.sum()))
    rec[:, 9] = depth
    r16 = np.where(rect[:, :1] < 0, 0, rect).astype(np.uint16)
    rec[:, 10:12] = r16.reshape(R, 4).copy().view(np.float32).reshape(R, 2)
    tt = np.where(rect[:, 0] < 0, 0, (rect[:, 2] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 1] + 1))
    return rec, rect, depth, tt.astype(np.uint32)


SORTS = [0, fgs.FGS_BIN_ONESWEEP]  # the per-tile sort and the device-wide onesweep sort


def _run(rec, tt, n, cams_py, capacity, flags=0, opts=None):
    dev = torch.device("cuda:0")
    cams = fgs.cameras(cams_py)
    R = rec.shape[0]
    records = torch.as_tensor(rec.reshape(-1)).to(dev)
    ttd = torch.as_tensor(tt.view(np.int32)).to(dev)
    keys = torch.empty(capacity, dtype=torch.int64, device=dev)
    vals = torch.empty(capacity + 4, dtype=torch.int32, device=dev)
    tiles = fgs.fgs_total_tiles(cams)
    ranges = torch.full((2 * tiles,), -7, dtype=torch.int32, device=dev)
    nint = torch.zeros(1, dtype=torch.int64, device=dev)
    wsb = fgs.fgs_workspace_size(n, cams, capacity, flags)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    fgs.fgs_bin_sort_ex(records, ttd, n, cams, keys, vals, capacity, ranges, nint, ws, wsb, flags,
                        opts=opts)
    st = fgs.fgs_read_status(ws)
    return dict(keys=keys.cpu().numpy().view(np.uint64), vals=vals.cpu().numpy().view(np.uint32),
                ranges=ranges.cpu().numpy().view(np.uint32).reshape(-1, 2), n=int(nint.item()),
                status=st, tiles=tiles)


def _oracle(rect, depth, n, cams_py):
    V = len(cams_py)
    view = np.repeat(np.arange(V), n)
    txs = [(c["width"] + 15) // 16 for c in cams_py]
    tys = [(c["height"] + 15) // 16 for c in cams_py]
    off = np.cumsum([0] + [a * b for a, b in zip(txs, tys)])
    return oracle.build_keys(view, rect, depth.view(np.uint32), off[:-1], txs, off[-1])


@pytest.mark.parametrize("n,sizes,seed,kw", [
    (1, [(64, 48)], 0, {}),
    (700, [(100, 90)], 1, {}),                                     # four ragged cells
    (9000, [(256, 256)], 2, dict(max_ext=6)),                      # sixteen full cells
    (3000, [(256, 256), (96, 40), (1752, 1168)], 3, dict(max_ext=4)),  # multi-view, ragged
    (20000, [(1752, 1168)], 4, dict(max_ext=10, big_frac=0.002)),  # ~1M pairs, huge rects
    (4000, [(16, 16)], 5, dict(tie_frac=0.9)),                     # one tile, heavy ties
    (3000, [(64, 64)], 6, dict(p_empty=1.0)),                      # nothing visible
    # 10 views x 30k records, 80k tiles, 5320 cells: more than a CTA counts in shared memory
    (30000, [(1752, 1168)] * 10, 9, dict(max_ext=3, p_empty=0.5)),
    # one cell of three tiles with ~2200 entries (the smaller class's second word count)
    (2200, [(48, 16)], 10, dict(max_ext=2, tie_frac=0.0)),
    # one cell with ~4800 entries (the larger class, in shared memory)
    (6000, [(16, 16)], 11, dict(tie_frac=0.0)),
    # one cell with ~16000 entries: longer than any shared-memory class, chunked sort
    (20000, [(16, 16)], 12, dict(tie_frac=0.0)),
    # chunked sort with many equal depths
    (30000, [(32, 32)], 13, dict(max_ext=1, tie_frac=0.6)),
    # every pair at one depth: the order is the record order alone
    (9000, [(16, 16)], 14, dict(tie_frac=1.0)),
    # cells whose depths all tie: too clustered for the bucket sort, sorted by the radix passes
    (3000, [(256, 256)], 15, dict(max_ext=5, tie_frac=1.0)),
    # a mix: half of the entries tie, half do not
    (6000, [(640, 480)], 16, dict(max_ext=4, tie_frac=0.5)),
    # 4096 cells (all counted in shared memory) and 1075 record blocks: the per-block count
    # table would exceed its bound, so the scatter counts its records again
    (1_100_000, [(4096, 4096)], 17, dict(max_ext=1, p_empty=0.6, tie_frac=0.1)),
])
@pytest.mark.parametrize("flags", SORTS)
def test_binsort_bit_exact(cuda_device, n, sizes, seed, kw, flags):
    cams_py = _cams(sizes)
    rng = np.random.default_rng(seed)
    rec, rect, depth, tt = _records(rng, n, cams_py, **kw)
    m = int(tt.astype(np.int64).sum())
    cap = max(m, 1) + 37
    out = _run(rec, tt, n, cams_py, cap, flags)
    assert out["status"] == 0 and out["n"] == m
    k, v, rg = _oracle(rect, depth, n, cams_py)
    assert np.array_equal(out["keys"][:m], k)
    assert np.array_equal(out["vals"][:m], v)
    assert np.array_equal(out["ranges"], rg)


@pytest.mark.parametrize("flags", SORTS)
def test_binsort_capacity_overflow_reports_status(cuda_device, flags):
    cams_py = _cams([(256, 256)])
    rng = np.random.default_rng(7)
    rec, rect, depth, tt = _records(rng, 4000, cams_py, max_ext=5)
    m = int(tt.astype(np.int64).sum())
    out = _run(rec, tt, 4000, cams_py, m // 2, flags)
    assert out["status"] == fgs.FGS_ERR_CAPACITY
    assert out["n"] == m  # the true count, so the caller can grow the buffers
    # a repeat with enough room succeeds (the status word is reset by the call)
    out = _run(rec, tt, 4000, cams_py, m, flags)
    assert out["status"] == 0


@pytest.mark.slow
@pytest.mark.parametrize("flags", SORTS)
def test_binsort_full_size_bit_exact(cuda_device, flags):
    """~14M pairs over the 1752x1168 tile grid (the intersection count of the 500k-Gaussian,
    180-degree workload), bit-exact against the oracle."""
    cams_py = _cams([(1752, 1168)])
    rng = np.random.default_rng(8)
    rec, rect, depth, tt = _records(rng, 500_000, cams_py, p_empty=0.3, max_ext=11,
                                    big_frac=0.0005, tie_frac=0.05)
    m = int(tt.astype(np.int64).sum())
    assert m > 8_000_000
    out = _run(rec, tt, 500_000, cams_py, m + 4096, flags)
    assert out["status"] == 0 and out["n"] == m
    k, v, rg = _oracle(rect, depth, 500_000, cams_py)
    assert np.array_equal(out["keys"][:m], k)
    assert np.array_equal(out["vals"][:m], v)
    assert np.array_equal(out["ranges"], rg)


@pytest.mark.parametrize("flags", SORTS)
def test_binsort_tiles_touched_differs_from_rect(cuda_device, flags):
    """Records made by a caller whose tiles_touched is not their rect's area: a record's pairs
    are the first min(tiles_touched, w h) tiles of its rect in row-major order (a shorter count
    takes whole rows and part of the next; a longer one stops at the rect). The per-tile counts
    and the scattered pairs must agree exactly, so the keys, values and ranges are those of
    that definition, written out here by brute force, for both sorts (the device-wide sort
    drops the surplus pairs of a longer count at emission)."""
    cams_py = _cams([(160, 96), (64, 64)])
    rng = np.random.default_rng(21)
    n = 1500
    rec, rect, depth, tt = _records(rng, n, cams_py, max_ext=4, tie_frac=0.2)
    area = tt.astype(np.int64)
    vis = area > 0
    pick = rng.random(tt.size)
    short = vis & (pick < 0.4)
    tt = tt.astype(np.int64)
    tt[short] = rng.integers(1, area[short] + 1)
    longer = vis & (pick > 0.8)
    tt[longer] = area[longer] + rng.integers(1, 4, int(longer.sum()))
    tt = tt.astype(np.uint32)
    cand = int(tt.astype(np.int64).sum())
    out = _run(rec, tt, n, cams_py, cand + 11, flags)
    assert out["status"] == 0
    txs = [(c["width"] + 15) // 16 for c in cams_py]
    tys = [(c["height"] + 15) // 16 for c in cams_py]
    offs = np.cumsum([0] + [a * b for a, b in zip(txs, tys)])
    bits = depth.view(np.uint32)
    key, val = [], []
    for r in range(tt.size):
        if tt[r] == 0 or rect[r, 0] < 0:
            continue
        v = r // n
        x0, y0, x1, y1 = (int(t) for t in rect[r])
        w, h = x1 - x0 + 1, y1 - y0 + 1
        for local in range(int(min(tt[r], w * h))):
            dy, dx = divmod(local, w)
            tile = int(offs[v]) + (y0 + dy) * txs[v] + x0 + dx
            key.append((tile << 32) | int(bits[r]))
            val.append(r)
    key = np.array(key, np.uint64)
    val = np.array(val, np.uint32)
    order = np.lexsort((val, key))
    key, val = key[order], val[order]
    m = key.size
    assert out["n"] == m
    assert np.array_equal(out["keys"][:m], key)
    assert np.array_equal(out["vals"][:m], val)
    tile = (key >> np.uint64(32)).astype(np.int64)
    cnt = np.bincount(tile, minlength=out["tiles"])
    rg = out["ranges"].astype(np.int64)
    assert np.array_equal(rg[:, 1] - rg[:, 0], cnt)
    starts = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    nz = cnt > 0
    assert np.array_equal(rg[nz, 0], starts[nz])


@pytest.mark.parametrize("n,size,flags", [
    (9000, (4096, 2048), 0),                    # 2 cell-scan partitions, 32 tile partitions
    (2000, (1752, 1168), 0),                    # 1 cell-scan partition, 8 tile partitions
    (9000, (256, 256), fgs.FGS_BIN_ONESWEEP),   # the record scan of the onesweep path
    (2000, (1752, 1168), fgs.FGS_BIN_ONESWEEP),  # its radix passes (several key partitions)
])
def test_binsort_timeout_reports_status_and_recovers(cuda_device, n, size, flags):
    """The timeout path of a real call: with FGS_OPT_NO_WAIT every decoupled look-back wait of
    the binning gives up before its first poll. The call must report FGS_ERR_TIMEOUT, the
    rasterizer must then draw the background only and the backward add nothing; the next call
    at the normal wait bound is bit-exact again. Nothing waits on anything that never comes:
    the waits give up by construction, and every kernel after the one that gave up leaves its
    outputs alone."""
    from paper_2409_04751_gb300 import scenes
    from paper_2409_04751_gb300.renderer import gaussians_of, scene_to_device
    dev = cuda_device
    scene = scenes.shell_scene(n, seed=90, sh_degree=1)
    cam = scenes.pose_camera(size[0], size[1], 180.0, seed=91)
    gs = scene_to_device(scene, dev)
    g = gaussians_of(gs)
    cams = fgs.cameras([cam])
    P = size[0] * size[1]
    tiles = fgs.fgs_total_tiles(cams)
    records = torch.empty(n * 12, dtype=torch.float32, device=dev)
    tt = torch.empty(n, dtype=torch.int32, device=dev)
    fgs.fgs_preprocess(g, cams, records, tt)
    cap = int(tt.sum().item()) + 64
    assert cap > 4096 + 64 or flags == 0  # several key partitions for the onesweep passes
    wsb = fgs.fgs_workspace_size(n, cams, cap, flags)
    bg = (0.25, 0.5, 0.75)

    def frame(opts):
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        keys = torch.zeros(cap, dtype=torch.int64, device=dev)
        vals = torch.zeros(cap + 4, dtype=torch.int32, device=dev)
        ranges = torch.zeros(2 * tiles, dtype=torch.int32, device=dev)
        nint = torch.zeros(1, dtype=torch.int64, device=dev)
        fgs.fgs_bin_sort_ex(records, tt, n, cams, keys, vals, cap, ranges, nint, ws, wsb, flags,
                            opts=opts)
        st = fgs.fgs_read_status(ws)
        img = torch.empty(3 * P, dtype=torch.float32, device=dev)
        fT = torch.empty(P, dtype=torch.float32, device=dev)
        npr = torch.empty(P, dtype=torch.int32, device=dev)
        fgs.fgs_rasterize(records, vals, ranges, cams, bg, img, fT, npr, ws, wsb)
        grads = {k: torch.full_like(gs[k], 7.0) for k in ("means", "scales", "quats",
                                                           "opacities", "sh")}
        dL = torch.ones(3 * P, dtype=torch.float32, device=dev)
        fgs.fgs_backward(g, cams, records, tt, vals, ranges, bg, fT, npr, dL, grads["means"],
                         grads["scales"], grads["quats"], grads["opacities"], grads["sh"], ws,
                         wsb)
        torch.cuda.synchronize()
        return st, int(nint.item()), keys, vals, ranges, img, fT, npr, grads

    ref = frame(None)
    assert ref[0] == fgs.FGS_OK
    st, _, _, _, _, img, fT, npr, grads = frame(fgs.options(no_wait=True))
    assert st == fgs.FGS_ERR_TIMEOUT
    img = img.view(3, -1)
    for c in range(3):
        assert torch.all(img[c] == bg[c])
    assert torch.all(fT == 1.0) and torch.all(npr == 0)
    for k, v in grads.items():
        assert torch.all(v == 0), k
    again = frame(fgs.options(wait_limit=0))  # the normal bound
    assert again[0] == fgs.FGS_OK and again[1] == ref[1]
    m = ref[1]
    assert torch.equal(again[2][:m], ref[2][:m]) and torch.equal(again[3][:m], ref[3][:m])
    assert torch.equal(again[4], ref[4]) and torch.equal(again[5], ref[5])
