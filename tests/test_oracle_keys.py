"""Pins of the oracle's tile binning + sort (Sec. 3.1 "Rendering": each Gaussian's tile
bounding box is traversed, the (tile, Gaussian) intersections are sorted by tile ID and
then depth; Sec. 4.1: duplicateWithKeys + radixSort).

A hand-worked example (tests/golden/keys_tiny.txt) and a numpy lexsort brute force.
"""
import os

import numpy as np

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _f32bits(x):
    return np.array([x], np.float32).view(np.uint32)[0]


def _load_golden():
    recs, want = [], []
    with open(os.path.join(HERE, "golden", "keys_tiny.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tag, *rest = line.split()
            if tag == "rec":
                v, x0, y0, x1, y1, d = rest
                recs.append((int(v), int(x0), int(y0), int(x1), int(y1), float(d)))
            elif tag == "pair":
                want.append((int(rest[0]), int(rest[1])))
    return recs, want


def test_hand_worked_example():
    recs, want = _load_golden()
    # two views: view 0 has 3x2 tiles (offset 0), view 1 has 2x2 tiles (offset 6)
    tile_offset, tiles_x, n_tiles = [0, 6], [3, 2], 10
    view = [r[0] for r in recs]
    rect = [r[1:5] for r in recs]
    db = [_f32bits(r[5]) for r in recs]
    keys, vals, ranges = oracle.build_keys(view, rect, db, tile_offset, tiles_x, n_tiles)
    got = [(int(k >> np.uint64(32)), int(v)) for k, v in zip(keys, vals)]
    assert got == want
    for k, v in zip(keys, vals):
        assert (int(k) & 0xFFFFFFFF) == int(db[v])
    # ranges: consecutive, covering every pair once
    for t in range(n_tiles):
        s, e = ranges[t]
        assert all(g[0] == t for g in got[s:e])
        assert sum(1 for g in got if g[0] == t) == e - s


def test_random_records_match_lexsort():
    rng = np.random.default_rng(21)
    tiles = [(7, 5), (3, 9), (11, 2)]
    off = np.cumsum([0] + [a * b for a, b in tiles])
    n = 3000
    view = rng.integers(0, 3, n)
    rect = np.zeros((n, 4), np.int32)
    for r in range(n):
        tx, ty = tiles[view[r]]
        x0, y0 = rng.integers(0, tx), rng.integers(0, ty)
        rect[r] = [x0, y0, min(tx - 1, x0 + rng.integers(0, 3)), min(ty - 1, y0 + rng.integers(0, 3))]
    rect[rng.random(n) < 0.2] = -1  # invisible records emit nothing
    depth = rng.choice(np.float32([0.5, 1.25, 2.0, 3.75]), n)  # many exact ties
    depth = np.where(rng.random(n) < 0.5, rng.uniform(0.2, 50, n).astype(np.float32), depth)
    db = depth.astype(np.float32).view(np.uint32)
    keys, vals, ranges = oracle.build_keys(view, rect, db, off[:-1], [t[0] for t in tiles], off[-1])
    ks, vs = [], []
    for r in range(n):
        if rect[r, 0] < 0:
            continue
        for ty in range(rect[r, 1], rect[r, 3] + 1):
            for tx in range(rect[r, 0], rect[r, 2] + 1):
                ks.append((int(off[view[r]] + ty * tiles[view[r]][0] + tx) << 32) | int(db[r]))
                vs.append(r)
    ks, vs = np.array(ks, np.uint64), np.array(vs, np.uint32)
    order = np.lexsort((vs, ks))
    assert np.array_equal(keys, ks[order]) and np.array_equal(vals, vs[order])
    tile = (ks[order] >> np.uint64(32)).astype(np.int64)
    for t in range(off[-1]):
        idx = np.nonzero(tile == t)[0]
        if len(idx):
            assert tuple(ranges[t]) == (idx[0], idx[-1] + 1)
        else:
            assert ranges[t][1] - ranges[t][0] == 0
