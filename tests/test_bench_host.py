"""Host-side helpers of the benchmark: the code hash that keys committed ncu figures to the
kernel source they were taken on (blind to comments and layout, not to code), the job rate and
the single-process max over ranks, and the render working-set formula."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_code_hash_ignores_comments_and_layout_only():
    a = "int f(int x) {\n  return x + 1;  // one more\n}\n"
    b = "/* header\n   comment */\nint f(int x)\n{\n    return x + 1;\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench.code_hash(a) == bench.code_hash(b)
    assert bench.code_hash(a) != bench.code_hash(c)


def test_rates_and_single_process_max():
    assert bench.job_rate(4, 10, 2.0) == pytest.approx(20.0)
    assert bench.max_over_ranks(1.5) == 1.5


def test_render_bytes_counts_every_buffer():
    from paper_2409_04751_gb300 import fgs, scenes
    cam = scenes.fisheye_camera(64, 32, 180.0)
    cams = fgs.cameras([cam])
    n, m = 1000, 5000
    got = bench.render_bytes(fgs, n, cams, 1, m)
    tiles, pix = 4 * 2, 64 * 32
    ws = fgs.fgs_workspace_size(n, cams, m, 0)
    assert got == n * 52 + m * 12 + tiles * 8 + ws + pix * 20


def test_compact_rounds_floats_only_and_keeps_structure():
    line = dict(value=1239.228629294, n=7049570, ok=True, name="x",
                nested=dict(a=[0.123456789, 2, None], b=(1.0 / 3.0,)))
    out = bench.compact(line)
    assert out["value"] == 1239.2 and out["n"] == 7049570 and out["ok"] is True
    assert out["nested"]["a"] == [0.12346, 2, None] and out["nested"]["b"] == [0.33333]
    assert list(out) == list(line)


def test_fp32_units_from_device_properties():
    class P:
        multi_processor_count, major, minor = 152, 10, 3
    assert bench.fp32_units(P()) == (152, 128)
    P.major, P.minor, P.multi_processor_count = 8, 0, 108
    assert bench.fp32_units(P()) == (108, 64)


def test_cell_entries_counts_the_cells_each_rect_covers():
    import numpy as np
    import torch
    # rects (x0, y0, x1, y1) in tiles: one cell, four cells across a corner, three in a row, and
    # a record without pairs
    rects = np.array([[0, 0, 3, 3], [3, 3, 4, 4], [0, 0, 8, 0], [5, 5, 9, 9]], np.uint16)
    tt = torch.tensor([16, 4, 9, 0], dtype=torch.int32)
    rec = np.zeros((4, 12), np.float32)
    rec[:, 10:12] = rects.reshape(4, 4).copy().view(np.float32).reshape(4, 2)
    assert bench.cell_entries(torch.as_tensor(rec.reshape(-1)), tt) == 1 + 4 + 3
