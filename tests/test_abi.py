"""The C ABI library loads and exports every function include/fgs.h declares; host-side
argument checks answer before any launch (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2409_04751_gb300 import build as cuda_build
from paper_2409_04751_gb300 import fgs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(fgs_[a-z_0-9]+)\s*\(", src, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return fgs.lib()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(fgs.EXPORTS)


def test_checked_build_exports_the_same_symbols():
    # the debugging build (index checks compiled in) is a drop-in replacement of libfgs.so
    cuda_build.build(check=True)
    chk = ctypes.CDLL(cuda_build.CHECK_LIB_PATH)
    for n in _declared():
        assert hasattr(chk, n), n
    chk.fgs_status_string.restype = ctypes.c_char_p
    assert b"checked build" in chk.fgs_status_string(fgs.FGS_ERR_BOUNDS)


def _cam(w=64, h=48):
    return fgs.cameras([dict(W=[1, 0, 0, 0, 1, 0, 0, 0, 1], b=[0, 0, 0], fx=20.0, fy=20.0,
                             cx=w / 2, cy=h / 2, width=w, height=h)])


def test_host_helpers(lib):
    cams = _cam(70, 33)
    assert fgs.fgs_total_tiles(cams) == 5 * 3
    assert fgs.fgs_total_pixels(cams) == 70 * 33
    a = fgs.fgs_workspace_size(1000, cams, 1 << 16)
    b = fgs.fgs_workspace_size(1000, cams, 1 << 18)
    assert 0 < a < b
    assert a % 256 == 0


def test_invalid_arguments_rejected_before_launch(lib):
    cams = _cam()
    INV = fgs.FGS_ERR_INVALID_ARG
    out = ctypes.c_size_t(0)
    assert lib.fgs_workspace_size(-1, cams, 1, 10, ctypes.byref(out)) == INV
    assert lib.fgs_workspace_size(10, cams, 1, 0, ctypes.byref(out)) == INV
    assert lib.fgs_workspace_size(10, cams, 0, 10, ctypes.byref(out)) == INV
    assert lib.fgs_workspace_size(10, cams, fgs.MAX_VIEWS + 1, 10, ctypes.byref(out)) == INV
    bad = _cam(0, 10)
    assert lib.fgs_workspace_size(10, bad, 1, 10, ctypes.byref(out)) == INV
    assert fgs.fgs_total_tiles(bad) == -1
    # camera model outside fgs_camera_model; every listed model accepted
    for m in (-1, fgs.FGS_CAM_PINHOLE + 1):
        bad = _cam()
        bad[0].model = m
        assert lib.fgs_workspace_size(10, bad, 1, 10, ctypes.byref(out)) == INV
    for m in range(fgs.FGS_CAM_PINHOLE + 1):
        ok = _cam()
        ok[0].model = m
        assert lib.fgs_workspace_size(10, ok, 1, 10, ctypes.byref(out)) == fgs.FGS_OK
    # preprocess: null Gaussians, bad degree, null pointers, misaligned records
    g = fgs.FgsGaussians(16, 16, 16, 16, 16, 10, 4)
    assert lib.fgs_preprocess(ctypes.byref(g), cams, 1, 256, 256, None) == INV
    g = fgs.FgsGaussians(0, 16, 16, 16, 16, 10, 3)
    assert lib.fgs_preprocess(ctypes.byref(g), cams, 1, 256, 256, None) == INV
    g = fgs.FgsGaussians(16, 16, 16, 16, 16, 10, 3)
    assert lib.fgs_preprocess(ctypes.byref(g), cams, 1, 264 + 4, 256, None) == INV
    assert lib.fgs_preprocess(None, cams, 1, 256, 256, None) == INV
    # bin_sort: workspace too small / misaligned, capacity out of range
    assert lib.fgs_bin_sort(256, 256, 10, cams, 1, 256, 256, 100, 256, 256, 256, 16, None) == INV
    assert lib.fgs_bin_sort(256, 256, 10, cams, 1, 256, 256, 0, 256, 256, 256, 1 << 30, None) == INV
    assert lib.fgs_bin_sort(256, 256, 10, cams, 1, 256, 256, 1 << 33, 256, 256, 256, 1 << 40, None) == INV
    assert lib.fgs_bin_sort(256, 256, 10, cams, 1, 256, 256, 100, 256, 256, 260, 1 << 30, None) == INV
    # rasterize / backward: null outputs
    assert lib.fgs_rasterize(256, 256, 256, cams, 1, None, 0, 256, 256, 256, 1 << 20, None) == INV
    assert lib.fgs_backward(ctypes.byref(fgs.FgsGaussians(16, 16, 16, 16, 16, 10, 3)), cams, 1,
                            256, 256, 256, 256, None, 256, 256, 0, 256, 256, 256, 256, 256, 256,
                            1 << 20, None) == INV
    assert fgs.status_string(fgs.FGS_ERR_CAPACITY).startswith("more intersections")
    # bin_sort_ex flags: unknown bits and ellipse + onesweep rejected; onesweep needs the larger
    # workspace
    a = fgs.fgs_workspace_size(1000, cams, 1 << 16)
    b = fgs.fgs_workspace_size(1000, cams, 1 << 16, fgs.FGS_BIN_ONESWEEP)
    assert b > a and fgs.fgs_workspace_size(1000, cams, 1 << 16, fgs.FGS_BIN_ELLIPSE) == a
    assert lib.fgs_workspace_size_ex(10, cams, 1, 10, 4, ctypes.byref(out)) == INV
    for fl in (4, fgs.FGS_BIN_ELLIPSE | fgs.FGS_BIN_ONESWEEP):
        assert lib.fgs_bin_sort_ex(256, 256, 10, cams, 1, 256, 256, 100, 256, 256, 256, 1 << 30,
                                   fl, None, None) == INV
    assert lib.fgs_bin_sort_ex(256, 256, 10, cams, 1, 256, 256, 100, 256, 256, 256, 1 << 12,
                               fgs.FGS_BIN_ONESWEEP, None, None) == INV  # workspace too small
    # more Gaussians than the 32-bit record index holds, bounded before any product with the
    # view count
    assert lib.fgs_bin_sort_ex(256, 256, 1 << 40, cams, 1, 256, 256, 100, 256, 256, 256,
                               1 << 30, 0, None, None) == INV
    assert lib.fgs_workspace_size(1 << 62, cams, 1, 10, ctypes.byref(out)) == INV


def test_options_checked_before_launch(lib):
    """fgs_options: work shapes outside the lists and unknown flag bits are refused by every
    call that takes them, before anything is launched."""
    cams = _cam()
    INV = fgs.FGS_ERR_INVALID_ARG
    bad = [fgs.options(fwd=3), fgs.options(fwd=8), fgs.options(bwd=16), fgs.options(bwd=-1),
           fgs.FgsOptions(0, 0, 4, 0)]
    g = fgs.FgsGaussians(16, 16, 16, 16, 16, 10, 3)
    for o in bad:
        r = ctypes.byref(o)
        assert lib.fgs_rasterize_ex(256, 256, 256, cams, 1, None, 256, 256, 256, 256, 1 << 20,
                                    r, None) == INV
        assert lib.fgs_backward_raster_ex(256, 256, 256, 10, cams, 1, None, 256, 256, 256, 256,
                                          1 << 20, r, None) == INV
        assert lib.fgs_backward_ex(ctypes.byref(g), cams, 1, 256, 256, 256, 256, None, 256, 256,
                                   256, 256, 256, 256, 256, 256, 256, 1 << 20, r, None) == INV
        assert lib.fgs_bin_sort_ex(256, 256, 10, cams, 1, 256, 256, 100, 256, 256, 256, 1 << 30,
                                   0, r, None) == INV
    # the measurement events come in pairs
    half = fgs.options(fwd=1, bwd=8)
    half.main_kernel_events[0] = 4096
    assert lib.fgs_rasterize_ex(256, 256, 256, cams, 1, None, 256, 256, 256, 256, 1 << 20,
                                ctypes.byref(half), None) == INV
    # null outputs are still refused when the options are fine
    ok = ctypes.byref(fgs.options(fwd=1, bwd=8, wait_limit=5))
    assert lib.fgs_rasterize_ex(256, 256, 256, cams, 1, None, 0, 256, 256, 256, 1 << 20, ok,
                                None) == INV
