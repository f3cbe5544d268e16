"""Thin Python binding of the C ABI in include/fgs.h (libfgs.so, sm_103a).

Argument marshalling only: every function here passes device pointers and sizes to the
library function of the same name and turns a non-OK status into an exception. Device memory
comes from torch; streams are torch's current stream unless given. There is no fallback: if the
library is not built the first call raises.
"""
import ctypes
import os

import torch

from .build import CHECK_LIB_PATH, LIB_PATH as PRODUCT_LIB_PATH

# FGS_CHECKED_BUILD=1 in the environment loads the checked build (libfgs_check.so: the same ABI,
# every index read from memory compared with its buffer's size, FGS_ERR_BOUNDS on a violation).
LIB_PATH = CHECK_LIB_PATH if os.environ.get("FGS_CHECKED_BUILD") == "1" else PRODUCT_LIB_PATH

RECORD_BYTES = 48
TILE = 16
MAX_VIEWS = 128

FGS_OK = 0
FGS_ERR_INVALID_ARG = 1
FGS_ERR_CAPACITY = 2
FGS_ERR_TIMEOUT = 3
FGS_ERR_CUDA = 4
FGS_ERR_BOUNDS = 5
# camera models (fgs_camera_model)
FGS_CAM_EQUIDISTANT = 0
FGS_CAM_EQUISOLID = 1
FGS_CAM_STEREOGRAPHIC = 2
FGS_CAM_ORTHOGRAPHIC = 3
FGS_CAM_EQUIRECTANGULAR = 4
FGS_CAM_PINHOLE = 5
# fgs_bin_sort_ex flags
FGS_BIN_ELLIPSE = 1
FGS_BIN_ONESWEEP = 2
# fgs_options flags
FGS_OPT_INSTRUMENT = 1
FGS_OPT_NO_WAIT = 2

EXPORTS = ["fgs_workspace_size", "fgs_workspace_size_ex", "fgs_total_tiles", "fgs_total_pixels",
           "fgs_preprocess", "fgs_bin_sort", "fgs_bin_sort_ex", "fgs_rasterize",
           "fgs_rasterize_ex", "fgs_backward", "fgs_backward_ex", "fgs_backward_raster",
           "fgs_backward_raster_ex", "fgs_backward_preprocess", "fgs_bin_sort_noalloc",
           "fgs_loss_l1", "fgs_adam_step", "fgs_read_status", "fgs_read_counters",
           "fgs_status_string"]


class FgsCamera(ctypes.Structure):
    _fields_ = [("W", ctypes.c_float * 9), ("b", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("model", ctypes.c_int32)]


class FgsOptions(ctypes.Structure):
    _fields_ = [("fwd_pixels_per_thread", ctypes.c_int32), ("bwd_pixels_per_thread", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("wait_limit", ctypes.c_uint32),
                ("main_kernel_events", ctypes.c_void_p * 2)]


def options(fwd=0, bwd=0, instrument=False, no_wait=False, wait_limit=0, events=None):
    """fgs_options of one call: rasterizer work shapes (0 = the library's default), the
    instrumented launches, the bound of the binning's look-back waits, and optionally two
    torch.cuda.Event (timing) recorded around the call's main kernel."""
    flags = (FGS_OPT_INSTRUMENT if instrument else 0) | (FGS_OPT_NO_WAIT if no_wait else 0)
    o = FgsOptions(int(fwd), int(bwd), flags, int(wait_limit))
    if events is not None:
        o.main_kernel_events[0] = _event_handle(events[0])
        o.main_kernel_events[1] = _event_handle(events[1])
    return o


def _event_handle(ev):
    """The cudaEvent_t of a torch.cuda.Event (created by recording it once)."""
    if not ev.cuda_event:
        ev.record()
    return ev.cuda_event


def _opt_ref(opts):
    return None if opts is None else ctypes.byref(opts)


class FgsGaussians(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacities", ctypes.c_void_p),
                ("sh", ctypes.c_void_p), ("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32)]


ADAM_MAX_GROUPS = 8
FGS_ACT_NONE, FGS_ACT_EXP, FGS_ACT_SIGMOID = 0, 1, 2


class FgsAdamGroup(ctypes.Structure):
    _fields_ = [("raw", ctypes.c_void_p), ("act", ctypes.c_void_p), ("grad", ctypes.c_void_p),
                ("m", ctypes.c_void_p), ("v", ctypes.c_void_p), ("count", ctypes.c_int64),
                ("activation", ctypes.c_int32), ("lr", ctypes.c_float)]


class FgsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


_lib = None


def lib():
    """Load libfgs.so, or libfgs_check.so under FGS_CHECKED_BUILD=1 (both built by
    __graft_entry__.build() / paper_2409_04751_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing; "
                               "run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        cam_p, g_p = ctypes.POINTER(FgsCamera), ctypes.POINTER(FgsGaussians)
        o_p = ctypes.POINTER(FgsOptions)
        L.fgs_workspace_size.argtypes = [i64, cam_p, i32, i64, ctypes.POINTER(ctypes.c_size_t)]
        L.fgs_workspace_size_ex.argtypes = [i64, cam_p, i32, i64, ctypes.c_uint32,
                                            ctypes.POINTER(ctypes.c_size_t)]
        L.fgs_loss_l1.argtypes = [vp, vp, vp, i64, ctypes.c_float, vp, vp]
        L.fgs_adam_step.argtypes = [ctypes.POINTER(FgsAdamGroup), i32, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_float, vp, vp]
        L.fgs_total_tiles.argtypes = [cam_p, i32]
        L.fgs_total_tiles.restype = i64
        L.fgs_total_pixels.argtypes = [cam_p, i32]
        L.fgs_total_pixels.restype = i64
        L.fgs_preprocess.argtypes = [g_p, cam_p, i32, vp, vp, vp]
        L.fgs_bin_sort.argtypes = [vp, vp, i64, cam_p, i32, vp, vp, i64, vp, vp, vp,
                                   ctypes.c_size_t, vp]
        L.fgs_rasterize.argtypes = [vp, vp, vp, cam_p, i32, vp, vp, vp, vp, vp,
                                    ctypes.c_size_t, vp]
        L.fgs_rasterize_ex.argtypes = [vp, vp, vp, cam_p, i32, vp, vp, vp, vp, vp,
                                       ctypes.c_size_t, o_p, vp]
        L.fgs_backward.argtypes = [g_p, cam_p, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                   vp, vp, vp, ctypes.c_size_t, vp]
        L.fgs_backward_ex.argtypes = [g_p, cam_p, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                      vp, vp, vp, vp, ctypes.c_size_t, o_p, vp]
        L.fgs_backward_raster.argtypes = [vp, vp, vp, i64, cam_p, i32, vp, vp, vp, vp, vp,
                                          ctypes.c_size_t, vp]
        L.fgs_backward_raster_ex.argtypes = [vp, vp, vp, i64, cam_p, i32, vp, vp, vp, vp, vp,
                                             ctypes.c_size_t, o_p, vp]
        L.fgs_backward_preprocess.argtypes = [g_p, cam_p, i32, vp, vp, vp, vp, vp, vp, vp, vp,
                                              ctypes.c_size_t, vp]
        L.fgs_bin_sort_noalloc.argtypes = [vp, vp, i64, cam_p, i32, vp, vp, i64, vp, vp, vp, vp]
        L.fgs_bin_sort_ex.argtypes = [vp, vp, i64, cam_p, i32, vp, vp, i64, vp, vp, vp,
                                      ctypes.c_size_t, ctypes.c_uint32, o_p, vp]
        L.fgs_read_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int)]
        L.fgs_read_counters.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint64)]
        L.fgs_status_string.argtypes = [ctypes.c_int]
        L.fgs_status_string.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("fgs_total_tiles", "fgs_total_pixels", "fgs_status_string"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().fgs_status_string(int(status)).decode()


def _check(status, where):
    if status != FGS_OK:
        raise FgsError(status, where)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def cameras(cams):
    """ctypes array of FgsCamera from camera dicts (W, b, fx, fy, cx, cy, width, height and
    optionally model, default FGS_CAM_EQUIDISTANT)."""
    arr = (FgsCamera * len(cams))()
    for k, c in enumerate(cams):
        W = [float(v) for v in torch.as_tensor(c["W"]).reshape(9).tolist()]
        b = [float(v) for v in torch.as_tensor(c["b"]).reshape(3).tolist()]
        arr[k].W[:] = W
        arr[k].b[:] = b
        arr[k].fx, arr[k].fy = float(c["fx"]), float(c["fy"])
        arr[k].cx, arr[k].cy = float(c["cx"]), float(c["cy"])
        arr[k].width, arr[k].height = int(c["width"]), int(c["height"])
        arr[k].model = int(c.get("model", FGS_CAM_EQUIDISTANT))
    return arr


def gaussians(means, scales, quats, opacities, sh, sh_degree):
    """FgsGaussians over contiguous FP32 device tensors (kept alive by the caller)."""
    n = int(means.shape[0])
    for t in (means, scales, quats, opacities, sh):
        assert t.dtype == torch.float32 and t.is_contiguous(), "FP32 contiguous tensors expected"
    return FgsGaussians(_ptr(means), _ptr(scales), _ptr(quats), _ptr(opacities), _ptr(sh), n,
                        int(sh_degree))


def fgs_workspace_size(n, cams, capacity, flags=0) -> int:
    out = ctypes.c_size_t(0)
    if flags:
        _check(lib().fgs_workspace_size_ex(int(n), cams, len(cams), int(capacity), int(flags),
                                           ctypes.byref(out)), "fgs_workspace_size_ex")
    else:
        _check(lib().fgs_workspace_size(int(n), cams, len(cams), int(capacity),
                                        ctypes.byref(out)), "fgs_workspace_size")
    return int(out.value)


def fgs_total_tiles(cams) -> int:
    return int(lib().fgs_total_tiles(cams, len(cams)))


def fgs_total_pixels(cams) -> int:
    return int(lib().fgs_total_pixels(cams, len(cams)))


def fgs_preprocess(g, cams, records, tiles_touched, stream=None):
    _check(lib().fgs_preprocess(ctypes.byref(g), cams, len(cams), _ptr(records),
                                _ptr(tiles_touched), _stream(stream)), "fgs_preprocess")


def fgs_bin_sort(records, tiles_touched, n, cams, keys, vals, capacity, tile_ranges,
                 n_intersections, workspace, workspace_bytes, stream=None):
    _check(lib().fgs_bin_sort(_ptr(records), _ptr(tiles_touched), int(n), cams, len(cams),
                              _ptr(keys), _ptr(vals), int(capacity), _ptr(tile_ranges),
                              _ptr(n_intersections), _ptr(workspace), int(workspace_bytes),
                              _stream(stream)), "fgs_bin_sort")


def fgs_bin_sort_ex(records, tiles_touched, n, cams, keys, vals, capacity, tile_ranges,
                    n_intersections, workspace, workspace_bytes, flags, stream=None, opts=None):
    """fgs_bin_sort with flags (FGS_BIN_ELLIPSE: keep only the pairs whose tile the alpha >=
    1/255 ellipse reaches; FGS_BIN_ONESWEEP: the device-wide radix sort) and options."""
    _check(lib().fgs_bin_sort_ex(_ptr(records), _ptr(tiles_touched), int(n), cams, len(cams),
                                 _ptr(keys), _ptr(vals), int(capacity), _ptr(tile_ranges),
                                 _ptr(n_intersections), _ptr(workspace), int(workspace_bytes),
                                 int(flags), _opt_ref(opts), _stream(stream)), "fgs_bin_sort_ex")


def fgs_loss_l1(images, targets, dL_dimages, n, scale, loss, stream=None):
    _check(lib().fgs_loss_l1(_ptr(images), _ptr(targets), _ptr(dL_dimages), int(n), float(scale),
                             _ptr(loss), _stream(stream)), "fgs_loss_l1")


def adam_groups(groups):
    """ctypes array of FgsAdamGroup from dicts (raw, act, grad, m, v tensors; activation; lr)."""
    arr = (FgsAdamGroup * len(groups))()
    for k, g in enumerate(groups):
        arr[k].raw = _ptr(g["raw"])
        arr[k].act = _ptr(g["act"]) if g.get("act") is not None else None
        arr[k].grad = _ptr(g["grad"])
        arr[k].m = _ptr(g["m"])
        arr[k].v = _ptr(g["v"])
        arr[k].count = int(g["raw"].numel())
        arr[k].activation = int(g.get("activation", FGS_ACT_NONE))
        arr[k].lr = float(g["lr"])
    return arr


def fgs_adam_step(groups, beta1, beta2, eps, step, stream=None):
    """groups: ctypes array from adam_groups(); step: device int64 tensor [1], the number of
    steps taken (advanced by the call)."""
    _check(lib().fgs_adam_step(groups, len(groups), float(beta1), float(beta2), float(eps),
                               _ptr(step), _stream(stream)), "fgs_adam_step")


def _bg_arg(bg):
    if bg is None:
        return None, None
    arr = (ctypes.c_float * 3)(*[float(v) for v in bg])
    return ctypes.cast(arr, ctypes.c_void_p).value, arr


def fgs_rasterize(records, vals, tile_ranges, cams, bg, images, final_T, n_processed,
                  workspace, workspace_bytes, stream=None, opts=None):
    """fgs_rasterize, or fgs_rasterize_ex when `opts` (options()) is given."""
    bgp, keep = _bg_arg(bg)
    args = (_ptr(records), _ptr(vals), _ptr(tile_ranges), cams, len(cams), bgp, _ptr(images),
            _ptr(final_T), _ptr(n_processed), _ptr(workspace), int(workspace_bytes))
    if opts is None:
        _check(lib().fgs_rasterize(*args, _stream(stream)), "fgs_rasterize")
    else:
        _check(lib().fgs_rasterize_ex(*args, ctypes.byref(opts), _stream(stream)),
               "fgs_rasterize_ex")
    del keep


def fgs_backward(g, cams, records, tiles_touched, vals, tile_ranges, bg, final_T, n_processed,
                 dL_dimages, d_means, d_scales, d_quats, d_opacities, d_sh, workspace,
                 workspace_bytes, stream=None, opts=None):
    """fgs_backward, or fgs_backward_ex when `opts` (options()) is given."""
    bgp, keep = _bg_arg(bg)
    args = (ctypes.byref(g), cams, len(cams), _ptr(records), _ptr(tiles_touched), _ptr(vals),
            _ptr(tile_ranges), bgp, _ptr(final_T), _ptr(n_processed), _ptr(dL_dimages),
            _ptr(d_means), _ptr(d_scales), _ptr(d_quats), _ptr(d_opacities), _ptr(d_sh),
            _ptr(workspace), int(workspace_bytes))
    if opts is None:
        _check(lib().fgs_backward(*args, _stream(stream)), "fgs_backward")
    else:
        _check(lib().fgs_backward_ex(*args, ctypes.byref(opts), _stream(stream)),
               "fgs_backward_ex")
    del keep


def fgs_backward_raster(records, vals, tile_ranges, n, cams, bg, final_T, n_processed,
                        dL_dimages, workspace, workspace_bytes, stream=None, opts=None):
    """fgs_backward_raster, or fgs_backward_raster_ex when `opts` (options()) is given."""
    bgp, keep = _bg_arg(bg)
    args = (_ptr(records), _ptr(vals), _ptr(tile_ranges), int(n), cams, len(cams), bgp,
            _ptr(final_T), _ptr(n_processed), _ptr(dL_dimages), _ptr(workspace),
            int(workspace_bytes))
    if opts is None:
        _check(lib().fgs_backward_raster(*args, _stream(stream)), "fgs_backward_raster")
    else:
        _check(lib().fgs_backward_raster_ex(*args, ctypes.byref(opts), _stream(stream)),
               "fgs_backward_raster_ex")
    del keep


def fgs_backward_preprocess(g, cams, records, tiles_touched, d_means, d_scales, d_quats,
                            d_opacities, d_sh, workspace, workspace_bytes, stream=None):
    _check(lib().fgs_backward_preprocess(ctypes.byref(g), cams, len(cams), _ptr(records),
                                         _ptr(tiles_touched), _ptr(d_means), _ptr(d_scales),
                                         _ptr(d_quats), _ptr(d_opacities), _ptr(d_sh),
                                         _ptr(workspace), int(workspace_bytes), _stream(stream)),
           "fgs_backward_preprocess")


def fgs_bin_sort_noalloc(records, tiles_touched, n, cams, keys, vals, capacity, tile_ranges,
                         n_intersections, status, stream=None):
    """fgs_bin_sort without a workspace (fixed scratch inside the library); `status` is a
    device uint32 buffer that receives the device status word."""
    _check(lib().fgs_bin_sort_noalloc(_ptr(records), _ptr(tiles_touched), int(n), cams,
                                      len(cams), _ptr(keys), _ptr(vals), int(capacity),
                                      _ptr(tile_ranges), _ptr(n_intersections), _ptr(status),
                                      _stream(stream)), "fgs_bin_sort_noalloc")


def fgs_read_status(workspace, stream=None) -> int:
    out = ctypes.c_int(0)
    _check(lib().fgs_read_status(_ptr(workspace), _stream(stream), ctypes.byref(out)),
           "fgs_read_status")
    return int(out.value)


def fgs_read_counters(workspace, stream=None):
    out = (ctypes.c_uint64 * 6)()
    _check(lib().fgs_read_counters(_ptr(workspace), _stream(stream), out), "fgs_read_counters")
    return [int(v) for v in out]
