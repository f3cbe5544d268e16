"""Buffer management around the C ABI: one forward (preprocess -> bin/sort -> rasterize) and
one backward over a set of fisheye views, with every buffer held on the device by torch.

All arithmetic runs in libfgs.so; this module only sizes and reuses buffers and strings the
four calls together on the current stream.
"""
from dataclasses import dataclass

import numpy as np
import torch

from . import fgs


def scene_to_device(scene, device="cuda"):
    """numpy scene dict -> dict of contiguous FP32 device tensors (+ sh_degree)."""
    out = {}
    for k in ("means", "scales", "quats", "opacities", "sh"):
        out[k] = torch.as_tensor(np.ascontiguousarray(scene[k], dtype=np.float32)).to(device)
    out["sh_degree"] = int(scene["sh_degree"])
    return out


def gaussians_of(gs):
    return fgs.gaussians(gs["means"], gs["scales"], gs["quats"], gs["opacities"], gs["sh"],
                         gs["sh_degree"])


@dataclass
class Frame:
    """Outputs of one forward, kept for the backward."""
    images: torch.Tensor        # [total_pixels * 3] planar per view
    final_T: torch.Tensor       # [total_pixels]
    n_processed: torch.Tensor   # [total_pixels] int32 (u32 values)
    records: torch.Tensor       # [R * 12] float32 (48-byte records)
    tiles_touched: torch.Tensor  # [R] int32
    keys: torch.Tensor          # [capacity] int64 (u64 values)
    vals: torch.Tensor          # [capacity + 4] int32 (u32 values)
    tile_ranges: torch.Tensor   # [total_tiles * 2] int32
    n_intersections: torch.Tensor  # [1] int64
    cams: object
    bg: tuple
    n: int

    def view_images(self, cams_py):
        """List of [3, H, W] views into the packed image buffer."""
        out, off = [], 0
        for c in cams_py:
            w, h = int(c["width"]), int(c["height"])
            out.append(self.images[3 * off:3 * (off + w * h)].view(3, h, w))
            off += w * h
        return out


class FisheyeRenderer:
    """Renders fisheye views of one Gaussian set through libfgs.

    capacity: key-buffer size (intersections); grows automatically on overflow when the
    forward is run with check=True (one host sync per call).
    binning: "rect" (the tile rect of each footprint, as the method bins) or "ellipse" (only
    the tiles the alpha >= 1/255 ellipse reaches; same images, shorter tile lists).
    sort: "tile" (the per-tile sort, default) or "onesweep" (the device-wide radix sort; rect
    binning only); same keys.
    fwd_ppt, bwd_ppt: pixels per thread of the two rasterizers (0 = the library's default);
    images do not depend on them, gradients only through the order of their sums. They are
    passed with every call (fgs_options), so renderers with different shapes can run side by
    side."""

    def __init__(self, device="cuda", capacity=1 << 20, growth=1.25, binning="rect",
                 sort="tile", fwd_ppt=0, bwd_ppt=0):
        self.device = torch.device(device)
        self.capacity = int(capacity)
        self.growth = float(growth)
        if binning not in ("rect", "ellipse") or sort not in ("tile", "onesweep"):
            raise ValueError("binning is 'rect' or 'ellipse', sort 'tile' or 'onesweep'")
        if binning == "ellipse" and sort == "onesweep":
            raise ValueError("the onesweep sort bins by the rect")
        self.flags = ((fgs.FGS_BIN_ELLIPSE if binning == "ellipse" else 0) |
                      (fgs.FGS_BIN_ONESWEEP if sort == "onesweep" else 0))
        self.set_shape(fwd_ppt, bwd_ppt)
        self._bufs = {}

    def set_shape(self, fwd_ppt=0, bwd_ppt=0):
        """Work shape of the rasterizers for this renderer's calls."""
        self.shape = (int(fwd_ppt), int(bwd_ppt))
        self.opts = fgs.options(fwd=self.shape[0], bwd=self.shape[1])

    def _buf(self, name, numel, dtype):
        b = self._bufs.get(name)
        if b is None or b.numel() < numel or b.dtype != dtype:
            b = torch.empty(max(int(numel), 1), dtype=dtype, device=self.device)
            self._bufs[name] = b
        return b[:max(int(numel), 1)]

    def forward(self, gs, cams_py, bg=None, check=True, stream=None):
        cams = fgs.cameras(cams_py)
        n = int(gs["means"].shape[0])
        V = len(cams_py)
        R = n * V
        g = gaussians_of(gs)
        P = fgs.fgs_total_pixels(cams)
        tiles = fgs.fgs_total_tiles(cams)
        records = self._buf("records", R * 12, torch.float32)
        tt = self._buf("tt", R, torch.int32)
        fgs.fgs_preprocess(g, cams, records, tt, stream)
        while True:
            cap = self.capacity
            ws_bytes = fgs.fgs_workspace_size(n, cams, cap, self.flags)
            keys = self._buf("keys", cap, torch.int64)
            vals = self._buf("vals", cap + 4, torch.int32)
            ranges = self._buf("ranges", 2 * tiles, torch.int32)
            nint = self._buf("nint", 1, torch.int64)
            ws = self._buf("ws", ws_bytes, torch.uint8)
            fgs.fgs_bin_sort_ex(records, tt, n, cams, keys, vals, cap, ranges, nint, ws,
                                ws_bytes, self.flags, stream, self.opts)
            if not check:
                break
            st = fgs.fgs_read_status(ws, stream)
            if st == fgs.FGS_ERR_CAPACITY:
                need = int(nint.item())
                self.capacity = int(need * self.growth) + 1024
                continue
            if st != fgs.FGS_OK:
                raise fgs.FgsError(st, "bin_sort (device)")
            break
        images = self._buf("images", 3 * P, torch.float32)
        final_T = self._buf("final_T", P, torch.float32)
        nproc = self._buf("nproc", P, torch.int32)
        bgt = None if bg is None else tuple(float(v) for v in bg)
        fgs.fgs_rasterize(records, vals, ranges, cams, bgt, images, final_T, nproc, ws, ws_bytes,
                          stream, self.opts)
        if check:
            st = fgs.fgs_read_status(ws, stream)
            if st != fgs.FGS_OK:
                raise fgs.FgsError(st, "rasterize (device)")
        return Frame(images, final_T, nproc, records, tt, keys, vals, ranges, nint, cams, bgt, n)

    def backward(self, gs, frame: Frame, dL_dimages, out=None, check=True, stream=None):
        """Gradients w.r.t. (means, scales, quats, opacities, sh), overwritten into `out`
        (dict of tensors shaped like gs) or fresh tensors."""
        if out is None:
            out = {k: torch.empty_like(gs[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
        ws = self._bufs["ws"]
        g = gaussians_of(gs)
        fgs.fgs_backward(g, frame.cams, frame.records, frame.tiles_touched, frame.vals,
                         frame.tile_ranges, frame.bg, frame.final_T, frame.n_processed,
                         dL_dimages, out["means"], out["scales"], out["quats"],
                         out["opacities"], out["sh"], ws, ws.numel(), stream, self.opts)
        if check:
            st = fgs.fgs_read_status(ws, stream)
            if st != fgs.FGS_OK:
                raise fgs.FgsError(st, "backward (device)")
        return out
