"""Child process of tests/test_gpu_checked_build.py: runs the hot path through whichever library
FGS_CHECKED_BUILD selects and writes what it produced to an .npz file.

  python tests/checked_child.py clean <out.npz>    valid workloads: outputs and status words
  python tests/checked_child.py corrupt <out.npz>  inputs with one index corrupted: status words
                                                  (only ever run with the checked build, whose
                                                  kernels turn the bad index into a status)
"""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2409_04751_gb300 import fgs, scenes  # noqa: E402
from paper_2409_04751_gb300.renderer import FisheyeRenderer, scene_to_device  # noqa: E402

DEV = torch.device("cuda:0")
GRADS = ("means", "scales", "quats", "opacities", "sh")


def _status(ws):
    return fgs.fgs_read_status(ws)


def _run(tag, scene, cams, out, binning="rect", sort="tile", shapes=((0, 0),), capacity=1 << 12):
    """Forward + backward of one workload (the renderer grows a too-small key buffer, so the
    capacity-overflow path runs first); bit-exact outputs and the gradients go to `out`."""
    gs = scene_to_device(scene, DEV)
    r = FisheyeRenderer(DEV, capacity=capacity, binning=binning, sort=sort)
    P = int(fgs.fgs_total_pixels(fgs.cameras(cams)))
    dL = torch.as_tensor(scenes.upstream_grad((3 * P,), 1e-2, seed=3)).to(DEV)
    for fwd, bwd in shapes:
        r.set_shape(fwd, bwd)
        fr = r.forward(gs, cams, bg=(0.1, 0.2, 0.3))
        m = int(fr.n_intersections.item())
        key = f"{tag}/f{fwd}b{bwd}"
        out[key + "/status_fwd"] = np.array([_status(r._bufs["ws"])])
        for name in ("images", "final_T", "n_processed", "tile_ranges"):
            out[f"{key}/{name}"] = getattr(fr, name).cpu().numpy()
        out[key + "/keys"] = fr.keys[:m].cpu().numpy()
        out[key + "/vals"] = fr.vals[:m].cpu().numpy()
        g = r.backward(gs, fr, dL)
        out[key + "/status_bwd"] = np.array([_status(r._bufs["ws"])])
        for k in GRADS:
            out[f"{key}/grad_{k}"] = g[k].cpu().numpy()


def _noalloc(out):
    scene, cams = scenes.config0()
    gs = scene_to_device(scene, DEV)
    r = FisheyeRenderer(DEV, capacity=1 << 16)
    fr = r.forward(gs, cams)
    cam = fgs.cameras(cams)
    n = int(scene["means"].shape[0])
    cap = 1 << 16
    keys = torch.empty(cap, dtype=torch.int64, device=DEV)
    vals = torch.empty(cap + 4, dtype=torch.int32, device=DEV)
    ranges = torch.empty(2 * int(fgs.fgs_total_tiles(cam)), dtype=torch.int32, device=DEV)
    nint = torch.empty(1, dtype=torch.int64, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    fgs.fgs_bin_sort_noalloc(fr.records, fr.tiles_touched, n, cam, keys, vals, cap, ranges, nint,
                             st)
    m = int(nint.item())
    out["noalloc/status"] = st.cpu().numpy()
    out["noalloc/keys"] = keys[:m].cpu().numpy()
    out["noalloc/vals"] = vals[:m].cpu().numpy()
    out["noalloc/tile_ranges"] = ranges.cpu().numpy()


def clean(path):
    out = {}
    scene, cams = scenes.config0()
    _run("config0", scene, cams, out, shapes=((1, 1), (2, 2), (4, 4), (4, 8)))
    _run("config0_ellipse", scene, cams, out, binning="ellipse")
    _run("config0_onesweep", scene, cams, out, sort="onesweep")
    multi = [scenes.pose_camera(320, 240, 190.0, seed=21), scenes.pose_camera(200, 200, 180.0, seed=22),
             scenes.pose_camera(96, 64, 200.0, seed=23)]
    _run("multiview", scenes.shell_scene(20_000, seed=20, sh_degree=3), multi, out)
    models = [scenes.pose_camera(256, 192, 170.0, seed=30 + m, model=m) for m in
              (fgs.FGS_CAM_EQUISOLID, fgs.FGS_CAM_STEREOGRAPHIC, fgs.FGS_CAM_ORTHOGRAPHIC,
               fgs.FGS_CAM_PINHOLE)]
    models.append(scenes.panorama_camera(256, 128))
    _run("camera_models", scenes.shell_scene(8_000, seed=31, sh_degree=2), models, out)
    # few large Gaussians: tiles of thousands of pairs (the long-segment sort class) and the stop
    _run("dense", scenes.shell_scene(3_000, seed=32, r_min=1.0, r_max=1.5, log_scale=(-1.0, 0.3)),
         [scenes.fisheye_camera(256, 256, 180.0)], out)
    # the full-size workload: 500k Gaussians, SH degree 3, 1752 x 1168 at 180 degrees
    s1, c1 = scenes.config1()
    _run("config1", s1, c1, out, capacity=1 << 22)
    _noalloc(out)
    out["loaded/libraries"] = np.array(_loaded())
    np.savez(path, **out)


def _loaded():
    """The libfgs*.so files mapped into this process."""
    names = set()
    with open("/proc/self/maps") as f:
        for line in f:
            p = line.split()[-1]
            if os.path.basename(p).startswith("libfgs"):
                names.add(os.path.basename(p))
    return sorted(names)


def corrupt(path):
    """One corrupted index per case, each on a fresh binning; every case must end in
    FGS_ERR_BOUNDS with no access outside a buffer (the checked kernels skip it)."""
    out = {}
    scene, cams = scenes.config0()
    gs = scene_to_device(scene, DEV)
    r = FisheyeRenderer(DEV, capacity=1 << 16)
    P = int(fgs.fgs_total_pixels(fgs.cameras(cams)))
    dL = torch.as_tensor(scenes.upstream_grad((3 * P,), 1e-2, seed=3)).to(DEV)
    n = int(scene["means"].shape[0])
    R = n * len(cams)

    def busy_tile(fr):
        """A tile whose first pixel blended at least one entry."""
        rg = fr.tile_ranges.view(-1, 2).cpu().numpy().astype(np.int64)
        W = int(cams[0]["width"])
        npro = fr.n_processed.view(-1).cpu().numpy()
        tx = (W + 15) // 16
        for t in np.flatnonzero(rg[:, 1] > rg[:, 0]):
            y, x = 16 * (t // tx), 16 * (t % tx)
            if npro[y * W + x] > 0:
                return int(t), int(rg[t, 0]), int(rg[t, 1])
        raise AssertionError("no busy tile")

    def raster(fr):
        ws = r._bufs["ws"]
        fgs.fgs_rasterize(fr.records, fr.vals, fr.tile_ranges, fr.cams, None, fr.images,
                          fr.final_T, fr.n_processed, ws, ws.numel(), None, r.opts)
        return _status(ws)

    def backward(fr):
        ws = r._bufs["ws"]
        fgs.fgs_backward_raster(fr.records, fr.vals, fr.tile_ranges, n, fr.cams, None,
                                fr.final_T, fr.n_processed, dL, ws, ws.numel(), opts=r.opts)
        return _status(ws)

    # forward: a list entry naming a record past the last one
    fr = r.forward(gs, cams)
    t, s, e = busy_tile(fr)
    fr.vals[s] = R + 7
    out["fwd_record_index"] = np.array([raster(fr)])
    # forward: a tile range ending past the key capacity
    fr = r.forward(gs, cams)
    fr.tile_ranges[2 * t + 1] = r.capacity + 1000
    out["fwd_range_end"] = np.array([raster(fr)])
    # forward: an inverted range
    fr = r.forward(gs, cams)
    fr.tile_ranges[2 * t] = e + 5
    out["fwd_range_inverted"] = np.array([raster(fr)])
    # backward (after a clean forward): a list entry past the last record inside the replayed part
    fr = r.forward(gs, cams)
    fr.vals[s] = R + 7
    out["bwd_record_index"] = np.array([backward(fr)])
    # backward: a tile range ending past the key capacity
    fr = r.forward(gs, cams)
    fr.tile_ranges[2 * t + 1] = r.capacity + 1000
    out["bwd_range_end"] = np.array([backward(fr)])
    # and a clean pass afterwards: the library is still usable and reports no error
    fr = r.forward(gs, cams)
    out["clean_after"] = np.array([backward(fr)])
    np.savez(path, **out)


if __name__ == "__main__":
    {"clean": clean, "corrupt": corrupt}[sys.argv[1]](sys.argv[2])
    torch.cuda.synchronize()
    print("child ok")
