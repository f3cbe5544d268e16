"""A workspace is scratch the caller hands over with arbitrary contents: every call must clear
or overwrite what it reads. The backward adds its screen-space sums into accumulators that the
same call zeroes (the tile-work kernel), and the bin/sort writes every tile range itself (no
clearing pass), so stale bytes in the workspace, or in the range buffer, and a second backward
on the same workspace must leave the outputs unchanged."""
import numpy as np
import pytest
import torch

from paper_2409_04751_gb300 import fgs, scenes
from paper_2409_04751_gb300.renderer import gaussians_of, scene_to_device

pytestmark = pytest.mark.gpu


def _frame(dev, gs, g, cams, n, size, fill):
    """preprocess, bin/sort, rasterize and backward on a workspace and range buffer whose bytes
    are all `fill` beforehand; returns (status, ranges, image, gradients of two backward calls)."""
    P = size[0] * size[1]
    tiles = fgs.fgs_total_tiles(cams)
    records = torch.empty(n * 12, dtype=torch.float32, device=dev)
    tt = torch.empty(n, dtype=torch.int32, device=dev)
    fgs.fgs_preprocess(g, cams, records, tt)
    cap = int(tt.sum().item()) + 64
    wsb = fgs.fgs_workspace_size(n, cams, cap, 0)
    ws = torch.full((wsb,), fill, dtype=torch.uint8, device=dev)
    keys = torch.empty(cap, dtype=torch.int64, device=dev)
    vals = torch.empty(cap + 4, dtype=torch.int32, device=dev)
    ranges = torch.full((2 * tiles,), int(np.frombuffer(bytes([fill] * 4), np.int32)[0]),
                        dtype=torch.int32, device=dev)
    nint = torch.zeros(1, dtype=torch.int64, device=dev)
    fgs.fgs_bin_sort(records, tt, n, cams, keys, vals, cap, ranges, nint, ws, wsb)
    img = torch.empty(3 * P, dtype=torch.float32, device=dev)
    fT = torch.empty(P, dtype=torch.float32, device=dev)
    npr = torch.empty(P, dtype=torch.int32, device=dev)
    bg = (0.1, 0.2, 0.3)
    fgs.fgs_rasterize(records, vals, ranges, cams, bg, img, fT, npr, ws, wsb)
    dL = torch.as_tensor(scenes.upstream_grad((3 * P,), 1e-2, seed=3)).to(dev)
    out = []
    for _ in range(2):
        grads = {k: torch.full_like(gs[k], 5.0)
                 for k in ("means", "scales", "quats", "opacities", "sh")}
        fgs.fgs_backward(g, cams, records, tt, vals, ranges, bg, fT, npr, dL, grads["means"],
                         grads["scales"], grads["quats"], grads["opacities"], grads["sh"], ws,
                         wsb)
        out.append({k: v.cpu().numpy() for k, v in grads.items()})
    torch.cuda.synchronize()
    return fgs.fgs_read_status(ws), ranges.cpu().numpy(), img.cpu().numpy(), out


@pytest.mark.parametrize("fill", [0x00, 0x3F, 0xFF])
def test_stale_workspace_changes_nothing(cuda_device, fill):
    dev = cuda_device
    n, size = 6000, (320, 240)
    scene = scenes.shell_scene(n, seed=41, sh_degree=2)
    cam = scenes.pose_camera(size[0], size[1], 180.0, seed=42)
    gs = scene_to_device(scene, dev)
    g = gaussians_of(gs)
    cams = fgs.cameras([cam])
    ref = _frame(dev, gs, g, cams, n, size, 0x00)
    got = _frame(dev, gs, g, cams, n, size, fill)
    assert ref[0] == fgs.FGS_OK and got[0] == fgs.FGS_OK
    assert np.array_equal(got[1], ref[1])  # every tile range written by the bin/sort
    assert np.array_equal(got[2], ref[2])  # the image
    for grads in (got[3][0], got[3][1], ref[3][1]):  # both calls, either workspace
        for k, v in grads.items():
            r = ref[3][0][k]
            rel = np.linalg.norm(v - r) / max(np.linalg.norm(r), 1e-30)
            assert rel < 1e-5, (k, rel)  # the sums' order varies: atomics, not accumulation
