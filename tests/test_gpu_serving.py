"""Continuous-batching server: every request's image equals the image of the same request
rendered alone with a plain single-view call, bit for bit, while requests of several scenes
and sizes arrive, overlap on the device and share batches (across scenes too)."""
import numpy as np
import pytest
import torch

from paper_2409_04751_gb300 import scenes
from paper_2409_04751_gb300.renderer import FisheyeRenderer, scene_to_device
from paper_2409_04751_gb300.serving import Server, poisson_requests

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone(cuda_device):
    scs = [scene_to_device(scenes.shell_scene(n, seed=70 + k, sh_degree=3))
           for k, n in enumerate((20_000, 50_000, 30_000))]
    reqs = poisson_requests(3000.0, 0.02, len(scs), seed=5, sizes=[128, 256, 384])
    assert len(reqs) >= 30
    srv = Server(scs, n_slots=3, max_batch_views=8, hbm_budget_bytes=2 << 30, keep_images=True)
    srv.calibrate([[scenes.pose_camera(256, 256, 180.0, seed=1)] for _ in scs])
    stats = srv.run(reqs)
    assert stats.views == len(reqs)
    assert stats.batches < len(reqs)  # requests really were batched together
    s = stats.summary()
    assert s["multi_scene_batches"] >= 1  # and across scenes
    assert sum(s["views_per_batch_hist"].values()) == stats.batches
    r = FisheyeRenderer("cuda", capacity=1 << 20)
    for q in reqs:
        fr = r.forward(scs[q.scene], [q.cam])
        assert torch.equal(fr.view_images([q.cam])[0], q.image), q.rid
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_capacity_overflow_is_retried(cuda_device):
    """A batch sized too small is detected on completion and re-run. At 384 x 384 one view of
    this scene holds about 110k pairs, more than the 65536-slot floor of a first batch sized
    from the far too small estimate, so the first batch overflows however the arrivals are
    grouped."""
    scs = [scene_to_device(scenes.shell_scene(30_000, seed=77, sh_degree=0))]
    reqs = poisson_requests(2000.0, 0.01, 1, seed=6, sizes=[384])
    srv = Server(scs, n_slots=2, max_batch_views=4, keep_images=True)
    srv.ipp = [0.01]  # far too small: the first batches overflow
    stats = srv.run(reqs)
    assert stats.retries >= 1 and stats.views == len(reqs)
    r = FisheyeRenderer("cuda", capacity=1 << 20)
    for q in reqs:
        fr = r.forward(scs[0], [q.cam])
        assert torch.equal(fr.view_images([q.cam])[0], q.image)
