"""HostPipeline (host-streamed fwd+bwd steps whose copies overlap the compute, the compute
replayed from CUDA graphs or called step by step): every step's image equals the plain call
sequence's bit for bit and its gradients to summation order, for a stream of steps with
different inputs."""
import numpy as np
import pytest
import torch

from paper_2409_04751_gb300 import scenes
from paper_2409_04751_gb300.pipeline import HostPipeline
from paper_2409_04751_gb300.renderer import FisheyeRenderer, scene_to_device
from tests import parity

pytestmark = pytest.mark.gpu

KEYS = ("means", "scales", "quats", "opacities", "sh")


@pytest.mark.parametrize("use_graph", [True, False])
def test_pipeline_steps_equal_plain_calls(cuda_device, use_graph):
    scene = scenes.shell_scene(20_000, seed=5, sh_degree=2)
    cams = [scenes.pose_camera(200, 150, 180.0, seed=51), scenes.pose_camera(96, 128, 190.0, seed=52)]
    P = sum(c["width"] * c["height"] for c in cams)
    n = scene["means"].shape[0]
    rng = np.random.default_rng(6)
    steps = []
    for s in range(4):
        sc = dict(scene)
        sc["means"] = (scene["means"] + rng.normal(0, 0.01, scene["means"].shape)).astype(np.float32)
        steps.append((sc, scenes.upstream_grad((3 * P,), 1.0, 60 + s)))
    pipe = HostPipeline(n, 2, cams, capacity=1 << 20, use_graph=use_graph)
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).pin_memory()
    host_in = [{k: pin(sc[k]) for k in KEYS} for sc, _ in steps]
    host_dL = [pin(d) for _, d in steps]
    host_img = [torch.empty(3 * P, dtype=torch.float32).pin_memory() for _ in steps]
    host_g = [{k: torch.empty_like(host_in[0][k]).pin_memory() for k in KEYS} for _ in steps]
    pipe.size(host_in[0])
    hs = [pipe.submit(host_in[s], host_dL[s], host_img[s], host_g[s]) for s in range(len(steps))]
    for h in hs:
        assert pipe.wait(h) == 0
    dev = torch.device("cuda:0")
    for s, (sc, dLs) in enumerate(steps):
        r = FisheyeRenderer(dev, capacity=1 << 20)
        gs = scene_to_device(sc, dev)
        fr = r.forward(gs, cams)
        assert torch.equal(fr.images[:3 * P].cpu(), host_img[s])
        g = r.backward(gs, fr, torch.as_tensor(dLs).to(dev))
        for k in KEYS:
            assert parity.rel_l2(host_g[s][k].numpy(), g[k].cpu().numpy()) < 1e-5, (s, k)
