"""The serving loop's admission policy, on CPU (no stream is created): a free slot takes the
oldest pending request and, in arrival order, the other pending requests of the same scene
while the batch stays within its view limit and the HBM budget left; requests of other scenes
keep their place; a batch that does not fit beside the work in flight waits, but an idle
device always admits the oldest request."""
import collections
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2409_04751_gb300 import scenes  # noqa: E402
from paper_2409_04751_gb300.serving import Request, Server  # noqa: E402


class _Shape:
    def __init__(self, n):
        self.shape = (n, 3)


def _server(n_per_scene, budget, max_views):
    s = object.__new__(Server)  # the admission policy needs no device
    s.scenes = [{"means": _Shape(n)} for n in n_per_scene]
    s.max_batch_views = max_views
    s.budget = int(budget)
    s.margin = 1.6
    s.pending = collections.deque()
    s.in_flight_bytes = 0
    s.ipp = [5.0 for _ in n_per_scene]
    return s


def _req(rid, scene, size=512):
    cam = scenes.fisheye_camera(size, size, 180.0)
    return Request(rid, scene, cam, t_arrival=float(rid))


def test_same_scene_requests_batch_in_arrival_order_up_to_the_view_limit():
    s = _server([200_000, 500_000], budget=1 << 40, max_views=3)
    for rid, sc in enumerate([0, 1, 0, 0, 1, 0]):
        s.pending.append(_req(rid, sc))
    scene, picked, cap, need = s._form_batch()
    assert scene == 0 and [r.rid for r in picked] == [0, 2, 3]
    assert [r.rid for r in s.pending] == [1, 4, 5]  # the others keep their order
    assert cap == s._capacity(0, picked) and need == s._bytes(0, picked, cap)
    scene, picked, _, _ = s._form_batch()
    assert scene == 1 and [r.rid for r in picked] == [1, 4]


def test_hbm_budget_limits_the_batch_and_defers_it_beside_work_in_flight():
    s = _server([500_000], budget=1 << 40, max_views=16)
    one = s._bytes(0, [_req(0, 0)], s._capacity(0, [_req(0, 0)]))
    s.budget = int(2.5 * one)
    for rid in range(6):
        s.pending.append(_req(rid, 0))
    _, picked, _, need = s._form_batch()
    assert 1 <= len(picked) < 6 and need <= s.budget  # stopped by the budget, not the limit
    # with work in flight, a batch that does not fit beside it waits (nothing is taken)
    s.in_flight_bytes = s.budget - one // 2
    before = [r.rid for r in s.pending]
    assert s._form_batch() is None
    assert [r.rid for r in s.pending] == before
    # an idle device admits the oldest request even when it alone exceeds the budget
    s.in_flight_bytes = 0
    s.budget = one // 4
    _, picked, _, _ = s._form_batch()
    assert [r.rid for r in picked] == [before[0]]


def test_capacity_grows_with_views_and_focal_length():
    s = _server([1_000_000], budget=1 << 40, max_views=16)
    a = s._capacity(0, [_req(0, 0, 512)])
    b = s._capacity(0, [_req(0, 0, 512), _req(1, 0, 512)])
    c = s._capacity(0, [_req(0, 0, 1024)])
    assert b > a and c > a
    narrow = Request(9, 0, scenes.fisheye_camera(512, 512, 150.0), 0.0)  # longer focal length
    assert s._capacity(0, [narrow]) > a
    assert np.isfinite(s._weight([narrow]))
