"""The serving loop's admission policy, on CPU (no stream is created): a free slot takes the
pending requests in arrival order, of any scene, while the batch stays within its view limit and
the HBM budget left, grouped by scene (one multi-view call per scene); a batch that does not fit
beside the work in flight waits, but an idle device always admits the oldest request. A free
slot starts at once on an idle device and, while other work is in flight, waits up to the
coalescing window unless a full batch is pending."""
import collections
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2409_04751_gb300 import scenes  # noqa: E402
from paper_2409_04751_gb300.serving import Request, Server, _Slot  # noqa: E402


class _Shape:
    def __init__(self, n):
        self.shape = (n, 3)


def _server(n_per_scene, budget, max_views, window_ms=0.5, n_slots=2):
    s = object.__new__(Server)  # the admission policy needs no device
    s.scenes = [{"means": _Shape(n)} for n in n_per_scene]
    s.max_batch_views = max_views
    s.budget = int(budget)
    s.margin = 2.0
    s.window_s = window_ms * 1e-3
    s.max_group_records = 1 << 40
    s.pending = collections.deque()
    s.in_flight_bytes = 0
    s.ipp = [5.0 for _ in n_per_scene]
    s.slots = [_Slot(stream=None) for _ in range(n_slots)]
    return s


def _req(rid, scene, size=512, t=None):
    cam = scenes.fisheye_camera(size, size, 180.0)
    return Request(rid, scene, cam, t_arrival=float(rid) if t is None else t)


def test_requests_batch_in_arrival_order_across_scenes_up_to_the_view_limit():
    s = _server([200_000, 500_000], budget=1 << 40, max_views=3)
    for rid, sc in enumerate([0, 1, 0, 0, 1, 0]):
        s.pending.append(_req(rid, sc))
    groups, need = s._form_batch()
    # the three oldest, grouped by scene in order of first appearance
    assert [(g.scene, [r.rid for r in g.reqs]) for g in groups] == [(0, [0, 2]), (1, [1])]
    assert [r.rid for r in s.pending] == [3, 4, 5]
    for g in groups:
        assert g.cap == s._capacity(g.scene, g.reqs) and g.bytes == s._bytes(g.scene, g.reqs, g.cap)
    assert need == sum(g.bytes for g in groups)
    groups, _ = s._form_batch()
    assert [(g.scene, [r.rid for r in g.reqs]) for g in groups] == [(0, [3, 5]), (1, [4])]
    assert not s.pending


def test_a_scene_group_stops_at_its_record_limit():
    s = _server([1_000_000, 100_000], budget=1 << 40, max_views=16)
    s.max_group_records = 3_000_000  # three views of the large scene
    for rid, sc in enumerate([0, 1, 0, 0, 1, 0, 1]):
        s.pending.append(_req(rid, sc))
    groups, _ = s._form_batch()
    # the fourth view of scene 0 would pass the limit: the batch ends before it
    assert [(g.scene, [r.rid for r in g.reqs]) for g in groups] == [(0, [0, 2, 3]), (1, [1, 4])]
    assert [r.rid for r in s.pending] == [5, 6]


def test_hbm_budget_limits_the_batch_and_defers_it_beside_work_in_flight():
    s = _server([500_000], budget=1 << 40, max_views=16)
    one = s._bytes(0, [_req(0, 0)], s._capacity(0, [_req(0, 0)]))
    s.budget = int(2.5 * one)
    for rid in range(6):
        s.pending.append(_req(rid, 0))
    groups, need = s._form_batch()
    picked = [r.rid for g in groups for r in g.reqs]
    assert 1 <= len(picked) < 6 and need <= s.budget  # stopped by the budget, not the limit
    # with work in flight, a batch that does not fit beside it waits (nothing is taken)
    s.in_flight_bytes = s.budget - one // 2
    before = [r.rid for r in s.pending]
    assert s._form_batch() is None
    assert [r.rid for r in s.pending] == before
    # an idle device admits the oldest request even when it alone exceeds the budget
    s.in_flight_bytes = 0
    s.budget = one // 4
    groups, _ = s._form_batch()
    assert [r.rid for g in groups for r in g.reqs] == [before[0]]


def test_a_free_slot_waits_to_coalesce_only_while_other_work_is_in_flight():
    s = _server([100_000, 100_000], budget=1 << 40, max_views=4, window_ms=0.5)
    assert not s._ready(10.0)  # nothing pending
    s.pending.append(_req(0, 0, t=10.0))
    assert s._ready(10.0001)  # idle device: start at once
    s.slots[1].batch = object()  # another batch in flight
    assert not s._ready(10.0001)  # young request, batch not full: wait
    assert s._ready(10.0005)  # the oldest has waited the window
    for rid in range(1, 4):
        s.pending.append(_req(rid, rid % 2, t=10.0001))
    assert s._ready(10.0002)  # a full batch is pending


def test_capacity_grows_with_views_and_focal_length():
    s = _server([1_000_000], budget=1 << 40, max_views=16)
    a = s._capacity(0, [_req(0, 0, 512)])
    b = s._capacity(0, [_req(0, 0, 512), _req(1, 0, 512)])
    c = s._capacity(0, [_req(0, 0, 1024)])
    assert b > a and c > a
    narrow = Request(9, 0, scenes.fisheye_camera(512, 512, 150.0), 0.0)  # longer focal length
    assert s._capacity(0, [narrow]) > a
    assert np.isfinite(s._weight([narrow]))
