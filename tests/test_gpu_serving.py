"""Serving: dock_submit / dock_poll / dock_cancel with continuous batching.
Requests of different lattice sides, trajectory lengths and sample counts are
submitted while others run; each result must equal the same request
registered alone, a request that arrives during a long one must finish first,
and a cancelled request must report DOCK_E_CANCELLED without disturbing the
others."""
import math
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2605_21398_gb300 import build, dock
    build.build()
    c = dock.Context(0)
    yield c
    _PAIRS.clear()
    c.close()


_PAIRS = {}


def _pair(ctx, w):
    key = (w.name, w.seed)
    if key not in _PAIRS:
        ob = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
        sw = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
        _PAIRS[key] = (ob, sw)
    return _PAIRS[key]


def _same(a, b):
    assert a["best_search"]["rot"] == b["best_search"]["rot"]
    assert a["best_search"]["score"] == b["best_search"]["score"]
    np.testing.assert_array_equal(a["q"], b["q"])
    np.testing.assert_array_equal(a["t"], b["t"])
    assert a["J"] == b["J"]
    assert a["n_evals"] == b["n_evals"]


def _wait(ctx, tickets, timeout_s=300):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = ctx.poll(t, timeout_us=1000)
                if r is not None:
                    out[t] = (r, time.perf_counter())
        assert time.time() - t0 < timeout_s
    return out


def test_served_results_equal_requests_alone(ctx, workload):
    w0 = workload("tiny32")
    w1 = workload("tiny32", replicate=2, poses=150)
    w2 = workload("free64")
    p0, p1, p2 = _pair(ctx, w0), _pair(ctx, w1), _pair(ctx, w2)
    th = math.radians(5)
    reqs = [(p2[0], p2[1], 1500, 300, th, 4), (p0[0], p0[1], 400, 100, th, 3), (p1[0], p1[1], 250, 50, th, 2),
            (p0[0], p0[1], 120, 0, th, 1), (p2[0], p2[1], 200, 64, th, 2)]
    tickets = [ctx.submit(r) for r in reqs]
    got = _wait(ctx, tickets)
    for r, t in zip(reqs, tickets):
        alone = ctx.register(*r)
        _same(got[t][0], alone)
        assert got[t][0]["latency_ms"] > 0


def test_late_requests_join_the_passes_of_a_running_one(ctx, workload):
    w2 = workload("free64")
    w0 = workload("tiny32")
    p2, p0 = _pair(ctx, w2), _pair(ctx, w0)
    th = math.radians(5)
    big = ctx.submit((p2[0], p2[1], 30000, 0, th, 2))
    time.sleep(0.02)
    small = [ctx.submit((p2[0], p2[1], 128, 0, th, 1)), ctx.submit((p0[0], p0[1], 128, 0, th, 1))]
    done = _wait(ctx, [big] + small)
    rb = done[big][0]
    for s in small:
        rs = done[s][0]
        # admitted while the long request was running and finished its search
        # passes before the long one's last pass: their work overlapped
        assert rb["first_pass"] < rs["first_pass"] <= rs["last_pass"] < rb["last_pass"]
    same = done[small[0]][0]
    _same(same, ctx.register(p2[0], p2[1], 128, 0, th, 1))


def test_cancel_and_unknown_ticket(ctx, workload):
    from paper_2605_21398_gb300 import dock
    w2 = workload("free64")
    p2 = _pair(ctx, w2)
    th = math.radians(5)
    t_big = ctx.submit((p2[0], p2[1], 30000, 0, th, 2))
    t_ok = ctx.submit((p2[0], p2[1], 100, 20, th, 1))
    ctx.cancel(t_big)
    with pytest.raises(dock.DockError) as e:
        while ctx.poll(t_big, timeout_us=100000) is None:
            pass
    assert e.value.status == -7
    r = None
    while r is None:
        r = ctx.poll(t_ok, timeout_us=100000)
    _same(r, ctx.register(p2[0], p2[1], 100, 20, th, 1))
    with pytest.raises(dock.DockError):
        ctx.poll(t_ok)          # collected already
    with pytest.raises(dock.DockError):
        ctx.poll(123456789)
