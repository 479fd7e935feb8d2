"""Serving admission by the HBM budget of dock_create, and host-side fault
injection on the context's allocator (dock_fail_allocation: the n-th device
allocation answers out of memory before touching the device; no GPU fault is
involved).  Requests that do not fit wait for memory instead of failing, the
memory held never exceeds the budget, a request that can never fit is
refused with DOCK_E_TOO_LARGE, and an allocation failure at any point of an
object build or a registration leaves the context usable with nothing
leaked."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TH = math.radians(5)
REQS = [(0, 900, 200, 2), (1, 700, 100, 3), (0, 500, 0, 1), (1, 1100, 300, 2), (0, 800, 150, 2)]


@pytest.fixture(scope="module")
def lib():
    from paper_2605_21398_gb300 import build, dock
    build.build()
    return dock


def _handles(c, ws):
    return [(c.object_grid(w.obj.verts, w.obj.tris, w.h, w.N),
             c.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)) for w in ws]


def _same(a, b):
    assert a["best_search"]["rot"] == b["best_search"]["rot"]
    np.testing.assert_array_equal(a["q"], b["q"])
    np.testing.assert_array_equal(a["t"], b["t"])
    assert a["J"] == b["J"]


def _wait(c, tickets):
    out = {}
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = c.poll(t, timeout_us=2000)
                if r is not None:
                    out[t] = r
    return out


def test_budget_bounds_held_memory_and_queued_requests_wait(lib, workload):
    ws = [workload("tiny32"), workload("tiny32", replicate=2, poses=150)]
    ref = lib.Context(0)
    try:
        hr = _handles(ref, ws)
        ref.register(hr[0][0], hr[0][1], 900, 200, TH, 3)   # grows the shared scratch
        held0, _, _ = ref.memory_stats()
        alone = [ref.register(hr[i][0], hr[i][1], ng, nl, TH, k) for i, ng, nl, k in REQS]
        _, peak_ref, _ = ref.memory_stats()
    finally:
        ref.close()
    one = peak_ref - held0        # the most one request held on top of the handles and scratch
    assert one > 0
    budget = held0 + int(1.5 * one)
    c = lib.Context(0, hbm_budget=budget)
    try:
        hb = _handles(c, ws)
        c.register(hb[0][0], hb[0][1], 900, 200, TH, 3)
        tickets = [c.submit((hb[i][0], hb[i][1], ng, nl, TH, k)) for i, ng, nl, k in REQS]
        got = _wait(c, tickets)
        for t, a in zip(tickets, alone):
            _same(got[t], a)
        held, peak, b = c.memory_stats()
        assert b == budget and peak <= budget, (peak, budget)
        # not every request fitted at once: some were admitted passes later
        firsts = [got[t]["first_pass"] for t in tickets]
        assert max(firsts) > min(firsts)
        # a request whose own device state exceeds the budget is refused
        big = c.submit((hb[0][0], hb[0][1], 50 * 900, 0, TH, 1))
        with pytest.raises(lib.DockError) as e:
            while c.poll(big, timeout_us=100000) is None:
                pass
        assert e.value.status == lib.E_TOO_LARGE
        # and the context serves on
        _same(c.register(hb[0][0], hb[0][1], *REQS[0][1:3], TH, REQS[0][3]), alone[0])
    finally:
        c.close()


def test_injected_allocation_failures_leave_the_context_usable(lib, workload):
    w = workload("tiny32")
    ref = lib.Context(0)
    try:
        (ob, sw), = _handles(ref, [w])
        want = ref.register(ob, sw, 400, 100, TH, 2)
        held_ref, _, _ = ref.memory_stats()     # handles, scratch and the context's table caches
    finally:
        ref.close()
    c = lib.Context(0)
    try:
        # every allocation point of an object build fails once, then it builds
        failures = 0
        for n in range(1, 64):
            c.fail_allocation(n)
            try:
                ob = c.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
            except lib.DockError as e:
                assert e.status == lib.E_NOMEM and "injected" in str(e)
                failures += 1
                continue
            finally:
                c.fail_allocation(0)
            break
        assert failures >= 2
        sw = c.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
        # every allocation point of a first registration fails once
        failures = 0
        for n in range(1, 64):
            c.fail_allocation(n)
            try:
                got = c.register(ob, sw, 400, 100, TH, 2)
            except lib.DockError as e:
                assert e.status == lib.E_NOMEM
                failures += 1
                continue
            finally:
                c.fail_allocation(0)
            break
        assert failures >= 2
        _same(got, want)
        _same(c.register(ob, sw, 400, 100, TH, 2), want)
        # the same memory as a clean run: a failure that leaked (the object's
        # grids, a job's block) would have left it behind once per attempt
        assert c.memory_stats()[0] == held_ref
    finally:
        c.close()
