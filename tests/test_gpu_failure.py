"""Failure detection on the GPU without a fault: the cluster plane pass waits
for its peers' blocks on an mbarrier with a bound of about a second of clock
cycles.  The test hook launches it with those blocks withheld (a wait that
nothing satisfies); every CTA's wait runs out, the kernel records
DOCK_E_TIMEOUT in the context's error word and returns, and the call reports
it.  In the persistent form the CTAs whose waits ran out stop their whole
cluster at its next cluster barrier (the stop flag written into every CTA's
shared memory first), so no CTA waits at a barrier a peer never reaches.
Nothing is in flight when a CTA gives up, and the context then serves the
same results as before."""
import time

import numpy as np
import pytest

from paper_2605_21398_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2605_21398_gb300 import build, dock
    build.build()
    c = dock.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("cl,tma", [(4, 0), (8, 1)])
def test_plane_pass_wait_runs_out_and_the_context_serves_on(ctx, workload, cl, tma):
    from paper_2605_21398_gb300 import dock
    w = workload("large128")
    ob = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    sw = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
    shape0 = ctx.get_tuning(w.N)
    ctx.set_tuning(N=w.N, plane_cl=cl, plane_tma=tma)
    try:
        q = synth.random_unit_quats(1, 31)[0]
        before = ctx.search_scores(ob, sw, q)
        t0 = time.perf_counter()
        with pytest.raises(dock.DockError) as e:
            ctx.test_plane_timeout(ob, sw, q)
        waited = time.perf_counter() - t0
        assert e.value.status == dock.E_TIMEOUT
        assert waited >= 0.5, waited          # the bounded waits ran out rather than failing at once
        after = ctx.search_scores(ob, sw, q)
        assert np.array_equal(before, after)
        cands = ctx.search_so3(ob, sw, 4, 2)
        assert cands[0]["rot"] >= 0
        # other shapes have no such wait: the hook refuses them
        saved = ctx.get_tuning(w.N)
        try:
            ctx.set_tuning(N=w.N, plane_cl=2)
            with pytest.raises(dock.DockError) as e2:
                ctx.test_plane_timeout(ob, sw, q)
            assert e2.value.status == dock.E_INVALID
        finally:
            ctx.set_tuning(**saved)
    finally:
        ctx.set_tuning(**shape0)
        ob.close()
        sw.close()
