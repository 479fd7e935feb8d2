"""The allocation-free search entry point (dock_search_peaks_noalloc): its first
call leaves device memory unchanged, it refuses a capturing stream, its peaks
equal the per-rotation peaks of dock_search_so3 on the same rotations on two
calls in a row with different rotation sets, and its size limits."""
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
    _KEEP.clear()
    c.close()


_KEEP = []


def _pair(ctx, w, N=None):
    ob = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, N or w.N)
    sw = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, N or w.N, contact=w.labels)
    _KEEP.append((ob, sw))
    return ob, sw


def _quats(w, n, seed):
    q = synth.random_unit_quats(n, seed)
    q[0] = w.gt_q
    return q


def test_first_noalloc_call_leaves_device_memory_unchanged(ctx, workload):
    # the call's defining property: the first one on a device places nothing
    # (the scratch is already resident once a context exists).  Runs first in
    # this file so that no earlier call of the entry point hides a lazy load.
    torch = pytest.importorskip("torch")
    w = workload("tiny32")
    ob, sw = _pair(ctx, w)
    q = _quats(w, 6, 503)
    ctx.search_so3(ob, sw, len(q), 1, sampler=3, quats=q)   # the search kernels are loaded by now
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(0)[0]
    got = ctx.search_peaks_noalloc(ob, sw, q)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info(0)[0]
    assert free1 == free0, (free0, free1)
    assert np.all(np.isfinite(got["score"]))


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_noalloc_rejects_a_capturing_stream(workload):
    torch = pytest.importorskip("torch")
    from paper_2605_21398_gb300 import dock
    w = workload("tiny32")
    s = torch.cuda.Stream()
    c = dock.Context(0, stream=s.cuda_stream)
    try:
        ob, sw = _pair(c, w)
        q = _quats(w, 2, 504)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            with pytest.raises(dock.DockError, match="capturing"):
                c.search_peaks_noalloc(ob, sw, q)
        # usable once the capture has ended
        assert np.all(np.isfinite(c.search_peaks_noalloc(ob, sw, q)["score"]))
    finally:
        _KEEP.clear()
        c.close()


@pytest.mark.parametrize("name", ["tiny32", "free64"])
def test_noalloc_peaks_equal_search_peaks_on_two_calls(ctx, workload, name):
    w = workload(name)
    ob, sw = _pair(ctx, w)
    # a longer call, then a shorter one with other rotations: stale keys of
    # the first call must not leak into the second
    for n, seed in ((48, 501), (13, 502)):
        q = _quats(w, n, seed)
        _, ref = ctx.search_so3(ob, sw, n, top_k=1, sampler=3, quats=q, want_peaks=True)
        got = ctx.search_peaks_noalloc(ob, sw, q)
        tol = 1e-4 * np.max(np.abs(ref["score"]))
        assert np.all(np.abs(got["score"] - ref["score"]) <= tol + 1e-4 * np.abs(ref["score"]))
        assert np.array_equal(got["idx"], ref["idx"])


def test_noalloc_rejects_sizes_beyond_its_scratch(ctx, workload):
    from paper_2605_21398_gb300 import dock
    w = workload("tiny32")
    ob, sw = _pair(ctx, w)
    with pytest.raises(dock.DockError, match="rotation count"):
        ctx.search_peaks_noalloc(ob, sw, synth.random_unit_quats(4097, 7))
    ob96, sw96 = _pair(ctx, w, N=96)
    with pytest.raises(dock.DockError, match="lattice side"):
        ctx.search_peaks_noalloc(ob96, sw96, synth.random_unit_quats(2, 8))
    # still usable after the rejections
    q = _quats(w, 5, 9)
    _, ref = ctx.search_so3(ob, sw, 5, top_k=1, sampler=3, quats=q, want_peaks=True)
    got = ctx.search_peaks_noalloc(ob, sw, q)
    assert np.array_equal(got["idx"], ref["idx"])
