"""The persistent cluster plane pass with TMA staging (canvas 256, 4 or 8 CTAs
per plane: clusters walk the planes of a launch, the tensor-memory-access unit
loads the next plane's columns while the current plane's C2R runs) does the
arithmetic of the one-cluster-per-plane pass in the same order, so over full
launches -- every cluster through hundreds of planes, every mbarrier phase
reused -- its peaks equal that pass's bit for bit (the oracle parity of both
is in test_gpu_plane_variants); and a batch of two objects at canvas 256,
whose planes interleave requests, equals each request registered alone."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2605_21398_gb300 import build, dock
    build.build()
    c = dock.Context(0)
    yield c
    _KEEP.clear()
    c.close()


_KEEP = {}


def _pair(ctx, w):
    key = (w.name, w.seed, len(w.poses_world))
    if key not in _KEEP:
        ob = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
        sw = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
        _KEEP[key] = (ob, sw)
    return _KEEP[key]


@pytest.mark.parametrize("cl", [4, 8])
def test_persistent_plane_pass_equals_one_cluster_per_plane_over_full_launches(ctx, workload, cl):
    w = workload("large128")
    ob, sw = _pair(ctx, w)
    saved = ctx.get_tuning(w.N)
    got = {}
    try:
        for tma in (0, 1):
            ctx.set_tuning(N=w.N, plane_cl=cl, zpass_cols=16, zpass_tc=0, plane_tma=tma, batch=42)
            _, pk = ctx.search_so3(ob, sw, 200, 4, want_peaks=True)
            got[tma] = pk
    finally:
        ctx.set_tuning(**saved)
    np.testing.assert_array_equal(got[1]["idx"], got[0]["idx"])
    np.testing.assert_array_equal(got[1]["score"], got[0]["score"])


def test_batch_of_two_objects_equals_requests_alone(ctx, workload):
    wa = workload("large128", poses=1200)
    wb = workload("large128", replicate=1, poses=900)
    pa, pb = _pair(ctx, wa), _pair(ctx, wb)
    th = math.radians(5)
    reqs = [(pa[0], pa[1], 70, 20, th, 2), (pb[0], pb[1], 50, 14, th, 2)]
    saved = ctx.get_tuning(wa.N)
    try:
        ctx.set_tuning(N=wa.N, plane_cl=4, zpass_cols=16, zpass_tc=0, plane_tma=1, batch=24)
        batch = ctx.register_batch(reqs)
        for rq, got in zip(reqs, batch):
            alone = ctx.register(*rq)
            assert got["best_search"]["rot"] == alone["best_search"]["rot"]
            assert got["best_search"]["score"] == alone["best_search"]["score"]
            np.testing.assert_array_equal(got["q"], alone["q"])
            np.testing.assert_array_equal(got["t"], alone["t"])
            assert got["J"] == alone["J"]
    finally:
        ctx.set_tuning(**saved)
