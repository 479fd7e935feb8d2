"""The z pass with its radix-16 DFT stages on the tensor cores (Eq. (9) as
dense products: 3 x TF32 tcgen05 products accumulated in FP32 in tensor
memory) against the FP64 oracle at canvas 256 (Eq. (7)): the full
correlation field within 1e-4 of max |C| and within FP32 accuracy (a small
multiple of the error of the FP32 butterfly path, which the split products
must not exceed by more than their own rounding); and a batch of two
requests with different objects, whose rotations share z-pass launches with
a spectrum tile that changes within a block, equal to each request
registered alone."""
import math

import numpy as np
import pytest

import oracle as O
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


_KEEP = {}


def _pair(ctx, w):
    key = (w.name, w.seed, len(w.poses_world))
    if key not in _KEEP:
        ob = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
        sw = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
        _KEEP[key] = (ob, sw)
    return _KEEP[key]


def test_full_field_matches_the_oracle_at_fp32_accuracy(ctx, workload):
    w = workload("large128")
    ob, sw = _pair(ctx, w)
    Go, _, _, fits = O.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    assert fits
    M = O.canvas_size(w.N)
    saved = ctx.get_tuning(w.N)
    try:
        for q in np.concatenate([[w.gt_q], synth.random_unit_quats(1, 77)]):
            S, _ = O.sweep_grid(w.poses_world, q, w.h, w.N, w.radius, w.length)
            Co = O.correlate_fft(Go, S, M)
            cmax = np.max(np.abs(Co))
            err = {}
            for tc in (0, 1):
                ctx.set_tuning(N=w.N, zpass_cols=16, zpass_tc=tc)
                assert ctx.get_tuning(w.N)["zpass_tc"] == tc
                err[tc] = np.max(np.abs(ctx.search_scores(ob, sw, q) - Co))
            print("max |C| %.1f, FP32 butterflies %.3g, 3 x TF32 products %.3g" % (cmax, err[0], err[1]))
            assert err[1] <= 1e-4 * cmax
            assert err[1] <= 3 * err[0] + 1e-6 * cmax, (err, cmax)
    finally:
        ctx.set_tuning(**saved)


def test_batch_of_two_objects_at_canvas_256_equals_requests_alone(ctx, workload):
    wa = workload("large128", poses=1200)
    wb = workload("large128", replicate=1, poses=900)
    pa, pb = _pair(ctx, wa), _pair(ctx, wb)
    th = math.radians(5)
    reqs = [(pa[0], pa[1], 70, 20, th, 2), (pb[0], pb[1], 50, 14, th, 2)]
    saved = ctx.get_tuning(wa.N)
    try:
        ctx.set_tuning(N=wa.N, zpass_cols=16, zpass_tc=1, batch=24, group=8)
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
