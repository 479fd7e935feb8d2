"""Batched registration of uneven requests: requests of different lattice
sides, objects, trajectory lengths, probes, samplers and sample counts go
through one call; requests of equal lattice side share every search launch.
Each result must equal the same request registered alone."""
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
    _PAIRS.clear()
    c.close()


_PAIRS = []


def _pair(ctx, w, radius=None):
    ob = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    sw = ctx.sweep_grid(w.poses_world, radius or w.radius, w.length, w.h, w.N, contact=w.labels)
    _PAIRS.append((ob, sw))
    return ob, sw


def _same(a, b):
    assert a["best_search"]["rot"] == b["best_search"]["rot"]
    assert a["best_search"]["score"] == b["best_search"]["score"]
    assert np.array_equal(a["best_search"]["dk"], b["best_search"]["dk"])
    assert a["best_cand"] == b["best_cand"]
    assert a["n_evals"] == b["n_evals"]
    np.testing.assert_array_equal(a["q"], b["q"])
    np.testing.assert_array_equal(a["t"], b["t"])
    assert a["J"] == b["J"]


def test_uneven_batch_equals_requests_alone(ctx, workload):
    from paper_2605_21398_gb300 import dock
    w0 = workload("tiny32")
    w1 = workload("tiny32", replicate=1, poses=120)
    w2 = workload("free64")
    p0 = _pair(ctx, w0)
    p1 = _pair(ctx, w1)
    p1b = _pair(ctx, w1, radius=0.8)       # same trajectory, thinner probe
    p2 = _pair(ctx, w2)
    th = math.radians(5)
    reqs = [
        (p0[0], p0[1], 300, 100, th, 4),
        (p2[0], p2[1], 256, 64, th, 3),
        (p1[0], p1[1], 200, 0, th, 2),
        (p1b[0], p1b[1], 150, 50, math.radians(8), 5, dock.SAMPLER_HOPF),
        (p0[0], p0[1], 64, 32, th, 1),
    ]
    batch = ctx.register_batch(reqs)
    assert len(batch) == len(reqs)
    for rq, got in zip(reqs, batch):
        alone = ctx.register(rq[0], rq[1], rq[2], rq[3], rq[4], rq[5], *rq[6:])
        _same(got, alone)
    # a second batch in another order gives the same results
    again = ctx.register_batch(reqs[::-1])
    for a, b in zip(again[::-1], batch):
        _same(a, b)


def test_batch_rejects_bad_request_before_any_work(ctx, workload):
    from paper_2605_21398_gb300 import dock
    w0 = workload("tiny32")
    ob, sw = _pair(ctx, w0)
    with pytest.raises(dock.DockError):
        ctx.register_batch([(ob, sw, 100, 10, math.radians(5), 2), (ob, sw, 0, 10, math.radians(5), 2)])
    # the context is still usable
    r = ctx.register_batch([(ob, sw, 100, 10, math.radians(5), 2)])
    assert r[0]["n_evals"] == 110
