"""Swept-volume voxeliser (Sec. IV-A.2, Eq. (5)-(6)) against the FP64 oracle,
bit for bit, over many rotations: the identity and the quarter turns about
each axis (rows parallel to probe axes and cap planes take the fallback
paths) and seeded random rotations, on the 64^3 workload (2000 poses, 30 %
lifted off the surface) and the 128^3 workload (5000 poses).  The FP32 chord
ends of the kernel decide a voxel only outside their error band; this test
is what holds that band to the exact predicate over many rows."""
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
    c.close()


def _axis_turns():
    s = math.sqrt(0.5)
    return np.array([[1.0, 0, 0, 0], [s, s, 0, 0], [s, 0, s, 0], [s, 0, 0, s], [0.0, 1, 0, 0]])


@pytest.mark.parametrize("name,n_random", [("free64", 43), ("large128", 5)])
def test_swept_bits_equal_the_oracle_over_many_rotations(ctx, workload, name, n_random):
    w = workload(name)
    sw = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
    try:
        quats = np.concatenate([_axis_turns(), synth.random_unit_quats(n_random, 907)])
        bits, orig = sw.voxelise(quats)
        bad = []
        for i, q in enumerate(quats):
            S, o = O.sweep_grid(w.poses_world, q, w.h, w.N, w.radius, w.length)
            assert np.array_equal(orig[i], o)
            if not np.array_equal(bits[i], S):
                bad.append((i, int((bits[i] != S).sum())))
        assert not bad, bad
    finally:
        sw.close()
