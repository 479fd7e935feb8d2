"""GPU parity of the docking search (Sec. IV) against the FP64 oracle.

Bars (per the stated tolerances): object grid O within one FP32 ulp of the
oracle's FP64 value rounded to FP32; swept occupancy bits and voxel indices
bit-exact; correlation scores within 1e-4 of max |C| per rotation; the peak
index exact whenever the oracle's top-two gap exceeds twice that tolerance.
"""
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
    _OBJ.clear()
    c.close()


_OBJ = {}


def _gpu_pair(ctx, w):
    key = (w.name, w.seed, w.N, w.h, len(w.poses_world))
    if key not in _OBJ:
        ob = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
        sw = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
        _OBJ[key] = (ob, sw)
    return _OBJ[key]


def _ulp_diff(a, b):
    a = np.asarray(a, dtype=np.float32).view(np.int32).astype(np.int64)
    b = np.asarray(b, dtype=np.float32).view(np.int32).astype(np.int64)
    a = np.where(a < 0, -(a & 0x7FFFFFFF), a)
    b = np.where(b < 0, -(b & 0x7FFFFFFF), b)
    return np.abs(a - b)


@pytest.mark.parametrize("name", ["tiny32", "free64"])
def test_object_grid_matches_oracle(ctx, workload, name):
    w = workload(name)
    ob, _ = _gpu_pair(ctx, w)
    G, o = ob.export_grid()
    Go, oo, f, fits = O.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    assert fits
    assert np.array_equal(o, oo)
    d = _ulp_diff(G, Go.astype(np.float32))
    assert d.max() <= 1, (d.max(), np.argwhere(d > 1)[:5])


def test_object_grid_with_touchable_sub_mesh_matches_oracle(ctx, workload):
    # Eq. (2) with a touchable sub-mesh: the triangles facing +z (upper
    # cap of the object) are touchable, the rest only bound the inside
    w = workload("tiny32")
    V, T = w.obj.verts, w.obj.tris
    nz = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])[:, 2]
    touch = (nz > 0).astype(np.uint8)
    assert 0 < touch.sum() < len(T)
    ob = ctx.object_grid(V, T, w.h, w.N, touchable=touch)
    try:
        G, o = ob.export_grid()
        Go, oo, _, fits = O.object_grid(V, T, w.h, w.N, touch=touch)
        assert fits and np.array_equal(o, oo)
        d = _ulp_diff(G, Go.astype(np.float32))
        assert d.max() <= 1, (d.max(), np.argwhere(d > 1)[:5])
        Gall, _, _, _ = O.object_grid(V, T, w.h, w.N)
        assert np.count_nonzero(Go != Gall) > 0      # the mask changes the grid
    finally:
        ob.close()


@pytest.mark.parametrize("name,nrot", [("tiny32", 6), ("free64", 3)])
def test_voxelised_swept_grid_is_bit_exact(ctx, workload, name, nrot):
    w = workload(name)
    _, sw = _gpu_pair(ctx, w)
    q = np.concatenate([[w.gt_q], synth.random_unit_quats(nrot - 1, 77)])
    bits, orig = sw.voxelise(q)
    for i in range(nrot):
        S, o = O.sweep_grid(w.poses_world, q[i], w.h, w.N, w.radius, w.length)
        assert np.array_equal(orig[i], o)
        assert S.sum() > 0
        assert np.array_equal(bits[i], S), (i, int((bits[i] != S).sum()))


def _second_best(C, idx):
    flat = C.reshape(-1).copy()
    flat[idx] = -np.inf
    return float(flat.max())


@pytest.mark.parametrize("name", ["tiny32", "free64"])
def test_full_correlation_field_matches_oracle(ctx, workload, name):
    w = workload(name)
    ob, sw = _gpu_pair(ctx, w)
    Go, oo, _, _ = O.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    M = O.canvas_size(w.N)
    for q in [w.gt_q, synth.random_unit_quats(1, 5)[0]]:
        C = ctx.search_scores(ob, sw, q)
        S, _ = O.sweep_grid(w.poses_world, q, w.h, w.N, w.radius, w.length)
        Co = O.correlate_fft(Go, S, M)
        tol = 1e-4 * np.max(np.abs(Co))
        assert np.max(np.abs(C - Co)) <= tol


@pytest.mark.parametrize("name,n", [("tiny32", 512), ("free64", 48)])
def test_search_peaks_and_top_k_match_oracle(ctx, workload, name, n):
    w = workload(name)
    ob, sw = _gpu_pair(ctx, w)
    Go, oo, _, _ = O.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    M = O.canvas_size(w.N)
    quats = O.super_fibonacci(n) if name == "tiny32" else synth.random_unit_quats(n, 11)
    quats[0] = w.gt_q
    K = min(w.top_k, n)
    cands, peaks = ctx.search_so3(ob, sw, n, K, sampler=3, quats=quats, want_peaks=True)
    ref = []
    for i, q in enumerate(quats):
        S, o_s = O.sweep_grid(w.poses_world, q, w.h, w.N, w.radius, w.length)
        C = O.correlate_fft(Go, S, M)
        sc, idx = O.peak(C)
        tol = 1e-4 * np.max(np.abs(C))
        ref.append((sc, idx, tol, sc - _second_best(C, idx), o_s))
        assert abs(peaks["score"][i] - sc) <= tol + 1e-4 * abs(sc), i
        if ref[-1][3] > 2 * tol:
            assert peaks["idx"][i] == idx, i
    # top-K over rotations: same order wherever consecutive scores are separated
    scores = np.array([r[0] for r in ref])
    order = O.top_k(scores, K)
    tols = np.array([r[2] for r in ref])
    for k, c in enumerate(cands):
        i = order[k]
        sep_prev = k == 0 or scores[order[k - 1]] - scores[i] > 2 * (tols[i] + tols[order[k - 1]])
        sep_next = k == K - 1 or scores[i] - scores[order[k + 1]] > 2 * (tols[i] + tols[order[k + 1]])
        if sep_prev and sep_next and ref[i][3] > 2 * ref[i][2]:
            assert c["rot"] == i
            dk = O.canvas_shift(ref[i][1], M, w.N)
            assert np.array_equal(c["dk"], dk)
            _, t = O.pose_from_peak(quats[i], dk, w.h, ref[i][4], oo)
            assert np.allclose(c["t"], t, atol=1e-9)
            assert np.allclose(c["q"], quats[i])


def test_planted_rotation_wins_the_search(ctx, workload):
    # at 64^3 / 0.25 mm (band = 2 voxels) the planted orientation out-scores
    # random ones; at 32^3 / 0.5 mm the one-voxel band does not discriminate
    w = workload("free64")
    ob, sw = _gpu_pair(ctx, w)
    quats = np.concatenate([[w.gt_q], synth.random_unit_quats(127, 3)])
    cands = ctx.search_so3(ob, sw, len(quats), 8, sampler=3, quats=quats)
    assert cands[0]["rot"] == 0
    assert np.linalg.norm(cands[0]["t"] - w.gt_t) <= 2 * math.sqrt(3) * w.h


def test_rotation_shards_merge_to_the_unsharded_top_k(ctx, workload):
    w = workload("tiny32")
    ob, sw = _gpu_pair(ctx, w)
    n, K = 200, 8
    full = ctx.search_so3(ob, sw, n, K)
    _, pk = ctx.search_so3(ob, sw, n, K, want_peaks=True)
    merged = []
    for r in [(0, 70), (70, 150), (150, 200)]:
        c, p = ctx.search_so3(ob, sw, n, K, rot_range=r, want_peaks=True)
        merged += [(x["score"], x["rot"]) for x in c if x["rot"] >= 0]
        assert np.array_equal(p["score"][r[0]:r[1]], pk["score"][r[0]:r[1]])
    merged.sort(key=lambda t: (-t[0], t[1]))
    assert [m[1] for m in merged[:K]] == [c["rot"] for c in full]


def test_contact_labels_do_not_change_the_search(ctx, workload):
    from paper_2605_21398_gb300 import dock
    w = workload("tiny32")
    ob, _ = _gpu_pair(ctx, w)
    sw1 = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=np.ones(len(w.labels), np.uint8))
    flipped = (np.random.default_rng(0).random(len(w.labels)) < 0.5).astype(np.uint8)
    sw2 = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=flipped)
    a, pa = ctx.search_so3(ob, sw1, 64, 8, want_peaks=True)
    b, pb = ctx.search_so3(ob, sw2, 64, 8, want_peaks=True)
    assert np.array_equal(pa, pb)


def test_samplers_match_oracle(ctx):
    from paper_2605_21398_gb300 import dock
    assert np.allclose(dock.sample_so3(1000, dock.SAMPLER_SF), O.super_fibonacci(1000), atol=1e-13)
    assert np.allclose(dock.sample_so3(300, dock.SAMPLER_HOPF), O.hopf_halton(300), atol=1e-13)
    q0 = synth.random_unit_quats(1, 9)[0]
    g = dock.sample_so3(500, dock.SAMPLER_GEOBALL, q0=q0, theta=math.radians(5))
    assert np.allclose(g, O.geoball_sf(500, q0, math.radians(5)), atol=1e-12)


def test_empty_swept_grid_gives_zero_scores_and_index_zero(ctx, workload):
    w = workload("tiny32")
    ob, _ = _gpu_pair(ctx, w)
    # a probe far smaller than a voxel covers no lattice point
    sw = ctx.sweep_grid(w.poses_world[:1], 1e-3, 1e-3, w.h, w.N)
    C = ctx.search_scores(ob, sw, np.array([1.0, 0, 0, 0]))
    assert np.all(C == 0)
    c, p = ctx.search_so3(ob, sw, 4, 2, want_peaks=True)
    assert np.all(p["score"] == 0) and np.all(p["idx"] == 0)


def test_invalid_inputs_are_rejected(ctx, workload):
    from paper_2605_21398_gb300 import dock
    w = workload("tiny32")
    bad = w.poses_world.copy()
    bad[3, :4] *= 1.01
    with pytest.raises(dock.DockError) as e:
        ctx.sweep_grid(bad, w.radius, w.length, w.h, w.N)
    assert e.value.status == dock.E_INVALID
    with pytest.raises(dock.DockError):
        ctx.sweep_grid(w.poses_world[:0], w.radius, w.length, w.h, w.N)
    with pytest.raises(dock.DockError):
        ctx.object_grid(w.obj.verts, w.obj.tris, w.h, 48)
    with pytest.raises(dock.DockError):
        ctx.object_grid(w.obj.verts * 3.0, w.obj.tris, w.h, w.N)   # does not fit the lattice
    ob, sw = _gpu_pair(ctx, w)
    with pytest.raises(dock.DockError):
        ctx.search_so3(ob, sw, 10, 0)
    qbad = np.array([[1.0, 0.1, 0, 0]])
    with pytest.raises(dock.DockError):
        ctx.search_so3(ob, sw, 1, 1, sampler=3, quats=qbad)


def test_large_lattice_sampled_parity(ctx, workload):
    # 128^3 lattice in the bench's launch configuration: bits exact for sampled
    # rotations, scores at the peak and at random shifts by the direct sum of
    # Eq. (7), the peak score against the oracle's FFT field.
    w = workload("large128")
    ob, sw = _gpu_pair(ctx, w)
    Go, oo, _, fits = O.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    assert fits
    G, o = ob.export_grid()
    assert np.array_equal(o, oo)
    assert _ulp_diff(G, Go.astype(np.float32)).max() <= 1
    M = O.canvas_size(w.N)
    quats = np.concatenate([[w.gt_q], synth.random_unit_quats(2, 21)])
    bits, orig = sw.voxelise(quats)
    cands, peaks = ctx.search_so3(ob, sw, len(quats), 3, sampler=3, quats=quats, want_peaks=True)
    rng = np.random.default_rng(4)
    for i, q in enumerate(quats):
        S, o_s = O.sweep_grid(w.poses_world, q, w.h, w.N, w.radius, w.length)
        assert np.array_equal(bits[i], S)
        C = O.correlate_fft(Go, S, M)
        sc, idx = O.peak(C)
        tol = 1e-4 * np.max(np.abs(C))
        assert abs(peaks["score"][i] - sc) <= tol + 1e-4 * abs(sc)
        if sc - _second_best(C, idx) > 2 * tol:
            assert peaks["idx"][i] == idx
        # at 128^3 the top of the field is flatter than the FP32 error, so the
        # gap test rarely holds: the chosen shift must then be one of the
        # oracle's maxima within the tolerance
        assert C.reshape(-1)[peaks["idx"][i]] >= sc - 2 * tol
        # direct Eq. (7) at a few shifts agrees with the FFT field
        N = w.N
        for _ in range(3):
            dk = rng.integers(-N // 2, N // 2, size=3)
            acc = 0.0
            zs = slice(max(0, -dk[2]), min(N, N - dk[2]))
            ys = slice(max(0, -dk[1]), min(N, N - dk[1]))
            xs = slice(max(0, -dk[0]), min(N, N - dk[0]))
            acc = float(np.sum(Go[zs, ys, xs] * S[zs.start + dk[2]:zs.stop + dk[2], ys.start + dk[1]:ys.stop + dk[1],
                                                   xs.start + dk[0]:xs.stop + dk[0]]))
            c = [(d + M) % M for d in dk]
            assert abs(C[c[2], c[1], c[0]] - acc) <= 1e-9 * max(1.0, abs(acc))


def test_n96_lattice_sampled_parity(ctx, workload):
    # 96^3 lattice (canvas 192^3, the radix-3 plans): bits exact and peaks
    # against the oracle's FFT field for two rotations
    w = workload("free64", N=96, h=16.0 / 96, poses=300, n_theta=48, n_phi=96, lines=3, noncontact=0.0)
    ob, sw = _gpu_pair(ctx, w)
    Go, oo, _, fits = O.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    assert fits
    M = O.canvas_size(w.N)
    assert M == 192
    quats = np.concatenate([[w.gt_q], synth.random_unit_quats(1, 23)])
    bits, orig = sw.voxelise(quats)
    cands, peaks = ctx.search_so3(ob, sw, len(quats), 2, sampler=3, quats=quats, want_peaks=True)
    for i, q in enumerate(quats):
        S, o_s = O.sweep_grid(w.poses_world, q, w.h, w.N, w.radius, w.length)
        assert np.array_equal(bits[i], S)
        C = O.correlate_fft(Go, S, M)
        sc, idx = O.peak(C)
        tol = 1e-4 * np.max(np.abs(C))
        assert abs(peaks["score"][i] - sc) <= tol + 1e-4 * abs(sc)
        if sc - _second_best(C, idx) > 2 * tol:
            assert peaks["idx"][i] == idx
