"""GPU parity of the label-aware score against the FP64 oracle.

Contact poses score O, poses labelled non-contact score min(O, 0) on the
voxels no contact pose reaches (the trajectory's non-contact evidence may
penalise overlap with the interior but earns no near-surface reward).  Bars
as in the plain search: split occupancy grids bit-exact, correlation within
1e-4 of max |C| per rotation, peak index exact wherever the oracle's top-two
gap exceeds twice that; requests without non-contact poses bit-identical to
the plain search.
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
    _KEEP.clear()
    _OBJ.clear()
    c.close()


_KEEP = []
_OBJ = {}


def _labels(w):
    # free64 carries its own labels (30 % of the poses on lifted retreat arcs,
    # labelled non-contact); tiny32 gets a seeded random 40 % non-contact
    if w.labels.min() == 0:
        return w.labels
    return (np.random.default_rng(w.seed + 5).random(len(w.labels)) >= 0.4).astype(np.uint8)


def _pair(ctx, w, labels, label_aware=True):
    if id(w) not in _OBJ:
        _OBJ[id(w)] = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    ob = _OBJ[id(w)]
    sw = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=labels)
    if label_aware:
        sw.set_label_aware(True)
    _KEEP.append(sw)
    return ob, sw


def _second_best(C, idx):
    flat = C.reshape(-1).copy()
    flat[idx] = -np.inf
    return float(flat.max())


@pytest.mark.parametrize("name,nrot", [("tiny32", 4), ("free64", 3)])
def test_label_split_grids_are_bit_exact(ctx, workload, name, nrot):
    w = workload(name)
    lab = _labels(w)
    _, sw = _pair(ctx, w, lab)
    q = np.concatenate([[w.gt_q], synth.random_unit_quats(nrot - 1, 78)])
    bc, bn, orig = sw.voxelise_labels(q)
    for i in range(nrot):
        S_c, S_n, o = O.sweep_grids_by_label(w.poses_world, lab, q[i], w.h, w.N, w.radius, w.length)
        assert np.array_equal(orig[i], o)
        assert S_c.sum() > 0 and S_n.sum() > 0
        assert np.array_equal(bc[i], S_c), (i, int((bc[i] != S_c).sum()))
        assert np.array_equal(bn[i], S_n), (i, int((bn[i] != S_n).sum()))


@pytest.mark.parametrize("name", ["tiny32", "free64"])
def test_label_aware_field_matches_oracle(ctx, workload, name):
    w = workload(name)
    lab = _labels(w)
    ob, sw = _pair(ctx, w, lab)
    Go, _, _, _ = O.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    M = O.canvas_size(w.N)
    for q in [w.gt_q, synth.random_unit_quats(1, 6)[0]]:
        C = ctx.search_scores(ob, sw, q)
        S_c, S_n, _ = O.sweep_grids_by_label(w.poses_world, lab, q, w.h, w.N, w.radius, w.length)
        Co = O.correlate_label_aware(Go, S_c, S_n, M)
        tol = 1e-4 * np.max(np.abs(Co))
        assert np.max(np.abs(C - Co)) <= tol
        # the label-aware field lies below the plain one and differs from it
        Cp = O.correlate_fft(Go, (S_c | S_n), M)
        assert np.max(Cp - Co) > 1.0 and np.min(Cp - Co) > -1e-9 * np.max(np.abs(Cp))


@pytest.mark.parametrize("name,n", [("tiny32", 96), ("free64", 24)])
def test_label_aware_peaks_and_top_k_match_oracle(ctx, workload, name, n):
    w = workload(name)
    lab = _labels(w)
    ob, sw = _pair(ctx, w, lab)
    Go, oo, _, _ = O.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    M = O.canvas_size(w.N)
    quats = synth.random_unit_quats(n, 12)
    quats[0] = w.gt_q
    K = min(8, n)
    cands, peaks = ctx.search_so3(ob, sw, n, K, sampler=3, quats=quats, want_peaks=True)
    res = O.search_label_aware(Go, oo, w.poses_world, lab, quats, w.h, w.N, w.radius, w.length)
    scores, tols, gaps = [], [], []
    for i, r in enumerate(res):
        tol = 1e-4 * np.max(np.abs(r["C"]))
        gap = r["score"] - _second_best(r["C"], r["idx"])
        assert abs(peaks["score"][i] - r["score"]) <= tol + 1e-4 * abs(r["score"]), i
        if gap > 2 * tol:
            assert peaks["idx"][i] == r["idx"], i
        scores.append(r["score"])
        tols.append(tol)
        gaps.append(gap)
    scores, tols = np.array(scores), np.array(tols)
    order = O.top_k(scores, K)
    for k, c in enumerate(cands):
        i = order[k]
        sep_prev = k == 0 or scores[order[k - 1]] - scores[i] > 2 * (tols[i] + tols[order[k - 1]])
        sep_next = k == K - 1 or scores[i] - scores[order[k + 1]] > 2 * (tols[i] + tols[order[k + 1]])
        if sep_prev and sep_next and gaps[i] > 2 * tols[i]:
            assert c["rot"] == i
            dk = O.canvas_shift(res[i]["idx"], M, w.N)
            assert np.array_equal(c["dk"], dk)
            _, t = O.pose_from_peak(quats[i], dk, w.h, res[i]["o_s"], oo)
            assert np.allclose(c["t"], t, atol=1e-9)


def test_all_contact_labels_give_the_plain_search_bit_for_bit(ctx, workload):
    w = workload("tiny32")
    ones = np.ones(len(w.poses_world), np.uint8)
    ob, sw_la = _pair(ctx, w, ones, label_aware=True)
    _, sw_pl = _pair(ctx, w, ones, label_aware=False)
    _, pa = ctx.search_so3(ob, sw_la, 64, 8, want_peaks=True)
    _, pb = ctx.search_so3(ob, sw_pl, 64, 8, want_peaks=True)
    assert np.array_equal(pa, pb)


def test_switching_label_aware_off_restores_the_plain_search(ctx, workload):
    w = workload("tiny32")
    lab = _labels(w)
    ob, sw = _pair(ctx, w, lab)
    _, p_la = ctx.search_so3(ob, sw, 48, 4, want_peaks=True)
    sw.set_label_aware(False)
    _, p_off = ctx.search_so3(ob, sw, 48, 4, want_peaks=True)
    _, p_pl = ctx.search_so3(ob, _pair(ctx, w, lab, label_aware=False)[1], 48, 4, want_peaks=True)
    assert np.array_equal(p_off, p_pl)
    assert not np.array_equal(p_la, p_off)


def test_all_non_contact_labels_reward_nothing(ctx, workload):
    # C = corr(min(O, 0), S) <= 0, and a shift that overlaps no interior voxel
    # scores 0, so every rotation's peak is 0 up to the FP32 tolerance
    w = workload("tiny32")
    ob, sw = _pair(ctx, w, np.zeros(len(w.poses_world), np.uint8))
    quats = np.concatenate([[w.gt_q], synth.random_unit_quats(3, 8)])
    _, pk = ctx.search_so3(ob, sw, len(quats), 2, sampler=3, quats=quats, want_peaks=True)
    for i, q in enumerate(quats):
        C = ctx.search_scores(ob, sw, q)
        tol = 1e-4 * np.abs(C).max()
        assert C.max() <= tol and C.min() < -1.0
        assert abs(pk["score"][i]) <= tol


def test_plain_request_sharing_a_pass_with_a_label_aware_one_is_unchanged(ctx, workload):
    # the pass runs the two-grid pipeline for both; the plain request adds no
    # second term, so its result equals the request registered alone
    w = workload("tiny32")
    lab = _labels(w)
    ob, sw_la = _pair(ctx, w, lab)
    _, sw_pl = _pair(ctx, w, lab, label_aware=False)
    th = math.radians(5)
    batch = ctx.register_batch([(ob, sw_la, 200, 50, th, 2), (ob, sw_pl, 200, 50, th, 2)])
    alone_pl = ctx.register(ob, sw_pl, 200, 50, th, 2)
    alone_la = ctx.register(ob, sw_la, 200, 50, th, 2)
    for got, ref in [(batch[1], alone_pl), (batch[0], alone_la)]:
        assert got["best_search"]["rot"] == ref["best_search"]["rot"]
        assert got["best_search"]["score"] == ref["best_search"]["score"]
        np.testing.assert_array_equal(got["q"], ref["q"])
        np.testing.assert_array_equal(got["t"], ref["t"])
        assert got["J"] == ref["J"]


def test_label_aware_sweep_is_rejected_by_the_no_alloc_search(ctx, workload):
    from paper_2605_21398_gb300 import dock
    w = workload("tiny32")
    ob, sw = _pair(ctx, w, _labels(w))
    with pytest.raises(dock.DockError):
        ctx.search_peaks_noalloc(ob, sw, synth.random_unit_quats(4, 1))
    sw.set_label_aware(False)
    assert len(ctx.search_peaks_noalloc(ob, sw, synth.random_unit_quats(4, 1))) == 4


def test_bad_label_aware_flag_is_rejected(ctx, workload):
    from paper_2605_21398_gb300 import dock
    w = workload("tiny32")
    _, sw = _pair(ctx, w, _labels(w), label_aware=False)
    assert dock.lib().dock_sweep_set_label_aware(ctx.h, sw.h, 2) != 0
    sw.set_label_aware(True)
    sw.set_label_aware(False)


@pytest.mark.parametrize("N,runs,zc", [(96, 0, 0), (128, 0, 16), (128, 1, 16), (128, 1, 32)])
def test_label_aware_parity_on_the_192_and_256_canvases(ctx, workload, N, runs, zc):
    # the dual z pass on the radix-3 (192) and 256 canvases: split grids,
    # field and peaks against the oracle (30 % retreat poses non-contact);
    # at 256 with the forward pass over whole slabs or from run lists (its
    # masked grid too) and the dual z pass over 16 or 32 columns per block
    w = workload("free64", N=N, h=16.0 / N, poses=300, n_theta=48, n_phi=96, lines=3, noncontact=0.3)
    shape0 = ctx.get_tuning(N)
    ctx.set_tuning(N=N, fwd_runs=runs, zpass_cols=zc)
    try:
        _label_aware_parity(ctx, w, N)
    finally:
        ctx.set_tuning(**shape0)


def _label_aware_parity(ctx, w, N):
    lab = w.labels
    assert 0 < int((lab == 0).sum()) < len(lab)
    ob, sw = _pair(ctx, w, lab)
    Go, oo, _, fits = O.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    assert fits
    M = O.canvas_size(N)
    quats = np.concatenate([[w.gt_q], synth.random_unit_quats(2, 32)])
    bc, bn, _ = sw.voxelise_labels(quats)
    _, peaks = ctx.search_so3(ob, sw, len(quats), 2, sampler=3, quats=quats, want_peaks=True)
    for i, q in enumerate(quats):
        S_c, S_n, _ = O.sweep_grids_by_label(w.poses_world, lab, q, w.h, w.N, w.radius, w.length)
        assert np.array_equal(bc[i], S_c) and np.array_equal(bn[i], S_n)
        Co = O.correlate_label_aware(Go, S_c, S_n, M)
        sc, idx = O.peak(Co)
        tol = 1e-4 * np.max(np.abs(Co))
        assert abs(peaks["score"][i] - sc) <= tol + 1e-4 * abs(sc), i
        if sc - _second_best(Co, idx) > 2 * tol:
            assert peaks["idx"][i] == idx, i
    C = ctx.search_scores(ob, sw, quats[0])
    S_c, S_n, _ = O.sweep_grids_by_label(w.poses_world, lab, quats[0], w.h, w.N, w.radius, w.length)
    Co = O.correlate_label_aware(Go, S_c, S_n, M)
    assert np.max(np.abs(C - Co)) <= 1e-4 * np.max(np.abs(Co))
