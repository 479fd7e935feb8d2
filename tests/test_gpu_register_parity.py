"""The three-stage registration (Fig. 2; Sec. IV-C, IV-D, V-C) on the GPU
against the oracle's `register`, stage by stage: global Super-Fibonacci peaks,
the local GeoBall-SF stage about the best global rotation, the merged top-K
(score descending, sample index ascending), the refined candidates and the
lowest-J winner; and dock_register end to end against those stages.  The
workload plants a rotation on a global sample (noise-free 64^3 raster, 600
poses), so that the discrete choices are clear of the FP32 tolerance."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2605_21398_gb300 import synth

pytestmark = pytest.mark.gpu

NG, NL, K, J_PLANT = 96, 24, 2, 37
THETA = math.radians(5.0)


@pytest.fixture(scope="module")
def ctx():
    from paper_2605_21398_gb300 import build, dock
    build.build()
    c = dock.Context(0)
    yield c
    c.close()


def _planted():
    w = synth.make_workload("free64", poses=600, noncontact=0.0, noise_t=0.0, noise_r=0.0)
    qp = O.super_fibonacci(NG)[J_PLANT]
    tp = np.array([0.7, -1.1, 0.4])
    return w, qp, tp, synth.transform_poses(qp, tp, w.traj.poses_obj)


def _pose_err(Ra, ta, Rb, tb, a):
    # rotation angle from |Ra - Rb|_F = 2 sqrt(2) sin(angle / 2): exact near 0,
    # where acos((trace - 1) / 2) loses half the digits
    dt = np.linalg.norm((Ra @ a + ta) - (Rb @ a + tb))
    s = min(1.0, np.linalg.norm(Ra - Rb) / (2.0 * math.sqrt(2.0)))
    return dt, math.degrees(2.0 * math.asin(s))


def _check_peaks(gpu, orc, label):
    for i, p in enumerate(orc):
        tol = 1e-4 * p["cmax"]
        assert abs(gpu["score"][i] - p["score"]) <= tol + 1e-4 * abs(p["score"]), (label, i)


def test_three_stage_registration_matches_the_oracle(ctx):
    from paper_2605_21398_gb300 import dock
    w, qp, tp, poses = _planted()
    prm = O.refine_params(w.radius, w.length)
    ref = O.register(w.obj.verts, w.obj.tris, poses, w.h, w.N, w.radius, w.length, NG, NL, THETA, K, prm,
                     workers=os.cpu_count() or 1)
    ob = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    sw = ctx.sweep_grid(poses, w.radius, w.length, w.h, w.N)
    try:
        # stage 1: global peaks; the best global sample is clear of the tolerance
        cg, pg = ctx.search_so3(ob, sw, NG, K, sampler=dock.SAMPLER_SF, want_peaks=True)
        _check_peaks(pg, ref["peaks"][:NG], "global")
        sg = np.array([p["score"] for p in ref["peaks"][:NG]])
        top2 = np.sort(sg)[::-1][:2]
        assert top2[0] - top2[1] > 2 * 1e-4 * ref["peaks"][ref["best_global"]]["cmax"]
        assert cg[0]["rot"] == ref["best_global"] == J_PLANT
        assert np.allclose(cg[0]["q"], ref["quats"][J_PLANT], atol=1e-15)
        # stage 2: local peaks about the same rotation
        cl, pl = ctx.search_so3(ob, sw, NL, K, sampler=dock.SAMPLER_GEOBALL, q0=cg[0]["q"], theta=THETA,
                                want_peaks=True)
        _check_peaks(pl, ref["peaks"][NG:], "local")
        # merged top-K: the oracle's order, every consecutive gap clear of the tolerance
        allsc = np.array([p["score"] for p in ref["peaks"]])
        tolk = 2 * 1e-4 * max(p["cmax"] for p in ref["peaks"])
        ranked = np.sort(allsc)[::-1]
        assert np.all(ranked[:K] - ranked[1:K + 1] > tolk)
        gsc = np.concatenate([pg["score"], pl["score"]])
        gorder = np.lexsort((np.arange(len(gsc)), -gsc))[:K]
        assert np.array_equal(gorder, ref["order"])
        byrot = {c["rot"]: c for c in cg if c["rot"] >= 0}
        byrot.update({NG + c["rot"]: c for c in cl if c["rot"] >= 0})
        cands = [byrot[int(i)] for i in gorder]
        a = ref["anchor"]
        for c, rc in zip(cands, ref["cands"]):
            assert np.array_equal(np.asarray(c["dk"]), rc["dk"])
            dt, dr = _pose_err(O.quat_to_mat(c["q"]), np.asarray(c["t"]), rc["R0"], rc["t0"], a)
            assert dt <= 1e-9 and dr <= 1e-9
        # stage 3: refinement of the candidates and the lowest-J winner
        out = ctx.refine_se3(ob, sw, cands)
        for o, rc in zip(out, ref["cands"]):
            dt, dr = _pose_err(O.quat_to_mat(o["q"]), np.asarray(o["t"]), rc["R"], rc["p"], a)
            assert dt <= 1e-3 and dr <= 1e-3, (dt, dr)
            assert abs(o["J"] - rc["J"]) <= 1e-3 * max(1.0, abs(rc["J"]))
        Js = np.array([o["J"] for o in out])
        Jo = np.array([rc["J"] for rc in ref["cands"]])
        # the winner is unique when the oracle's gap exceeds the GPU's J errors
        # on both sides of it; then the GPU must pick the same candidate
        assert np.sort(Jo)[1] - np.sort(Jo)[0] > 2 * np.max(np.abs(Js - Jo))
        best = int(np.lexsort((np.arange(K), Js))[0])
        assert best == ref["best"]
        # dock_register runs the same stages
        res = ctx.register(ob, sw, NG, NL, THETA, K)
        assert res["best_cand"] == ref["best"] and res["n_evals"] == NG + NL
        dt, dr = _pose_err(O.quat_to_mat(res["q"]), np.asarray(res["t"]), O.quat_to_mat(out[best]["q"]),
                           np.asarray(out[best]["t"]), a)
        assert dt <= 1e-9 and dr <= 1e-7
        rb = ref["cands"][ref["best"]]
        dt, dr = _pose_err(O.quat_to_mat(res["q"]), np.asarray(res["t"]), rb["R"], rb["p"], a)
        assert dt <= 1e-3 and dr <= 1e-3, (dt, dr)
        # and lands on the planted pose
        dt, dr = _pose_err(O.quat_to_mat(res["q"]), np.asarray(res["t"]), O.quat_to_mat(qp), tp, a)
        assert dt <= 0.01 and dr <= 0.05, (dt, dr)
    finally:
        ob.close()
        sw.close()
