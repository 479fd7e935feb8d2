"""Refinement parity (Sec. V-B/C) on the 128^3 workload's mesh (65k triangles,
a deep BVH) against the FP64 oracle, on a seeded subset of 400 of its 5000
probe poses (the oracle's cost grows with poses x triangles): per-pose
distances, J and grad J, refined poses from perturbed starts (1e-3 mm at the
anchor, 1e-3 deg), and the autograd wrapper against central differences
(step 1e-6) of the oracle's J at generic points."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2605_21398_gb300 import synth

pytestmark = pytest.mark.gpu

SUB = 400


@pytest.fixture(scope="module")
def setup(workload):
    from paper_2605_21398_gb300 import build, dock
    build.build()
    O.set_threads(os.cpu_count() or 1)
    w = workload("large128")
    idx = np.sort(np.random.default_rng(1303).choice(len(w.poses_world), SUB, replace=False))
    poses = np.ascontiguousarray(w.poses_world[idx])
    c = dock.Context(0)
    ob = c.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    sw = c.sweep_grid(poses, w.radius, w.length, w.h, w.N)
    yield c, ob, sw, w, poses
    c.close()


def _perturbed(w, rot_deg, trans):
    q = synth.quat_mul(synth.axis_angle_quat(np.radians(rot_deg)), w.gt_q)
    return q, w.gt_t + np.asarray(trans)


def _pose_err(qa, ta, Ra_b, tb, a):
    Ra = O.quat_to_mat(qa)
    dt = np.linalg.norm((Ra @ a + ta) - (Ra_b @ a + tb))
    c = (np.trace(Ra @ Ra_b.T) - 1) / 2
    return dt, math.degrees(math.acos(max(-1.0, min(1.0, c))))


def test_distances_match_oracle_on_the_large_mesh(setup):
    ctx, ob, sw, w, poses = setup
    starts = [(w.gt_q, w.gt_t), _perturbed(w, [0.4, -0.3, 0.2], [0.03, -0.02, 0.04])]
    d, wit, nrm = ctx.distances(ob, sw, np.array([np.concatenate([q, t]) for q, t in starts]))
    for b, (q, t) in enumerate(starts):
        do, wo, no, tri = O.distances(w.obj.verts, w.obj.tris, poses, O.quat_to_mat(q), t, w.radius, w.length)
        sel = do < O.TAU_OUT2
        assert sel.sum() > 50
        assert np.max(np.abs(d[b][sel] - do[sel])) < 2e-5
        assert np.all((d[b][~sel] >= O.TAU_OUT2 - 2e-5) | ~np.isfinite(d[b][~sel]))


def test_objective_gradient_and_refined_poses_match_oracle_on_the_large_mesh(setup):
    import torch
    ctx, ob, sw, w, poses = setup
    a = O.mesh_anchor(w.obj.verts)
    prm = O.refine_params(w.radius, w.length)
    rng = np.random.default_rng(7)
    starts = [_perturbed(w, rng.normal(size=3) * 0.5, rng.normal(size=3) * 0.05) for _ in range(3)]
    base = np.array([np.concatenate([q, t]) for q, t in starts])
    xis = np.array([np.concatenate([rng.normal(size=3) * 0.02, rng.normal(size=3) * 0.004]) for _ in range(3)])
    xi = torch.tensor(xis, dtype=torch.float32, device="cuda")
    J = torch.empty(3, dtype=torch.float32, device="cuda")
    G = torch.empty((3, 6), dtype=torch.float32, device="cuda")
    ctx.objective_fwd(ob, sw, base, xi.data_ptr(), 3, J.data_ptr(), G.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for k in range(3):
        Jo, Go, _, _ = O.objective(w.obj.verts, w.obj.tris, poses, O.quat_to_mat(base[k, :4]), base[k, 4:], a,
                                   xi[k].double().cpu().numpy(), prm)
        assert abs(J[k].item() - Jo) <= 1e-3 * max(1.0, abs(Jo))
        g = G[k].double().cpu().numpy()
        assert np.linalg.norm(g - Go) <= 2e-3 * max(1.0, np.linalg.norm(Go)), (g, Go)
    out = ctx.refine_se3(ob, sw, [dict(q=q, t=t) for q, t in starts])
    for (q, t), o in zip(starts, out):
        ref = O.refine(w.obj.verts, w.obj.tris, poses, O.quat_to_mat(q), t, a, prm)
        dt, dr = _pose_err(o["q"], o["t"], ref["R"], ref["p"], a)
        assert dt <= 1e-3 and dr <= 1e-3, (dt, dr, o["J"], ref["J"])
        assert abs(o["J"] - ref["J"]) <= 1e-3 * max(1.0, abs(ref["J"]))


def test_autograd_backward_matches_central_differences_on_the_large_mesh(setup):
    import torch
    from paper_2605_21398_gb300.autograd import objective
    ctx, ob, _, w, poses = setup
    a = O.mesh_anchor(w.obj.verts)
    prm = O.refine_params(w.radius, w.length)
    rng = np.random.default_rng(21)
    checked = 0
    for _ in range(6):
        q0, p0 = _perturbed(w, [0.4, -0.3, 0.2], rng.normal(size=3) * 0.05)
        xi0 = np.concatenate([rng.normal(size=3) * 0.02, rng.normal(size=3) * 0.004])
        R, p = O.pose_of_xi(O.quat_to_mat(q0), p0, a, xi0)
        do, _, _, _ = O.distances(w.obj.verts, w.obj.tris, poses, R, p, w.radius, w.length)
        sel = np.flatnonzero((do > 0.01) & (do < 0.19))   # generic points: outside witnesses
        if len(sel) < 10:
            continue
        sub = np.ascontiguousarray(poses[sel])
        sws = ctx.sweep_grid(sub, w.radius, w.length, w.h, w.N)
        try:
            xi = torch.tensor(xi0[None], dtype=torch.float32, device="cuda", requires_grad=True)
            J = objective(xi, ctx, ob, sws, np.concatenate([q0, p0])[None])
            J.sum().backward()
            g = xi.grad[0].double().cpu().numpy()
        finally:
            sws.close()
        step = 1e-6
        fd = np.zeros(6)
        for j in range(6):
            e = np.zeros(6)
            e[j] = step
            fd[j] = (O.objective(w.obj.verts, w.obj.tris, sub, O.quat_to_mat(q0), p0, a, xi0 + e, prm)[0]
                     - O.objective(w.obj.verts, w.obj.tris, sub, O.quat_to_mat(q0), p0, a, xi0 - e, prm)[0]) / (2 * step)
        assert np.linalg.norm(g - fd) <= 1e-3 * np.linalg.norm(fd) + 2e-3, (g, fd)
        checked += 1
        if checked == 2:
            break
    assert checked >= 1
