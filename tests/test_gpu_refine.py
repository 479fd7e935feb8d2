"""GPU parity of the refinement (Sec. V) against the FP64 oracle: distances,
objective and gradient, the autograd wrapper against central differences of
the oracle's J, refined poses, and the three-stage registration."""
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
    key = (w.name, w.seed)
    if key not in _OBJ:
        ob = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
        sw = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
        _OBJ[key] = (ob, sw)
    return _OBJ[key]


def _perturbed(w, rot_deg, trans):
    q = synth.quat_mul(synth.axis_angle_quat(np.radians(rot_deg)), w.gt_q)
    return q, w.gt_t + np.asarray(trans)


def _pose7(q, t):
    return np.concatenate([q, t])


def test_distances_match_oracle(ctx, workload):
    w = workload("tiny32")
    ob, sw = _gpu_pair(ctx, w)
    poses = [(w.gt_q, w.gt_t), _perturbed(w, [0.3, -0.2, 0.1], [0.04, 0.0, -0.03]),
             _perturbed(w, [-1.0, 0.5, 0.7], [-0.05, 0.08, 0.02])]
    d, wit, nrm = ctx.distances(ob, sw, np.array([_pose7(q, t) for q, t in poses]))
    for b, (q, t) in enumerate(poses):
        R = O.quat_to_mat(q)
        do, wo, no, tri = O.distances(w.obj.verts, w.obj.tris, w.poses_world, R, t, w.radius, w.length)
        sel = do < O.TAU_OUT2
        assert sel.sum() > 10
        assert np.max(np.abs(d[b][sel] - do[sel])) < 2e-5
        # beyond the cutoff both sides contribute nothing
        assert np.all((d[b][~sel] >= O.TAU_OUT2 - 2e-5) | ~np.isfinite(d[b][~sel]))
        # normals agree for outside witnesses (where f_p is smooth)
        ok = sel & (do > 1e-3)
        if ok.sum() > 0:
            cosang = np.sum(nrm[b][ok] * no[ok], axis=1)
            assert np.mean(cosang > 1 - 1e-3) > 0.95


def test_objective_and_gradient_match_oracle(ctx, workload):
    import torch
    w = workload("tiny32")
    ob, sw = _gpu_pair(ctx, w)
    a = O.mesh_anchor(w.obj.verts)
    prm = O.refine_params(w.radius, w.length)
    rng = np.random.default_rng(3)
    base, xis = [], []
    for k in range(4):
        q, t = _perturbed(w, rng.normal(size=3) * 0.5, rng.normal(size=3) * 0.05)
        base.append(_pose7(q, t))
        xis.append(np.concatenate([rng.normal(size=3) * 0.02, rng.normal(size=3) * 0.004]))
    base = np.array(base)
    xi = torch.tensor(np.array(xis), dtype=torch.float32, device="cuda")
    J = torch.empty(4, dtype=torch.float32, device="cuda")
    G = torch.empty((4, 6), dtype=torch.float32, device="cuda")
    ctx.objective_fwd(ob, sw, base, xi.data_ptr(), 4, J.data_ptr(), G.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for k in range(4):
        R0 = O.quat_to_mat(base[k, :4])
        Jo, Go, _, _ = O.objective(w.obj.verts, w.obj.tris, w.poses_world, R0, base[k, 4:], a,
                                   xi[k].double().cpu().numpy(), prm)
        assert abs(J[k].item() - Jo) <= 1e-3 * max(1.0, abs(Jo))
        g = G[k].double().cpu().numpy()
        assert np.linalg.norm(g - Go) <= 2e-3 * max(1.0, np.linalg.norm(Go))


def test_gradient_matches_oracle_while_penetrating(ctx, workload):
    # deep contacts: witnesses inside the probe, many on its medial surface,
    # where the derivative of d needs the subgradient the triangle selects
    import torch
    w = workload("tiny32", lines=5, pitch=1.5)
    ob = ctx.object_grid(w.obj.verts, w.obj.tris, w.h, w.N)
    sw = ctx.sweep_grid(w.poses_world, w.radius, w.length, w.h, w.N, contact=w.labels)
    a = O.mesh_anchor(w.obj.verts)
    prm = O.refine_params(w.radius, w.length)
    q0, t0 = _perturbed(w, [1.0, -0.5, 0.7], [0.1, -0.05, 0.08])
    rng = np.random.default_rng(0)
    xis = np.array([rng.normal(0, 0.02, 6) * np.array([1, 1, 1, 0.02, 0.02, 0.02]) for _ in range(3)])
    base = np.array([_pose7(q0, t0)] * 3)
    xi = torch.tensor(xis, dtype=torch.float32, device="cuda")
    J = torch.empty(3, dtype=torch.float32, device="cuda")
    G = torch.empty((3, 6), dtype=torch.float32, device="cuda")
    ctx.objective_fwd(ob, sw, base, xi.data_ptr(), 3, J.data_ptr(), G.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for k in range(3):
        Jo, Go, _, d = O.objective(w.obj.verts, w.obj.tris, w.poses_world, O.quat_to_mat(q0), t0, a,
                                   xi[k].double().cpu().numpy(), prm)
        assert (d < -O.TAU_IN2).sum() > 10
        assert abs(J[k].item() - Jo) <= 1e-3 * max(1.0, abs(Jo))
        g = G[k].double().cpu().numpy()
        assert np.linalg.norm(g - Go) <= 2e-3 * max(1.0, np.linalg.norm(Go)), (g, Go)
    ob.close()
    sw.close()


def test_autograd_backward_matches_central_differences(ctx, workload):
    import torch
    from paper_2605_21398_gb300.autograd import objective
    w = workload("tiny32")
    ob, _ = _gpu_pair(ctx, w)
    a = O.mesh_anchor(w.obj.verts)
    prm = O.refine_params(w.radius, w.length)
    rng = np.random.default_rng(14)
    checked = 0
    for trial in range(8):
        q0, p0 = _perturbed(w, [0.4, -0.3, 0.2], rng.normal(size=3) * 0.05)
        xi0 = np.concatenate([rng.normal(size=3) * 0.02, rng.normal(size=3) * 0.004])
        R, p = O.pose_of_xi(O.quat_to_mat(q0), p0, a, xi0)
        do, _, _, _ = O.distances(w.obj.verts, w.obj.tris, w.poses_world, R, p, w.radius, w.length)
        sel = np.flatnonzero((do > 0.01) & (do < 0.19))   # generic points: outside witnesses
        if len(sel) < 5:
            continue
        sw = ctx.sweep_grid(w.poses_world[sel], w.radius, w.length, w.h, w.N)
        xi = torch.tensor(xi0[None], dtype=torch.float32, device="cuda", requires_grad=True)
        J = objective(xi, ctx, ob, sw, _pose7(q0, p0)[None])
        J.sum().backward()
        g = xi.grad[0].double().cpu().numpy()
        step = 1e-6
        fd = np.zeros(6)
        for j in range(6):
            e = np.zeros(6)
            e[j] = step
            fd[j] = (O.objective(w.obj.verts, w.obj.tris, w.poses_world[sel], O.quat_to_mat(q0), p0, a, xi0 + e, prm)[0]
                     - O.objective(w.obj.verts, w.obj.tris, w.poses_world[sel], O.quat_to_mat(q0), p0, a, xi0 - e,
                                   prm)[0]) / (2 * step)
        assert np.linalg.norm(g - fd) <= 1e-3 * np.linalg.norm(fd) + 2e-3, (g, fd)
        checked += 1
    assert checked >= 2


def _pose_err(qa, ta, qb, tb, anchor):
    Ra, Rb = O.quat_to_mat(qa), O.quat_to_mat(qb)
    dt = np.linalg.norm((Ra @ anchor + ta) - (Rb @ anchor + tb))
    c = (np.trace(Ra @ Rb.T) - 1) / 2
    return dt, math.degrees(math.acos(max(-1.0, min(1.0, c))))


def test_refined_poses_match_oracle(ctx, workload):
    w = workload("tiny32")
    ob, sw = _gpu_pair(ctx, w)
    a = O.mesh_anchor(w.obj.verts)
    prm = O.refine_params(w.radius, w.length)
    starts = [_perturbed(w, [0.3, 0.2, -0.1], [0.05, 0.03, -0.04]), _perturbed(w, [1.0, -0.5, 0.7], [0.1, -0.05, 0.08])]
    cands = [dict(q=q, t=t) for q, t in starts]
    out = ctx.refine_se3(ob, sw, cands)
    for c, o in zip(starts, out):
        ref = O.refine(w.obj.verts, w.obj.tris, w.poses_world, O.quat_to_mat(c[0]), c[1], a, prm)
        qo = synth.mat_to_quat(ref["R"])
        dt, dr = _pose_err(o["q"], o["t"], qo, ref["p"], a)
        assert dt <= 1e-3 and dr <= 1e-3, (dt, dr, o["J"], ref["J"])
        assert abs(o["J"] - ref["J"]) <= 1e-3 * max(1.0, abs(ref["J"]))


def test_register_recovers_the_planted_pose(ctx, workload):
    w = workload("free64")
    ob, sw = _gpu_pair(ctx, w)
    # Table I sample counts: n_g = 20000 global, n_l = 5000 local, theta = 5 deg
    res = ctx.register(ob, sw, n_global=20000, n_local=5000, theta=math.radians(5), top_k=8)
    a = O.mesh_anchor(w.obj.verts)
    dt, dr = _pose_err(res["q"], res["t"], w.gt_q, w.gt_t, a)
    # pose noise of 0.1 mm / 0.5 deg per probe pose bounds the attainable
    # accuracy (the minimiser of J is not the planted pose): 0.21-0.26 mm seen
    assert dt < 0.3 and dr < 3.0, (dt, dr)
    assert res["n_evals"] == 20000 + 5000
