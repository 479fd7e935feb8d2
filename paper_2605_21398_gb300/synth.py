"""Seeded synthetic inputs shaped like the paper's simulation workloads (Sec. VI-A).

This module is the one piece shared by the CUDA path and the FP64 oracle.  It
holds none of the registration method's arithmetic: no SDF, no voxelisation,
no correlation, no sampler, no refinement.  It only *makes inputs*:

* a watertight star-shaped object mesh r(theta, phi) = r0 (1 + sum c_lm Y_lm),
  real orthonormal spherical harmonics of degree 1..L, c_lm ~ N(0, sigma2 / l),
  tessellated on a latitude/longitude grid with closed poles;
* a contact trajectory of a flat-ended cylindrical probe in three segments with
  three tool-axis directions (Sec. VI-A: "three segments with different contact
  directions").  Each pose is made by dropping the probe along its own axis onto
  the mesh until first contact (the drop-cutter construction of CAM tools), so a
  contact pose touches the mesh exactly;
* a planted ground-truth object pose, optional retreat arcs labelled
  non-contact, random label flips and Gaussian pose noise (Sec. VI-A: 0.02 mm).

Conventions used everywhere in this repository:
* a pose is 7 doubles (qw, qx, qy, qz, tx, ty, tz) mapping probe-local points
  to world points: x_world = R(q) x_local + t;
* the probe's local frame has its flat tip face centred at the origin and its
  body along +z, z in [0, L], radius r;
* the object pose maps object-frame points to world points.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# --------------------------------------------------------------------------
# small quaternion helpers (input construction only)
# --------------------------------------------------------------------------


def quat_mul(a, b):
    """Hamilton product a*b of (w, x, y, z) quaternions (arrays broadcast)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    w1, x1, y1, z1 = np.moveaxis(a, -1, 0)
    w2, x2, y2, z2 = np.moveaxis(b, -1, 0)
    return np.stack([
        w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
        w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
        w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
        w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2,
    ], axis=-1)


def quat_to_mat(q):
    q = np.asarray(q, dtype=np.float64)
    w, x, y, z = np.moveaxis(q, -1, 0)
    m = np.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y),
    ], axis=-1)
    return m.reshape(q.shape[:-1] + (3, 3))


def mat_to_quat(m):
    """Rotation matrix -> unit quaternion (w >= 0), Shepperd's branch choice."""
    m = np.asarray(m, dtype=np.float64)
    tr = m[0, 0] + m[1, 1] + m[2, 2]
    if tr > 0:
        s = math.sqrt(tr + 1.0) * 2
        q = [0.25 * s, (m[2, 1] - m[1, 2]) / s, (m[0, 2] - m[2, 0]) / s, (m[1, 0] - m[0, 1]) / s]
    elif m[0, 0] > m[1, 1] and m[0, 0] > m[2, 2]:
        s = math.sqrt(1.0 + m[0, 0] - m[1, 1] - m[2, 2]) * 2
        q = [(m[2, 1] - m[1, 2]) / s, 0.25 * s, (m[0, 1] + m[1, 0]) / s, (m[0, 2] + m[2, 0]) / s]
    elif m[1, 1] > m[2, 2]:
        s = math.sqrt(1.0 + m[1, 1] - m[0, 0] - m[2, 2]) * 2
        q = [(m[0, 2] - m[2, 0]) / s, (m[0, 1] + m[1, 0]) / s, 0.25 * s, (m[1, 2] + m[2, 1]) / s]
    else:
        s = math.sqrt(1.0 + m[2, 2] - m[0, 0] - m[1, 1]) * 2
        q = [(m[1, 0] - m[0, 1]) / s, (m[0, 2] + m[2, 0]) / s, (m[1, 2] + m[2, 1]) / s, 0.25 * s]
    q = np.array(q)
    q /= np.linalg.norm(q)
    return q if q[0] >= 0 else -q


def random_quat(rng, n=None):
    """Uniformly distributed unit quaternions (Shoemake's subgroup algorithm)."""
    size = () if n is None else (n,)
    u1, u2, u3 = rng.random(size), rng.random(size), rng.random(size)
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)], axis=-1)
    return q


def axis_angle_quat(v):
    """Quaternion of the rotation vector v (radians)."""
    v = np.asarray(v, dtype=np.float64)
    th = np.linalg.norm(v, axis=-1, keepdims=True)
    half = 0.5 * th
    with np.errstate(invalid="ignore", divide="ignore"):
        s = np.where(th > 1e-12, np.sin(half) / np.where(th > 0, th, 1), 0.5)
    return np.concatenate([np.cos(half), v * s], axis=-1)


# --------------------------------------------------------------------------
# star-shaped object mesh
# --------------------------------------------------------------------------


def _real_sph_harm(L, theta, phi):
    """Real orthonormal spherical harmonics Y_lm, l = 1..L, m = -l..l.

    Fully normalised associated Legendre functions by the standard three-term
    recurrences; returns an array (n_points, L*(L+2)) ordered (l, m) with m
    running -l..l.  Sign conventions do not matter (coefficients are random).
    """
    x = np.cos(theta)
    sx = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    P = {}
    P[(0, 0)] = np.full_like(x, math.sqrt(1.0 / (4 * math.pi)))
    for m in range(1, L + 1):
        P[(m, m)] = math.sqrt((2 * m + 1) / (2.0 * m)) * sx * P[(m - 1, m - 1)]
    for m in range(0, L):
        P[(m + 1, m)] = math.sqrt(2 * m + 3.0) * x * P[(m, m)]
    for m in range(0, L + 1):
        for l in range(m + 2, L + 1):
            a = math.sqrt((4.0 * l * l - 1) / (l * l - m * m))
            b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1) ** 2 - 1))
            P[(l, m)] = a * (x * P[(l - 1, m)] - b * P[(l - 2, m)])
    cols = []
    for l in range(1, L + 1):
        for m in range(-l, l + 1):
            if m == 0:
                cols.append(P[(l, 0)])
            elif m > 0:
                cols.append(math.sqrt(2.0) * P[(l, m)] * np.cos(m * phi))
            else:
                cols.append(math.sqrt(2.0) * P[(l, -m)] * np.sin(-m * phi))
    return np.stack(cols, axis=-1)


@dataclasses.dataclass
class StarObject:
    verts: np.ndarray      # (V, 3) float64, object frame, mm
    tris: np.ndarray       # (T, 3) int32, outward (counter-clockwise seen from outside)
    degree: int
    coeffs: np.ndarray     # (L*(L+2),) after the amplitude cap
    scale_applied: float   # 1.0 unless the amplitude cap rescaled the coefficients


def star_mesh(degree, sigma2, n_theta, n_phi, seed, r0=5.0, cap=0.3):
    """Watertight lat-long mesh of r(theta,phi) = r0 (1 + P(theta,phi)).

    P = sum_{l=1..L} sum_m c_lm Y_lm with c_lm ~ N(0, sigma2 / l).  If
    max |P| over the vertices exceeds `cap`, the coefficients are scaled by
    cap / max|P| (deterministic), which keeps the object inside its lattice.
    Triangle count = 2 n_phi (n_theta - 1).
    """
    rng = np.random.default_rng(seed)
    ls = np.concatenate([[l] * (2 * l + 1) for l in range(1, degree + 1)])
    c = rng.normal(0.0, 1.0, size=ls.shape) * np.sqrt(sigma2 / ls)
    th = np.pi * np.arange(1, n_theta) / n_theta
    ph = 2 * np.pi * np.arange(n_phi) / n_phi
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    dirs_th = np.concatenate([[0.0], TH.ravel(), [np.pi]])
    dirs_ph = np.concatenate([[0.0], PH.ravel(), [0.0]])
    Y = _real_sph_harm(degree, dirs_th, dirs_ph)
    P = Y @ c
    mx = float(np.max(np.abs(P)))
    scale = 1.0
    if mx > cap:
        scale = cap / mx
        c = c * scale
        P = P * scale
    r = r0 * (1.0 + P)
    u = np.stack([np.sin(dirs_th) * np.cos(dirs_ph), np.sin(dirs_th) * np.sin(dirs_ph),
                  np.cos(dirs_th)], axis=-1)
    verts = r[:, None] * u
    # indices: 0 = north pole, 1 + i*n_phi + j = ring i (theta_{i+1}), last = south pole
    nr = n_theta - 1
    south = 1 + nr * n_phi
    tris = []
    for j in range(n_phi):
        j1 = (j + 1) % n_phi
        tris.append((0, 1 + j, 1 + j1))
    for i in range(nr - 1):
        for j in range(n_phi):
            j1 = (j + 1) % n_phi
            a = 1 + i * n_phi + j
            b = 1 + i * n_phi + j1
            cc = 1 + (i + 1) * n_phi + j
            d = 1 + (i + 1) * n_phi + j1
            tris.append((a, cc, d))
            tris.append((a, d, b))
    for j in range(n_phi):
        j1 = (j + 1) % n_phi
        tris.append((south, 1 + (nr - 1) * n_phi + j1, 1 + (nr - 1) * n_phi + j))
    tris = np.asarray(tris, dtype=np.int32)
    return StarObject(verts=np.ascontiguousarray(verts), tris=tris, degree=degree,
                      coeffs=c, scale_applied=scale)


# --------------------------------------------------------------------------
# drop-to-contact trajectory
# --------------------------------------------------------------------------


def _frame_from_axis(a):
    """Orthonormal (e1, e2, a) with a = third axis; deterministic choice."""
    a = a / np.linalg.norm(a)
    h = np.array([1.0, 0.0, 0.0]) if abs(a[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = h - a * (h @ a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    return e1, e2, a


class _DropCutter:
    """First contact of a flat-ended cylinder moved tip-first along -a.

    For a fixed tool axis a the first contact offset along a is the largest
    axial coordinate over the parts of the mesh that lie within radius r of the
    tool's line.  Per triangle that maximum is reached at an end of an edge's
    chord through the infinite cylinder, or at the point of the plane/cylinder
    ellipse that is highest along a when it lies inside the triangle.
    """

    def __init__(self, verts, tris, a, r, cell=0.5):
        self.a = a / np.linalg.norm(a)
        self.e1, self.e2, _ = _frame_from_axis(self.a)
        self.r = float(r)
        self.V = verts
        self.T = tris
        tv = verts[tris]                                     # (T,3,3)
        u = tv @ self.e1
        v = tv @ self.e2
        self.lo = np.stack([u.min(1), v.min(1)], -1) - r
        self.hi = np.stack([u.max(1), v.max(1)], -1) + r
        self.cell = cell
        self.org = self.lo.min(0)
        ij_lo = np.floor((self.lo - self.org) / cell).astype(int)
        ij_hi = np.floor((self.hi - self.org) / cell).astype(int)
        self.bins = {}
        for t in range(len(tris)):
            for i in range(ij_lo[t, 0], ij_hi[t, 0] + 1):
                for j in range(ij_lo[t, 1], ij_hi[t, 1] + 1):
                    self.bins.setdefault((i, j), []).append(t)
        self.bins = {k: np.asarray(v, dtype=np.int64) for k, v in self.bins.items()}

    def drop(self, q2):
        """q2 = (u, v) position of the tool line in the (e1, e2) plane.

        Returns the axial offset s* (tip centre = u e1 + v e2 + s* a), or None
        when the line misses the mesh.
        """
        key = tuple(np.floor((np.asarray(q2) - self.org) / self.cell).astype(int))
        cand = self.bins.get(key)
        if cand is None:
            return None
        q2 = np.asarray(q2, dtype=np.float64)
        ok = np.all((self.lo[cand] <= q2) & (q2 <= self.hi[cand]), axis=1)
        cand = cand[ok]
        if len(cand) == 0:
            return None
        a, e1, e2, r = self.a, self.e1, self.e2, self.r
        p0 = q2[0] * e1 + q2[1] * e2
        tv = self.V[self.T[cand]]                            # (n,3,3)
        best = -np.inf
        # edges
        for k in range(3):
            A = tv[:, k, :]
            B = tv[:, (k + 1) % 3, :]
            w0 = A - p0
            d = B - A
            ad = d @ a
            aw = w0 @ a
            qa = np.einsum("ij,ij->i", d, d) - ad * ad
            qb = 2 * (np.einsum("ij,ij->i", w0, d) - aw * ad)
            qc = np.einsum("ij,ij->i", w0, w0) - aw * aw - r * r
            disc = qb * qb - 4 * qa * qc
            with np.errstate(invalid="ignore", divide="ignore"):
                sq = np.sqrt(np.maximum(disc, 0.0))
                g1 = np.where(qa > 1e-300, (-qb - sq) / (2 * qa), 0.0)
                g2 = np.where(qa > 1e-300, (-qb + sq) / (2 * qa), 1.0)
            # segment inside the chord when qa ~ 0 and qc <= 0
            flat = qa <= 1e-300
            g1 = np.where(flat, np.where(qc <= 0, 0.0, 2.0), g1)
            g2 = np.where(flat, np.where(qc <= 0, 1.0, -1.0), g2)
            valid = (disc >= 0) | flat
            lo = np.maximum(g1, 0.0)
            hi = np.minimum(g2, 1.0)
            valid &= lo <= hi
            for g in (lo, hi):
                ax = aw + g * ad
                if np.any(valid):
                    best = max(best, float(np.max(np.where(valid, ax, -np.inf))))
        # interior ellipse points
        v0, v1, v2 = tv[:, 0], tv[:, 1], tv[:, 2]
        nrm = np.cross(v1 - v0, v2 - v0)
        g = nrm @ a
        al = nrm @ e1
        be = nrm @ e2
        K = np.einsum("ij,ij->i", nrm, v0 - p0)
        ab = np.sqrt(al * al + be * be)
        good = np.abs(g) > 1e-12 * np.linalg.norm(nrm, axis=1)
        with np.errstate(invalid="ignore", divide="ignore"):
            # t(phi) = (K - r (al cos + be sin)) / g, maximised over phi
            sgn = np.sign(g)
            cphi = np.where(ab > 0, -sgn * al / np.where(ab > 0, ab, 1), 0.0)
            sphi = np.where(ab > 0, -sgn * be / np.where(ab > 0, ab, 1), 0.0)
            rr = np.where(ab > 0, r, 0.0)
            t = (K - rr * (al * cphi + be * sphi)) / np.where(good, g, 1.0)
        pts = p0 + rr[:, None] * (cphi[:, None] * e1 + sphi[:, None] * e2) + t[:, None] * a
        # inside-triangle test in the triangle's plane
        def _bary(p):
            e0 = v1 - v0
            e1_ = v2 - v0
            w = p - v0
            d00 = np.einsum("ij,ij->i", e0, e0)
            d01 = np.einsum("ij,ij->i", e0, e1_)
            d11 = np.einsum("ij,ij->i", e1_, e1_)
            d20 = np.einsum("ij,ij->i", w, e0)
            d21 = np.einsum("ij,ij->i", w, e1_)
            den = d00 * d11 - d01 * d01
            bv = (d11 * d20 - d01 * d21) / den
            bw = (d00 * d21 - d01 * d20) / den
            return bv, bw
        bv, bw = _bary(pts)
        inside = good & (bv >= 0) & (bw >= 0) & (bv + bw <= 1)
        if np.any(inside):
            best = max(best, float(np.max(t[inside])))
        return None if not np.isfinite(best) else best


def _axis_quat(a, e1):
    """Quaternion whose rotation maps local (x, y, z) to (e1, a x e1, a)."""
    e2 = np.cross(a, e1)
    m = np.stack([e1, e2, a], axis=1)
    return mat_to_quat(m)


@dataclasses.dataclass
class Trajectory:
    poses_obj: np.ndarray    # (P, 7) probe -> object frame
    contact_geom: np.ndarray  # (P,) uint8: 1 where the pose touches the mesh (before noise)
    labels: np.ndarray       # (P,) uint8: the contact labels handed to the method
    axes: np.ndarray         # (3, 3) tool-axis direction of each segment


def contact_trajectory(obj: StarObject, n_poses, radius, length, seed,
                       noncontact_frac=0.0, lift_range=(0.5, 2.0), sweep=4.5, axes_mode="ortho", wobble=2.0,
                       lines=1, pitch=1.5):
    """Three drop-to-contact segments with different tool-axis directions.

    axes_mode "ortho": the three columns of a random rotation, each tilted by
    a random 10-20 degrees (no exact symmetry between segments); "cone":
    three axes inside a 60 degree cone (probing from one side).  Segment s
    uses tool axis a_s (pointing from the tip to the shank) and moves the tool
    line across the object face seen from a_s: lateral offset
    sweep*(2 tau - 1) along e1 plus a wobble of up to `wobble` mm along e2.
    With `lines` > 1 a segment is a zig-zag raster instead: `lines` parallel
    passes `pitch` mm apart along e2, each across the part of [-sweep, sweep]
    where the tool line meets the object (no wobble).
    With `noncontact_frac` > 0, contiguous runs of poses are lifted along the
    axis by U(lift_range) mm on a half-sine profile and labelled non-contact.
    """
    rng = np.random.default_rng(seed)
    q = random_quat(rng)
    Rm = quat_to_mat(q)
    if axes_mode == "cone":
        t60 = math.radians(60.0)
        local = np.array([[0.0, 0.0, 1.0],
                          [math.sin(t60), 0.0, math.cos(t60)],
                          [math.sin(t60) * math.cos(math.radians(135)), math.sin(t60) * math.sin(math.radians(135)),
                           math.cos(t60)]])
        axes = local @ Rm.T
    else:
        axes = Rm.T.copy()
        for s_ in range(3):
            tilt = math.radians(rng.uniform(10.0, 20.0))
            v = rng.normal(size=3)
            v -= axes[s_] * (v @ axes[s_])
            v /= np.linalg.norm(v)
            axes[s_] = math.cos(tilt) * axes[s_] + math.sin(tilt) * v
    sizes = [n_poses // 3 + (1 if s < n_poses % 3 else 0) for s in range(3)]
    poses, geom = [], []
    for s in range(3):
        a = axes[s]
        e1, e2, a = _frame_from_axis(a)
        dc = _DropCutter(obj.verts, obj.tris, a, radius)
        qa = _axis_quat(a, e1)
        n = sizes[s]
        wob = wobble * rng.random()
        ph = 2 * np.pi * rng.random()
        lifted = np.zeros(n)
        if noncontact_frac > 0 and n > 0:
            nlift = int(round(noncontact_frac * n))
            nruns = max(1, nlift // 40)
            per = max(1, nlift // nruns)
            starts = np.sort(rng.choice(max(1, n - per), size=nruns, replace=False))
            for st in starts:
                amp = rng.uniform(*lift_range)
                k = np.arange(per)
                prof = amp * (0.25 + 0.75 * np.sin(np.pi * (k + 0.5) / per))
                lifted[st:st + per] = np.maximum(lifted[st:st + per], prof[: len(lifted[st:st + per])])
        path = _segment_path(dc, n, sweep, wob, ph, lines, pitch)
        for k in range(n):
            u, v = path[k]
            sstar = dc.drop((u, v))
            if sstar is None:
                raise RuntimeError("tool line missed the object; shrink the sweep")
            tip = u * e1 + v * e2 + (sstar + lifted[k]) * a
            poses.append(np.concatenate([qa, tip]))
            geom.append(0 if lifted[k] > 0 else 1)
    poses = np.asarray(poses)
    geom = np.asarray(geom, dtype=np.uint8)
    return Trajectory(poses_obj=poses, contact_geom=geom, labels=geom.copy(), axes=axes)


def _segment_path(dc, n, sweep, wob, ph, lines, pitch):
    """(u, v) tool-line offsets of the n poses of one segment."""
    if lines <= 1:
        tau = (np.arange(n) + 0.5) / n
        return np.stack([sweep * (2 * tau - 1), wob * np.sin(2 * np.pi * tau + ph)], axis=1)
    counts = [n // lines + (1 if l < n % lines else 0) for l in range(lines)]
    grid = np.linspace(-sweep, sweep, 129)
    out = []
    for l in range(lines):
        v = pitch * (l - 0.5 * (lines - 1))
        hit = np.array([dc.drop((u, v)) is not None for u in grid])
        if not hit.any():
            raise RuntimeError("raster line missed the object; reduce the pitch")
        # the longest run of hits, shrunk by one grid step at each end
        best, cur, start = (0, 0, 0), 0, 0
        for i, hv in enumerate(hit):
            if hv:
                if cur == 0:
                    start = i
                cur += 1
                if cur > best[0]:
                    best = (cur, start, i)
            else:
                cur = 0
        lo = grid[min(best[1] + 1, best[2])]
        hi = grid[max(best[2] - 1, best[1])]
        tau = (np.arange(counts[l]) + 0.5) / max(counts[l], 1)
        u = lo + (hi - lo) * (tau if l % 2 == 0 else 1.0 - tau)
        out.append(np.stack([u, np.full_like(u, v)], axis=1))
    return np.concatenate(out, axis=0)


def transform_poses(T_q, T_t, poses):
    """World poses of probe poses given in the object frame: T * P_i."""
    q = quat_mul(np.broadcast_to(T_q, poses[:, :4].shape), poses[:, :4])
    t = poses[:, 4:] @ quat_to_mat(T_q).T + T_t
    return np.concatenate([q, t], axis=1)


def add_pose_noise(poses, rng, sigma_t, sigma_r_deg):
    out = poses.copy()
    if sigma_t > 0:
        out[:, 4:] += rng.normal(0, sigma_t, size=(len(poses), 3))
    if sigma_r_deg > 0:
        dq = axis_angle_quat(rng.normal(0, math.radians(sigma_r_deg), size=(len(poses), 3)))
        out[:, :4] = quat_mul(dq, out[:, :4])
    out[:, :4] /= np.linalg.norm(out[:, :4], axis=1, keepdims=True)
    return out


# --------------------------------------------------------------------------
# the workload configurations
# --------------------------------------------------------------------------

# name: (degree, sigma2, n_theta, n_phi, N, h, probe r, probe L, poses, n_rot, top_k,
#        noncontact_frac, label_flip_frac, noise_t, noise_r_deg)
CONFIGS = {
    "tiny32": dict(degree=4, sigma2=0.04, n_theta=24, n_phi=48, N=32, h=0.5, radius=1.0, length=8.0,
                   poses=200, n_rot=512, top_k=8, noncontact=0.0, flip=0.0, noise_t=0.0, noise_r=0.0),
    "free64": dict(degree=8, sigma2=0.05, n_theta=72, n_phi=144, N=64, h=0.25, radius=0.8, length=12.0,
                   poses=2000, n_rot=4096, top_k=32, noncontact=0.3, flip=0.0, noise_t=0.1, noise_r=0.5,
                   lines=5, pitch=1.5),
    "large128": dict(degree=12, sigma2=0.05, n_theta=128, n_phi=256, N=128, h=0.15, radius=0.8, length=12.0,
                     poses=5000, n_rot=32768, top_k=64, noncontact=0.0, flip=0.2, noise_t=0.02, noise_r=0.0,
                     lines=5, pitch=1.5),
}


@dataclasses.dataclass
class Workload:
    name: str
    obj: StarObject
    traj: Trajectory
    poses_world: np.ndarray   # (P, 7)
    labels: np.ndarray        # (P,) uint8
    gt_q: np.ndarray          # (4,) object -> world
    gt_t: np.ndarray          # (3,)
    N: int
    h: float
    radius: float
    length: float
    n_rot: int
    top_k: int
    seed: int


def make_workload(name, replicate=0, **overrides):
    """Build one seeded workload; seed = 1000 * config index + replicate."""
    cfg = dict(CONFIGS[name])
    cfg.update(overrides)
    idx = list(CONFIGS).index(name) + 1 if name in CONFIGS else 9
    seed = 1000 * idx + replicate
    obj = star_mesh(cfg["degree"], cfg["sigma2"], cfg["n_theta"], cfg["n_phi"], seed, cap=cfg.get("cap", 0.3))
    traj = contact_trajectory(obj, cfg["poses"], cfg["radius"], cfg["length"], seed + 7,
                              noncontact_frac=cfg["noncontact"], sweep=cfg.get("sweep", 4.5),
                              axes_mode=cfg.get("axes_mode", "ortho"), wobble=cfg.get("wobble", 2.0),
                              lines=cfg.get("lines", 1), pitch=cfg.get("pitch", 1.5))
    rng = np.random.default_rng(seed + 13)
    gt_q = random_quat(rng)
    gt_t = rng.uniform(-2.0, 2.0, size=3)
    pw = transform_poses(gt_q, gt_t, traj.poses_obj)
    pw = add_pose_noise(pw, rng, cfg["noise_t"], cfg["noise_r"])
    labels = traj.labels.copy()
    if cfg["flip"] > 0:
        nflip = int(round(cfg["flip"] * len(labels)))
        idxs = rng.choice(np.flatnonzero(labels == 1), size=min(nflip, int(labels.sum())), replace=False)
        labels[idxs] = 0
    return Workload(name=name, obj=obj, traj=traj, poses_world=np.ascontiguousarray(pw),
                    labels=labels, gt_q=gt_q, gt_t=gt_t, N=cfg["N"], h=cfg["h"],
                    radius=cfg["radius"], length=cfg["length"], n_rot=cfg["n_rot"],
                    top_k=cfg["top_k"], seed=seed)


def random_unit_quats(n, seed):
    """Seeded uniform unit quaternions, used as explicit rotation inputs."""
    return random_quat(np.random.default_rng(seed), n)
