"""FP64 CPU oracle for complementary-shape docking registration.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the bench's CPU
baseline leg may import this package; the product (the CUDA library and its
binding) never does, and the two share no code.  The heavy geometric loops
live in oracle.c (FP64, no fused multiply-add); this module drives them and
adds the steps that are plain definitions or textbook library primitives:

* correlation, Sec. IV-B Eq. (7): C[dk] = sum_k O[k] S[k + dk] on a zero
  padded canvas of side M >= n_o + n_s - 1, evaluated with numpy's FP64 FFT
  as C = F^-1( conj(F(O)) . F(S) )  (Eq. (9) read so that it agrees with
  Eq. (7) and Eq. (8); see `correlate_fft`), and by the direct sum for tiny
  grids (`correlate_direct`);
* translation from the peak, Eq. (8), composed with the sampled rotation;
* orientation samplers, Sec. IV-C: Super-Fibonacci, a Hopf-coordinate map of a
  Halton sequence, and GeoBall-SF (Algorithm 1, Eq. (10)-(12));
* the per-rotation argmax and the global top-K;
* the label-aware score (Sec. I and IV-A: trajectories hold contact and
  non-contact evidence): voxels swept by a contact pose score O, voxels swept
  only by non-contact poses score min(O, 0), the penetration part alone.
* the rotation mechanism Sec. IV-D prints: the object grid rotated and
  resampled by trilinear interpolation per sample, correlated with the fixed
  swept grid (`search_rotate_object`).

The refinement is solved two ways: a fixed-iteration projected Gauss-Newton
solver (`refine`, the GPU default) and the L-BFGS-B of Sec. V-C
(`refine_lbfgsb`, scipy's implementation as the library step).  `register`
chains the three stages of Fig. 2: global search, local GeoBall-SF search
about the best global rotation, refinement of the merged top-K.

Parity unpinned: the Super-Fibonacci constants beyond the paper's
nearest-neighbour statistic (Sec. VI: 8.0 deg at n = 20000), and the
iterates of L-BFGS-B (only its minimiser is compared).
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)

# Table I (Sec. VI) and the readings listed in the design notes.
TAU_OUT1 = 0.5     # tau_out,1 (mm), object band outside
TAU_IN1 = 0.2      # tau_in,1 (mm), object band inside
DEEP_VALUE = -50.0  # O_t for f <= -tau_in,1 (Table I rho = -50, taken as the value)
TAU_OUT2 = 0.2     # tau_out,2 (mm), score window
TAU_IN2 = 0.03     # tau_in,2 (mm)
K_SLOPE = 15.0     # penalty slope k of Eq. (18)
LAMBDA = 1e-3      # Table I "10e-4"
MU = 1e-6          # Gauss-Newton damping (mm^-2)
B_T = 1.0          # box bound on |u|_inf (mm)
B_R = math.radians(5.0)   # box bound on |w|_inf (rad)
STEP_T = 0.05      # per-iteration trust region, translation (mm)
STEP_R = math.radians(0.5)  # per-iteration trust region, rotation (rad)
ITERS = 20
DECAY = 1.0        # trust-region shrink factor per iteration (1 = fixed radii)

SF_PHI = math.sqrt(2.0)
SF_PSI = 1.533751168755204288118041  # real root of psi^4 = psi + 4


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_object_grid.restype = ctypes.c_int
        L.orc_probe_sdf.restype = ctypes.c_double
        L.orc_tri_min.restype = ctypes.c_double
        L.orc_objective.restype = ctypes.c_double
        L.orc_refine.restype = ctypes.c_double
        L.orc_chol6.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, t=_dp):
    return a.ctypes.data_as(t)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------
# rotations
# ----------------------------------------------------------------------------

def quat_to_mat(q):
    q = _c64(q)
    R = np.empty(9)
    lib().orc_quat_to_mat(_p(q), _p(R))
    return R.reshape(3, 3)


def quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def quat_dist(q1, q2):
    """Eq. (10): half the relative rotation angle, arccos |<q1, q2>|."""
    c = abs(float(np.dot(q1, q2)))
    return math.acos(min(1.0, c))


# ----------------------------------------------------------------------------
# grids, Eq. (1)-(6)
# ----------------------------------------------------------------------------

def object_grid(verts, tris, h, N, touch=None, tau_out=TAU_OUT1, tau_in=TAU_IN1, deep=DEEP_VALUE):
    """O[kz, ky, kx] (float64), the lattice origin o_o, the clamped SDF, and a
    flag telling whether the mesh (widened by tau_out) fits the lattice."""
    V = _c64(verts)
    T = np.ascontiguousarray(tris, dtype=np.int32)
    tp = None
    if touch is not None:
        touch = np.ascontiguousarray(touch, dtype=np.uint8)
        tp = _p(touch, _u8p)
    O = np.empty((N, N, N))
    f = np.empty((N, N, N))
    o = np.empty(3)
    rc = lib().orc_object_grid(_p(V), ctypes.c_int64(len(V)), _p(T, _ip), ctypes.c_int64(len(T)), tp,
                               ctypes.c_double(h), ctypes.c_int32(N), ctypes.c_double(tau_out),
                               ctypes.c_double(tau_in), ctypes.c_double(deep), _p(o), _p(O), _p(f))
    return O, o, f, rc == 0


def sweep_origin(poses, q, h, N):
    P = _c64(poses)
    q = _c64(q)
    o = np.empty(3)
    lib().orc_sweep_origin(_p(P), ctypes.c_int64(len(P)), _p(q), ctypes.c_double(h), ctypes.c_int32(N), _p(o))
    return o


def sweep_grid(poses, q, h, N, r, L, use=None):
    """S_R[jz, jy, jx] (uint8) and its origin o_s,R for rotation q.  With
    `use` (one flag per pose) only the flagged poses are swept; the origin
    still follows all poses."""
    P = _c64(poses)
    q = _c64(q)
    S = np.empty((N, N, N), dtype=np.uint8)
    o = np.empty(3)
    u = None
    if use is not None:
        u = np.ascontiguousarray(use, dtype=np.uint8)
        assert u.shape == (len(P),)
    lib().orc_sweep_grid_sel(_p(P), ctypes.c_int64(len(P)), None if u is None else _p(u, _u8p), _p(q),
                             ctypes.c_double(h), ctypes.c_int32(N), ctypes.c_double(r), ctypes.c_double(L),
                             _p(o), _p(S, _u8p))
    return S, o


def sweep_grids_by_label(poses, labels, q, h, N, r, L):
    """Label-aware split of the sweep (Sec. I and IV-A: trajectories carry
    contact and non-contact evidence).  S_c: voxels swept by a contact pose;
    S_n: voxels swept only by non-contact poses (S_n and S_c are disjoint,
    their union is the plain S_R).  Both on the lattice of all poses."""
    lab = np.asarray(labels).astype(bool)
    S_c, o = sweep_grid(poses, q, h, N, r, L, use=lab)
    S_any, _ = sweep_grid(poses, q, h, N, r, L, use=~lab)
    S_n = (S_any & (1 - S_c)).astype(np.uint8)
    return S_c, S_n, o


# ----------------------------------------------------------------------------
# correlation, Eq. (7)-(9)
# ----------------------------------------------------------------------------

def canvas_size(N):
    """Smallest even side >= 2N - 1 (Sec. IV-B: n_o + n_s - 1 per axis)."""
    return 2 * N


def correlate_fft(O, S, M):
    """C[cz, cy, cx] = sum_k O[k] S[(k + c) mod M] on an M^3 zero canvas.

    With F(x)[w] = sum_k x[k] exp(-2 pi i w.k / M) this is
    C = F^-1(conj(F(O)) . F(S)).  (Eq. (9) prints the conjugate on F(S), which
    would give C[-dk]; Eq. (7) and Eq. (8) are taken as normative.)"""
    FO = np.fft.rfftn(O, s=(M, M, M), axes=(0, 1, 2))
    FS = np.fft.rfftn(S.astype(np.float64), s=(M, M, M), axes=(0, 1, 2))
    return np.fft.irfftn(np.conj(FO) * FS, s=(M, M, M), axes=(0, 1, 2))


def correlate_direct(O, S, M):
    """Eq. (7) by its definition: brute force over every canvas shift."""
    N = O.shape[0]
    C = np.zeros((M, M, M))
    Sp = np.zeros((M, M, M))
    Sp[:N, :N, :N] = S
    for cz in range(M):
        for cy in range(M):
            for cx in range(M):
                acc = 0.0
                for kz in range(N):
                    for ky in range(N):
                        for kx in range(N):
                            o = O[kz, ky, kx]
                            if o != 0.0:
                                acc += o * Sp[(kz + cz) % M, (ky + cy) % M, (kx + cx) % M]
                C[cz, cy, cx] = acc
    return C


def canvas_shift(idx, M, N):
    """Linear canvas index (cz*M + cy)*M + cx -> shift (dx, dy, dz); an index
    c maps to c if c <= N-1, else c - M."""
    cz, rem = divmod(int(idx), M * M)
    cy, cx = divmod(rem, M)
    return np.array([c if c <= N - 1 else c - M for c in (cx, cy, cz)], dtype=np.int64)


def peak(C):
    """Per-rotation argmax; ties go to the lowest linear index."""
    flat = C.reshape(-1)
    i = int(np.argmax(flat))
    return float(flat[i]), i


def pose_from_peak(q, dk, h, o_s, o_o):
    """T = (R, R (h dk + o_s,R - o_o)): Eq. (8) with the sampled rotation."""
    R = quat_to_mat(q)
    t = R @ (h * np.asarray(dk, dtype=np.float64) + o_s - o_o)
    return R, t


def top_k(scores, k):
    """Indices of the k best rotations: score descending, rotation ascending."""
    scores = np.asarray(scores)
    order = np.lexsort((np.arange(len(scores)), -scores))
    return order[:k]


def penetration_part(O):
    """min(O, 0): the interior penalty of Eq. (1)-(4) without the near-surface
    reward.  A pose that did not touch the object may not overlap it, but its
    approach to the surface earns nothing."""
    return np.minimum(O, 0.0)


def correlate_label_aware(O, S_c, S_n, M, fft=True):
    """C = corr(O, S_c) + corr(min(O, 0), S_n): voxels reached by a contact
    pose score O (Eq. (7)), voxels reached only by non-contact poses score the
    penetration part alone."""
    f = correlate_fft if fft else correlate_direct
    return f(O, S_c, M) + f(penetration_part(O), S_n, M)


def search_label_aware(O, o_o, poses, labels, quats, h, N, r, L, fft=True):
    """`search` with the label-aware score (`correlate_label_aware`)."""
    M = canvas_size(N)
    out = []
    for q in quats:
        S_c, S_n, o_s = sweep_grids_by_label(poses, labels, q, h, N, r, L)
        C = correlate_label_aware(O, S_c, S_n, M, fft=fft)
        sc, idx = peak(C)
        out.append(dict(score=sc, idx=idx, dk=canvas_shift(idx, M, N), o_s=o_s, C=C, S_c=S_c, S_n=S_n))
    return out


def search(O, o_o, poses, quats, h, N, r, L, fft=True):
    """For each rotation: the swept grid, the correlation and its peak.
    Returns a list of dicts (score, idx, dk, o_s, S)."""
    M = canvas_size(N)
    out = []
    for q in quats:
        S, o_s = sweep_grid(poses, q, h, N, r, L)
        C = correlate_fft(O, S, M) if fft else correlate_direct(O, S, M)
        sc, idx = peak(C)
        out.append(dict(score=sc, idx=idx, dk=canvas_shift(idx, M, N), o_s=o_s, C=C, S=S))
    return out


def set_threads(n):
    """Threads of the oracle's parallel per-pose loops (1 = serial); results
    do not depend on it (every sum over poses runs in pose order)."""
    lib().orc_set_threads(int(n))


def max_threads():
    return int(lib().orc_max_threads())


def _rotation_peak(args):
    O, poses, q, h, N, r, L, M = args
    S, o_s = sweep_grid(poses, q, h, N, r, L)
    C = correlate_fft(O, S, M)
    sc, idx = peak(C)
    return sc, idx, o_s, float(np.max(np.abs(C)))


def search_peaks(O, poses, quats, h, N, r, L, workers=1):
    """`search` without keeping the grids: per rotation the peak score, its
    canvas index and shift, the swept-lattice origin and max |C| (the scale of
    the score tolerance).  Rotations are independent; with workers > 1 they
    run in a thread pool (the C voxeliser and the FFT release the GIL), each
    rotation computed exactly as alone."""
    M = canvas_size(N)
    args = [(O, poses, q, h, N, r, L, M) for q in quats]
    if workers > 1:
        import concurrent.futures as cf
        with cf.ThreadPoolExecutor(workers) as ex:
            res = list(ex.map(_rotation_peak, args))
    else:
        res = [_rotation_peak(a) for a in args]
    return [dict(score=sc, idx=idx, dk=canvas_shift(idx, M, N), o_s=o_s, cmax=cm) for sc, idx, o_s, cm in res]


def register(verts, tris, poses, h, N, r, L, n_global, n_local, theta, n_cand, prm, sampler="sf", workers=1):
    """The three stages of a registration (Fig. 2; Sec. IV-C, IV-D, V-C):

    1. global search (Sec. IV-C.1): the peak of Eq. (7) for each of n_global
       Super-Fibonacci (or Hopf) rotations;
    2. local search (Sec. IV-C.2, Algorithm 1): the peaks of n_local GeoBall-SF
       rotations in the ball of half-angle theta about the best global
       rotation (score descending, sample index ascending); these samples are
       numbered after the global ones;
    3. the n_cand best peaks of both stages together (same order) become candidate
       poses by Eq. (8) with the sampled rotation, each is refined (Sec. V-C,
       the fixed-iteration Gauss-Newton of `refine`) and the candidate with the
       lowest J wins (ties: the lower candidate index).

    Returns the global and local peaks, the candidates and their refinements,
    and the winner."""
    O, o_o, _, fits = object_grid(verts, tris, h, N)
    if not fits:
        raise ValueError("mesh does not fit the lattice")
    qg = super_fibonacci(n_global) if sampler == "sf" else hopf_halton(n_global)
    pg = search_peaks(O, poses, qg, h, N, r, L, workers)
    sg = np.array([p["score"] for p in pg])
    best_g = int(top_k(sg, 1)[0])
    quats = qg
    peaks = pg
    if n_local > 0:
        ql = geoball_sf(n_local, qg[best_g], theta)
        pl = search_peaks(O, poses, ql, h, N, r, L, workers)
        quats = np.concatenate([qg, ql])
        peaks = pg + pl
    scores = np.array([p["score"] for p in peaks])
    order = top_k(scores, n_cand)
    anchor = mesh_anchor(verts)
    cands = []
    for k, i in enumerate(order):
        R, t = pose_from_peak(quats[i], peaks[i]["dk"], h, peaks[i]["o_s"], o_o)
        ref = refine(verts, tris, poses, R, t, anchor, prm)
        cands.append(dict(rot=int(i), q=quats[i], dk=peaks[i]["dk"], score=peaks[i]["score"], R0=R, t0=t,
                          J=ref["J"], R=ref["R"], p=ref["p"], xi=ref["xi"]))
    Js = np.array([c["J"] for c in cands])
    best = int(np.lexsort((np.arange(len(Js)), Js))[0])
    return dict(quats=quats, peaks=peaks, best_global=best_g, order=order, cands=cands, best=best, anchor=anchor,
                o_o=o_o)


# ----------------------------------------------------------------------------
# Sec. IV-D as printed: rotate the object grid, keep the swept grid fixed
# ----------------------------------------------------------------------------

IDENTITY_Q = np.array([1.0, 0.0, 0.0, 0.0])


def rotate_object(O, o_o, q, h):
    """(O_R, o_R): O rotated by R(q) and resampled by trilinear interpolation
    (zero outside O's lattice) onto the lattice h k + o_R, with
    o_R = h round(R c_o / h) - (N/2) h, c_o = o_o + (N/2) h."""
    N = O.shape[0]
    Oc = _c64(O)
    OR = np.empty((N, N, N))
    oR = np.empty(3)
    lib().orc_rotate_object(_p(Oc), ctypes.c_int32(N), _p(_c64(o_o)), _p(_c64(q)), ctypes.c_double(h), _p(OR),
                            _p(oR))
    return OR, oR


def pose_from_peak_rotated_object(q, dk, h, o_s, o_R):
    """Object voxel k of O_R (world point h k + o_R for the pose (R, 0)) meets
    swept voxel k + dk (world point h (k + dk) + o_s): T = (R, h dk + o_s - o_R)."""
    return quat_to_mat(q), h * np.asarray(dk, dtype=np.float64) + o_s - o_R


def search_rotate_object(O, o_o, poses, quats, h, N, r, L, fft=True):
    """Sec. IV-D as printed: S on the world-aligned lattice of the mean tip,
    fixed; per rotation O_R and C = Eq. (7) of O_R with S; the peak and its pose."""
    M = canvas_size(N)
    S, o_s = sweep_grid(poses, IDENTITY_Q, h, N, r, L)
    out = []
    for q in quats:
        OR, oR = rotate_object(O, o_o, q, h)
        C = correlate_fft(OR, S, M) if fft else correlate_direct(OR, S, M)
        sc, idx = peak(C)
        dk = canvas_shift(idx, M, N)
        R, t = pose_from_peak_rotated_object(q, dk, h, o_s, oR)
        out.append(dict(score=sc, idx=idx, dk=dk, o_s=o_s, o_R=oR, C=C, t=t))
    return out


# ----------------------------------------------------------------------------
# orientation samplers, Sec. IV-C
# ----------------------------------------------------------------------------

def super_fibonacci(n):
    """Super-Fibonacci spiral on S^3 (Alexa, CVPR 2022): sample i uses
    s = i + 1/2, t = s/n, r = sqrt(t), R = sqrt(1 - t), alpha = 2 pi s / phi,
    beta = 2 pi s / psi; q = (r sin alpha, r cos alpha, R sin beta, R cos beta)
    with phi = sqrt 2 and psi^4 = psi + 4."""
    s = np.arange(n, dtype=np.float64) + 0.5
    t = s / n
    r = np.sqrt(t)
    R = np.sqrt(1.0 - t)
    al = 2.0 * math.pi * s / SF_PHI
    be = 2.0 * math.pi * s / SF_PSI
    return np.stack([r * np.sin(al), r * np.cos(al), R * np.sin(be), R * np.cos(be)], axis=1)


def _radical_inverse(i, base):
    f, x = 1.0, 0.0
    while i > 0:
        f /= base
        x += f * (i % base)
        i //= base
    return x


def hopf_halton(n):
    """Hopf coordinates (theta, phi, psi) of a Halton (2, 3, 5) sequence
    (Yershova et al. 2010): theta = arccos(1 - 2 u1), phi = 2 pi u2,
    psi = 2 pi u3, q = (cos(theta/2) cos(psi/2), cos(theta/2) sin(psi/2),
    sin(theta/2) cos(phi + psi/2), sin(theta/2) sin(phi + psi/2))."""
    u = np.array([[_radical_inverse(i + 1, b) for b in (2, 3, 5)] for i in range(n)])
    th = np.arccos(1.0 - 2.0 * u[:, 0])
    ph = 2 * math.pi * u[:, 1]
    ps = 2 * math.pi * u[:, 2]
    return np.stack([np.cos(th / 2) * np.cos(ps / 2), np.cos(th / 2) * np.sin(ps / 2),
                     np.sin(th / 2) * np.cos(ph + ps / 2), np.sin(th / 2) * np.sin(ph + ps / 2)], axis=1)


def geoball_radial_table(theta, nodes=4097):
    """Tabulated (r, F(r)) of Eq. (11)-(12) on [0, sin theta]: density
    rho(r) ~ r L(r), L(r) = 2 arccos(cos theta / sqrt(1 - r^2)), cumulative by
    the trapezoid rule, normalised to F(sin theta) = 1."""
    rmax = math.sin(theta)
    r = np.linspace(0.0, rmax, nodes)
    arg = np.clip(math.cos(theta) / np.sqrt(1.0 - r * r), -1.0, 1.0)
    Lr = 2.0 * np.arccos(arg)
    rho = r * Lr
    F = np.concatenate([[0.0], np.cumsum(0.5 * (rho[1:] + rho[:-1]) * np.diff(r))])
    F /= F[-1]
    return r, F


def geoball_sf(n, q0, theta, nodes=4097):
    """Algorithm 1 (GeoBall-SF): n low-discrepancy unit quaternions uniformly
    distributed in B(q0, theta).  gamma of u1 = s/gamma mod 1 is taken as n."""
    r_tab, F_tab = geoball_radial_table(theta, nodes)
    out = np.empty((n, 4))
    for i in range(n):
        s = i + 0.5
        u1 = (s / n) % 1.0
        u2 = (s / SF_PHI) % 1.0
        u3 = (s / SF_PSI) % 1.0
        r = float(np.interp(u1, F_tab, r_tab))
        R = math.sqrt(1.0 - r * r)
        Lr = 2.0 * math.acos(min(1.0, math.cos(theta) / R))
        al = (u2 - 0.5) * Lr
        be = 2.0 * math.pi * u3
        ql = np.array([R * math.cos(al), R * math.sin(al), r * math.cos(be), r * math.sin(be)])
        out[i] = quat_mul(q0, ql)
    return out


def nn_rotation_angles(quats):
    """Nearest-neighbour rotation angle (radians, 2 x Eq. (10)) per sample."""
    q = np.asarray(quats)
    G = np.abs(q @ q.T)
    np.fill_diagonal(G, -1.0)
    c = np.clip(G.max(axis=1), -1.0, 1.0)
    return 2.0 * np.arccos(c)


# ----------------------------------------------------------------------------
# refinement, Sec. V
# ----------------------------------------------------------------------------

def refine_params(r, L, iters=60):
    return np.array([r, L, TAU_OUT2, TAU_IN2, K_SLOPE, LAMBDA, MU, iters, 0, 0,
                     ITERS, STEP_T, STEP_R, B_T, B_R, DECAY], dtype=np.float64)


def probe_sdf(x, r, L):
    x = _c64(x)
    g = np.empty(3)
    f = lib().orc_probe_sdf(_p(x), ctypes.c_double(r), ctypes.c_double(L), _p(g))
    return f, g


def probe_normal(x, r, L):
    x = _c64(x)
    n = np.empty(3)
    lib().orc_probe_normal(_p(x), ctypes.c_double(r), ctypes.c_double(L), _p(n))
    return n


def tri_min(v0, v1, v2, r, L, iters=60):
    v0, v1, v2 = _c64(v0), _c64(v1), _c64(v2)
    lam = np.empty(3)
    d = lib().orc_tri_min(_p(v0), _p(v1), _p(v2), ctypes.c_double(r), ctypes.c_double(L), ctypes.c_int(iters),
                          _p(lam))
    return d, lam


def score(d, tau_out=TAU_OUT2, tau_in=TAU_IN2, k=K_SLOPE):
    s, s1, s2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_score(ctypes.c_double(d), ctypes.c_double(tau_out), ctypes.c_double(tau_in), ctypes.c_double(k),
                    ctypes.byref(s), ctypes.byref(s1), ctypes.byref(s2))
    return s.value, s1.value, s2.value


def so3_exp_V(w):
    w = _c64(w)
    R = np.empty(9)
    V = np.empty(9)
    lib().orc_so3_exp_V(_p(w), _p(R), _p(V))
    return R.reshape(3, 3), V.reshape(3, 3)


def pose_of_xi(R0, p0, anchor, xi):
    R0, p0, a, xi = _c64(R0), _c64(p0), _c64(anchor), _c64(xi)
    R = np.empty(9)
    p = np.empty(3)
    lib().orc_pose_of_xi(_p(R0), _p(p0), _p(a), _p(xi), _p(R), _p(p))
    return R.reshape(3, 3), p


def distances(verts, tris, poses, R, p, r, L, eps=TAU_OUT2, iters=60):
    V = _c64(verts)
    T = np.ascontiguousarray(tris, dtype=np.int32)
    P = _c64(poses)
    R = _c64(R)
    p = _c64(p)
    n = len(P)
    d = np.empty(n)
    w = np.empty((n, 3))
    nn = np.empty((n, 3))
    tri = np.empty(n, dtype=np.int64)
    lib().orc_distances(_p(V), ctypes.c_int64(len(V)), _p(T, _ip), ctypes.c_int64(len(T)), _p(P), ctypes.c_int64(n),
                        _p(R), _p(p), ctypes.c_double(r), ctypes.c_double(L), ctypes.c_double(eps),
                        ctypes.c_int(iters), _p(d), _p(w), _p(nn), _p(tri, _i64p))
    return d, w, nn, tri


def objective(verts, tris, poses, R0, p0, anchor, xi, prm):
    V = _c64(verts)
    T = np.ascontiguousarray(tris, dtype=np.int32)
    P = _c64(poses)
    R0, p0, a, xi, prm = _c64(R0), _c64(p0), _c64(anchor), _c64(xi), _c64(prm)
    G = np.empty(6)
    H = np.empty(36)
    d = np.empty(len(P))
    J = lib().orc_objective(_p(V), ctypes.c_int64(len(V)), _p(T, _ip), ctypes.c_int64(len(T)), _p(P),
                            ctypes.c_int64(len(P)), _p(R0), _p(p0), _p(a), _p(xi), _p(prm), _p(G), _p(H), _p(d))
    return J, G, H.reshape(6, 6), d


def refine(verts, tris, poses, R0, p0, anchor, prm):
    V = _c64(verts)
    T = np.ascontiguousarray(tris, dtype=np.int32)
    P = _c64(poses)
    R0, p0, a, prm = _c64(R0), _c64(p0), _c64(anchor), _c64(prm)
    xi = np.empty(6)
    hist = np.empty(int(prm[10]))
    J = lib().orc_refine(_p(V), ctypes.c_int64(len(V)), _p(T, _ip), ctypes.c_int64(len(T)), _p(P),
                         ctypes.c_int64(len(P)), _p(R0), _p(p0), _p(a), _p(prm), _p(xi), _p(hist))
    R, p = pose_of_xi(R0, p0, anchor, xi)
    return dict(J=J, xi=xi, R=R, p=p, J_hist=hist)


def refine_lbfgsb(verts, tris, poses, R0, p0, anchor, prm, b_t=B_T, b_r=B_R, maxiter=200, pgtol=1e-5,
                  ftol=2.220446049250313e-09, m=8):
    """Sec. V-C as printed: J(xi) of Eq. (19) minimised by L-BFGS-B (Byrd,
    Lu, Nocedal and Zhu, 1995; scipy's implementation is the library step)
    from xi_0 = 0 under the box of Eq. (20), with the analytic gradient of
    Eq. (28); it stops on the projected-gradient norm (pgtol) or the relative
    decrease of J (ftol)."""
    from scipy.optimize import minimize

    def fun(x):
        J, G, _, _ = objective(verts, tris, poses, R0, p0, anchor, x, prm)
        return J, G

    bounds = [(-b_t, b_t)] * 3 + [(-b_r, b_r)] * 3
    res = minimize(fun, np.zeros(6), jac=True, method="L-BFGS-B", bounds=bounds,
                   options=dict(maxiter=maxiter, gtol=pgtol, ftol=ftol, maxcor=m))
    R, p = pose_of_xi(R0, p0, anchor, res.x)
    return dict(J=float(res.fun), xi=res.x, R=R, p=p, nit=int(res.nit), nfev=int(res.nfev), G=res.jac)


def chol6(H, b):
    H, b = _c64(H), _c64(b)
    x = np.empty(6)
    rc = lib().orc_chol6(_p(H), _p(b), _p(x))
    return x if rc == 0 else None


def mesh_anchor(verts):
    """Anchor a = geometry centre of the mesh, read as its AABB centre."""
    V = np.asarray(verts)
    return 0.5 * (V.min(axis=0) + V.max(axis=0))
