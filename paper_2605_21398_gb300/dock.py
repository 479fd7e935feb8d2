"""Thin ctypes binding of the docking C ABI (include/dock.h).

Argument marshalling only: every step of the registration path runs in the
CUDA library.  The library is loaded from paper_2605_21398_gb300/_build; if it
is missing the import of this module raises instead of falling back to
anything else.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdock.so")

OK, PENDING = 0, 1
E_INVALID, E_NOMEM, E_TOO_LARGE, E_CUDA, E_CUDA_FATAL, E_TIMEOUT, E_CANCELLED, E_BUSY, E_OVERFLOW = \
    -1, -2, -3, -4, -5, -6, -7, -8, -9
SAMPLER_SF, SAMPLER_HOPF, SAMPLER_GEOBALL, SAMPLER_EXPLICIT = 0, 1, 2, 3
SOLVER_GAUSS_NEWTON, SOLVER_LBFGSB = 0, 1


class DockError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("dock status %d: %s" % (status, msg))
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("tau_out1", ctypes.c_double), ("tau_in1", ctypes.c_double), ("deep_value", ctypes.c_double),
                ("tau_out2", ctypes.c_double), ("tau_in2", ctypes.c_double), ("k_slope", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("mu", ctypes.c_double), ("b_t", ctypes.c_double),
                ("b_r", ctypes.c_double), ("step_t", ctypes.c_double), ("step_r", ctypes.c_double),
                ("iters", ctypes.c_int32), ("tri_iters", ctypes.c_int32), ("solver", ctypes.c_int32),
                ("lbfgs_evals", ctypes.c_int32), ("lbfgs_pgtol", ctypes.c_double), ("lbfgs_ftol", ctypes.c_double)]


class Probe(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("radius", ctypes.c_double), ("length", ctypes.c_double)]


class Candidate(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double * 4), ("t", ctypes.c_double * 3), ("score", ctypes.c_float),
                ("rot", ctypes.c_int32), ("dk", ctypes.c_int32 * 3), ("canvas_idx", ctypes.c_int32)]


class Peak(ctypes.Structure):
    _fields_ = [("score", ctypes.c_float), ("canvas_idx", ctypes.c_int32)]


class SearchDesc(ctypes.Structure):
    _fields_ = [("sampler", ctypes.c_int32), ("n", ctypes.c_int32), ("quats", ctypes.POINTER(ctypes.c_double)),
                ("q0", ctypes.c_double * 4), ("theta", ctypes.c_double), ("gamma", ctypes.c_double),
                ("top_k", ctypes.c_int32), ("rot_begin", ctypes.c_int32), ("rot_end", ctypes.c_int32),
                ("batch", ctypes.c_int32)]


class Refined(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double * 4), ("t", ctypes.c_double * 3), ("xi", ctypes.c_double * 6),
                ("J", ctypes.c_double), ("cand", ctypes.c_int32), ("iters", ctypes.c_int32)]


class RegisterDesc(ctypes.Structure):
    _fields_ = [("n_global", ctypes.c_int32), ("n_local", ctypes.c_int32), ("theta", ctypes.c_double),
                ("top_k", ctypes.c_int32), ("sampler", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double * 4), ("t", ctypes.c_double * 3), ("J", ctypes.c_double),
                ("best_cand", ctypes.c_int32), ("n_evals", ctypes.c_int32), ("best_search", Candidate),
                ("latency_ms", ctypes.c_double), ("first_pass", ctypes.c_int64), ("last_pass", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("obj", ctypes.c_void_p), ("sweep", ctypes.c_void_p), ("desc", RegisterDesc)]


class Tuning(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("batch", ctypes.c_int32), ("group", ctypes.c_int32),
                ("vox_blocks", ctypes.c_int32), ("plane_cl", ctypes.c_int32), ("zpass_cols", ctypes.c_int32),
                ("vox_overlap", ctypes.c_int32), ("zpass_tc", ctypes.c_int32),
                ("plane_tma", ctypes.c_int32), ("fwd_runs", ctypes.c_int32), ("fft_plan", ctypes.c_int32),
                ("us_per_rotation", ctypes.c_double)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_lib = None

# (name, restype, argtypes)
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_st = ctypes.c_int32
SIGNATURES = [
    ("dock_create", _st, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t, _vp]),
    ("dock_destroy", None, [_vp]),
    ("dock_last_error", ctypes.c_char_p, [_vp]),
    ("dock_params_default", None, [ctypes.POINTER(Params)]),
    ("dock_version", ctypes.c_char_p, []),
    ("dock_object_grid", _st, [_vp, _dp, ctypes.c_int64, _ip, ctypes.c_int64, _u8p, ctypes.c_double, ctypes.c_int32,
                               ctypes.POINTER(Params), ctypes.POINTER(_vp)]),
    ("dock_object_free", None, [_vp]),
    ("dock_object_export_grid", _st, [_vp, _vp, _fp, _dp]),
    ("dock_sweep_grid", _st, [_vp, ctypes.POINTER(Probe), _dp, _u8p, ctypes.c_int64, ctypes.c_double, ctypes.c_int32,
                              ctypes.POINTER(_vp)]),
    ("dock_sweep_free", None, [_vp]),
    ("dock_sweep_voxelise", _st, [_vp, _vp, _dp, ctypes.c_int32, _u8p, _dp]),
    ("dock_sweep_set_label_aware", _st, [_vp, _vp, ctypes.c_int32]),
    ("dock_sweep_set_rotate_object", _st, [_vp, _vp, ctypes.c_int32]),
    ("dock_object_rotated", _st, [_vp, _vp, _dp, ctypes.c_int32, _fp, _dp]),
    ("dock_sweep_voxelise_labels", _st, [_vp, _vp, _dp, ctypes.c_int32, _u8p, _u8p, _dp]),
    ("dock_search_so3", _st, [_vp, _vp, _vp, ctypes.POINTER(SearchDesc), ctypes.POINTER(Candidate),
                              ctypes.POINTER(Peak)]),
    ("dock_search_scores", _st, [_vp, _vp, _vp, _dp, _fp]),
    ("dock_search_peaks_noalloc", _st, [_vp, _vp, _vp, _dp, ctypes.c_int32, ctypes.POINTER(Peak)]),
    ("dock_sample_so3", _st, [ctypes.POINTER(SearchDesc), _dp]),
    ("dock_refine_se3", _st, [_vp, _vp, _vp, ctypes.POINTER(Candidate), ctypes.c_int32, ctypes.POINTER(Params),
                              ctypes.POINTER(Refined)]),
    ("dock_objective_fwd", _st, [_vp, _vp, _vp, _dp, _vp, ctypes.c_int32, ctypes.POINTER(Params), _vp, _vp, _vp]),
    ("dock_objective_bwd", _st, [_vp, _vp, _vp, _dp, _vp, ctypes.c_int32, ctypes.POINTER(Params), _vp, _vp, _vp]),
    ("dock_distances", _st, [_vp, _vp, _vp, _dp, ctypes.c_int32, ctypes.POINTER(Params), _fp, _fp, _fp]),
    ("dock_register", _st, [_vp, _vp, _vp, ctypes.POINTER(RegisterDesc), ctypes.POINTER(Params),
                            ctypes.POINTER(Result)]),
    ("dock_register_batch", _st, [_vp, ctypes.POINTER(Request), ctypes.c_int32, ctypes.POINTER(Params),
                                  ctypes.POINTER(Result)]),
    ("dock_submit", _st, [_vp, ctypes.POINTER(Request), ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_uint64)]),
    ("dock_poll", _st, [_vp, ctypes.c_uint64, ctypes.POINTER(Result), ctypes.c_int64]),
    ("dock_cancel", _st, [_vp, ctypes.c_uint64]),
    ("dock_autotune", _st, [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_char_p, ctypes.POINTER(Tuning)]),
    ("dock_load_tuning", _st, [_vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32)]),
    ("dock_get_tuning", _st, [_vp, ctypes.c_int32, ctypes.POINTER(Tuning)]),
    ("dock_set_tuning", _st, [_vp, ctypes.POINTER(Tuning)]),
    ("dock_memory_stats", _st, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                ctypes.POINTER(ctypes.c_size_t)]),
    ("dock_fail_allocation", _st, [_vp, ctypes.c_int32]),
    ("dock_test_plane_timeout", _st, [_vp, _vp, _vp, _dp, _fp]),
    ("dock_set_profiling", _st, [_vp, ctypes.c_int]),
    ("dock_get_kernel_stats", ctypes.c_int32, [_vp, ctypes.POINTER(KernelStat), ctypes.c_int32]),
    ("dock_reset_kernel_stats", None, [_vp]),
]


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("the CUDA library %s is not built; run paper_2605_21398_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the legacy default stream


def stream_arg(stream):
    """A CUDA stream handle for the ABI.  torch reports its legacy default
    stream as 0, which the ABI would read as 'the context stream'."""
    return ctypes.c_void_p(CUDA_STREAM_LEGACY if not stream else stream)


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def default_params():
    p = Params()
    lib().dock_params_default(ctypes.byref(p))
    return p


class Context:
    """A library context on one device and stream."""

    def __init__(self, device=0, hbm_budget=0, stream=None):
        h = _vp()
        st = lib().dock_create(ctypes.byref(h), device, hbm_budget, stream)
        if st != OK:
            raise DockError(st, "dock_create failed")
        self.h = h
        self._children = weakref.WeakSet()

    def check(self, st):
        if st < 0:
            raise DockError(st, lib().dock_last_error(self.h).decode())
        return st

    def close(self):
        """Frees the handles made on this context, then the context."""
        if self.h:
            for ch in list(self._children):
                ch.close()
            lib().dock_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- handles
    def object_grid(self, verts, tris, h, N, touchable=None, params=None):
        return DockObject(self, verts, tris, h, N, touchable, params)

    def sweep_grid(self, poses, radius, length, h, N, contact=None):
        return DockSweep(self, poses, radius, length, h, N, contact)

    # ----------------------------------------------------------------- search
    def search_so3(self, obj, sw, n, top_k, sampler=SAMPLER_SF, quats=None, q0=None, theta=0.0, gamma=0.0,
                   rot_range=None, batch=0, want_peaks=False):
        d = SearchDesc()
        d.sampler = sampler
        d.n = n
        keep = None
        if quats is not None:
            keep, d.quats = _d(quats)
        if q0 is not None:
            for i in range(4):
                d.q0[i] = float(q0[i])
        d.theta = theta
        d.gamma = gamma
        d.top_k = top_k
        d.rot_begin, d.rot_end = (rot_range if rot_range is not None else (0, 0))
        d.batch = batch
        out = (Candidate * top_k)()
        peaks = (Peak * n)() if want_peaks else None
        self.check(lib().dock_search_so3(self.h, obj.h, sw.h, ctypes.byref(d), out, peaks))
        del keep
        cands = [candidate_dict(c) for c in out]
        if want_peaks:
            return cands, np.array([(p.score, p.canvas_idx) for p in peaks],
                                   dtype=[("score", np.float32), ("idx", np.int64)])
        return cands

    def search_peaks_noalloc(self, obj, sw, quats):
        """Per-rotation peaks through the entry point that allocates no device
        memory (library-owned scratch; N <= 64, at most 4096 rotations)."""
        q = np.ascontiguousarray(quats, dtype=np.float64).reshape(-1, 4)
        n = q.shape[0]
        peaks = (Peak * max(n, 1))()
        self.check(lib().dock_search_peaks_noalloc(self.h, obj.h, sw.h, q.ctypes.data_as(_dp), n, peaks))
        return np.array([(p.score, p.canvas_idx) for p in peaks[:n]], dtype=[("score", np.float32), ("idx", np.int64)])

    def test_plane_timeout(self, obj, sw, quat):
        """Runs the search of one rotation with the cluster plane pass's peer
        blocks withheld (its bounded waits run out); raises DockError (E_TIMEOUT)."""
        M = 2 * obj.N
        C = np.empty((M, M, M), dtype=np.float32)
        q, qp = _d(quat)
        self.check(lib().dock_test_plane_timeout(self.h, obj.h, sw.h, qp, C.ctypes.data_as(_fp)))
        return C

    def search_scores(self, obj, sw, quat):
        M = 2 * obj.N
        C = np.empty((M, M, M), dtype=np.float32)
        q, qp = _d(quat)
        self.check(lib().dock_search_scores(self.h, obj.h, sw.h, qp, C.ctypes.data_as(_fp)))
        return C

    # ------------------------------------------------------------- refinement
    def refine_se3(self, obj, sw, cands, params=None):
        K = len(cands)
        arr = (Candidate * K)()
        for i, c in enumerate(cands):
            arr[i] = candidate_struct(c)
        out = (Refined * K)()
        p = params or default_params()
        self.check(lib().dock_refine_se3(self.h, obj.h, sw.h, arr, K, ctypes.byref(p), out))
        return [dict(q=np.array(o.q[:]), t=np.array(o.t[:]), xi=np.array(o.xi[:]), J=o.J, cand=o.cand,
                     iters=o.iters) for o in out]

    def distances(self, obj, sw, obj_poses, params=None):
        P = np.ascontiguousarray(obj_poses, dtype=np.float64).reshape(-1, 7)
        B = len(P)
        n = sw.P
        d = np.empty((B, n), dtype=np.float32)
        w = np.empty((B, n, 3), dtype=np.float32)
        nn = np.empty((B, n, 3), dtype=np.float32)
        p = params or default_params()
        self.check(lib().dock_distances(self.h, obj.h, sw.h, P.ctypes.data_as(_dp), B, ctypes.byref(p),
                                        d.ctypes.data_as(_fp), w.ctypes.data_as(_fp), nn.ctypes.data_as(_fp)))
        return d, w, nn

    def objective_fwd(self, obj, sw, base_poses, xi_ptr, B, J_ptr, grad_ptr, stream, params=None):
        P = np.ascontiguousarray(base_poses, dtype=np.float64).reshape(-1, 7)
        p = params or default_params()
        self.check(lib().dock_objective_fwd(self.h, obj.h, sw.h, P.ctypes.data_as(_dp), ctypes.c_void_p(xi_ptr), B,
                                            ctypes.byref(p), ctypes.c_void_p(J_ptr),
                                            ctypes.c_void_p(grad_ptr) if grad_ptr else None,
                                            stream_arg(stream)))

    def objective_bwd(self, obj, sw, base_poses, xi_ptr, B, gJ_ptr, gxi_ptr, stream, params=None):
        P = np.ascontiguousarray(base_poses, dtype=np.float64).reshape(-1, 7)
        p = params or default_params()
        self.check(lib().dock_objective_bwd(self.h, obj.h, sw.h, P.ctypes.data_as(_dp), ctypes.c_void_p(xi_ptr), B,
                                            ctypes.byref(p), ctypes.c_void_p(gJ_ptr), ctypes.c_void_p(gxi_ptr),
                                            stream_arg(stream)))

    def register(self, obj, sw, n_global, n_local, theta, top_k, sampler=SAMPLER_SF, params=None):
        d = RegisterDesc(n_global, n_local, theta, top_k, sampler)
        r = Result()
        p = params or default_params()
        self.check(lib().dock_register(self.h, obj.h, sw.h, ctypes.byref(d), ctypes.byref(p), ctypes.byref(r)))
        return result_dict(r)

    @staticmethod
    def _request(rq):
        obj, sw, ng, nl, th, k = rq[:6]
        smp = rq[6] if len(rq) > 6 else SAMPLER_SF
        return Request(obj.h, sw.h, RegisterDesc(ng, nl, th, k, smp))

    def submit(self, request, params=None):
        """Queue one registration (obj, sweep, n_global, n_local, theta, top_k[, sampler]); returns a ticket."""
        r = self._request(request)
        p = params or default_params()
        t = ctypes.c_uint64()
        self.check(lib().dock_submit(self.h, ctypes.byref(r), ctypes.byref(p), ctypes.byref(t)))
        return t.value

    def poll(self, ticket, timeout_us=0):
        """Result dict when done, None while pending; raises DockError on a failed or cancelled request."""
        r = Result()
        st = lib().dock_poll(self.h, ticket, ctypes.byref(r), int(timeout_us))
        if st == 1:
            return None
        self.check(st)
        return result_dict(r)

    def cancel(self, ticket):
        self.check(lib().dock_cancel(self.h, ticket))

    def register_batch(self, requests, params=None):
        """requests: list of (obj, sweep, n_global, n_local, theta, top_k[, sampler]); one result per request."""
        n = len(requests)
        arr = (Request * n)()
        for i, rq in enumerate(requests):
            arr[i] = self._request(rq)
        out = (Result * n)()
        p = params or default_params()
        self.check(lib().dock_register_batch(self.h, arr, n, ctypes.byref(p), out))
        return [result_dict(out[i]) for i in range(n)]

    # -------------------------------------------------------------- tuning
    def autotune(self, obj, sw, n_rot=256, cache_path=None):
        t = Tuning()
        self.check(lib().dock_autotune(self.h, obj.h, sw.h, n_rot,
                                       cache_path.encode() if cache_path else None, ctypes.byref(t)))
        return tuning_dict(t)

    def load_tuning(self, cache_path):
        n = ctypes.c_int32()
        self.check(lib().dock_load_tuning(self.h, cache_path.encode(), ctypes.byref(n)))
        return n.value

    def get_tuning(self, N):
        t = Tuning()
        self.check(lib().dock_get_tuning(self.h, N, ctypes.byref(t)))
        return tuning_dict(t)

    def memory_stats(self):
        """(held, peak, budget) device bytes of the context and its handles."""
        h, p, b = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
        self.check(lib().dock_memory_stats(self.h, ctypes.byref(h), ctypes.byref(p), ctypes.byref(b)))
        return h.value, p.value, b.value

    def fail_allocation(self, n):
        """Host fault injection: the n-th device allocation from now on fails (0 = off)."""
        self.check(lib().dock_fail_allocation(self.h, n))

    def set_tuning(self, **shape):
        """Sets the launch shape of lattice side shape['N'] (other keys as get_tuning)."""
        cur = self.get_tuning(shape["N"])
        cur.update(shape)
        t = Tuning(cur["N"], cur["batch"], cur["group"], cur["vox_blocks"], cur["plane_cl"], cur["zpass_cols"],
                   cur["vox_overlap"], cur["zpass_tc"], cur["plane_tma"], cur["fwd_runs"], cur["fft_plan"],
                   cur["us_per_rotation"])
        self.check(lib().dock_set_tuning(self.h, ctypes.byref(t)))

    # -------------------------------------------------------------- profiling
    def set_profiling(self, on):
        self.check(lib().dock_set_profiling(self.h, 1 if on else 0))

    def kernel_stats(self):
        buf = (KernelStat * 64)()
        n = lib().dock_get_kernel_stats(self.h, buf, 64)
        return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms) for i in range(n)}

    def reset_kernel_stats(self):
        lib().dock_reset_kernel_stats(self.h)


def tuning_dict(t):
    return dict(N=t.N, batch=t.batch, group=t.group, vox_blocks=t.vox_blocks, plane_cl=t.plane_cl,
                zpass_cols=t.zpass_cols, vox_overlap=t.vox_overlap, zpass_tc=t.zpass_tc, plane_tma=t.plane_tma,
                fwd_runs=t.fwd_runs, fft_plan=t.fft_plan,
                us_per_rotation=t.us_per_rotation)


def result_dict(r):
    return dict(q=np.array(r.q[:]), t=np.array(r.t[:]), J=r.J, best_cand=r.best_cand, n_evals=r.n_evals,
                best_search=candidate_dict(r.best_search), latency_ms=r.latency_ms, first_pass=r.first_pass,
                last_pass=r.last_pass)


def candidate_dict(c):
    return dict(q=np.array(c.q[:]), t=np.array(c.t[:]), score=float(c.score), rot=int(c.rot),
                dk=np.array(c.dk[:], dtype=np.int64), canvas_idx=int(c.canvas_idx))


def candidate_struct(d):
    c = Candidate()
    for i in range(4):
        c.q[i] = float(d["q"][i])
    for i in range(3):
        c.t[i] = float(d["t"][i])
        c.dk[i] = int(d.get("dk", [0, 0, 0])[i])
    c.score = float(d.get("score", 0.0))
    c.rot = int(d.get("rot", -1))
    c.canvas_idx = int(d.get("canvas_idx", -1))
    return c


class DockObject:
    def __init__(self, ctx, verts, tris, h, N, touchable=None, params=None):
        self.ctx = ctx
        V, Vp = _d(verts)
        T = np.ascontiguousarray(tris, dtype=np.int32)
        tp = None
        if touchable is not None:
            touchable = np.ascontiguousarray(touchable, dtype=np.uint8)
            tp = touchable.ctypes.data_as(_u8p)
        h_ = _vp()
        p = params or default_params()
        ctx.check(lib().dock_object_grid(ctx.h, Vp, len(V), T.ctypes.data_as(_ip), len(T), tp, h, N, ctypes.byref(p),
                                         ctypes.byref(h_)))
        self.h = h_
        ctx._children.add(self)
        self.N = N
        self.hvox = h

    def export_grid(self):
        N = self.N
        G = np.empty((N, N, N), dtype=np.float32)
        o = np.empty(3)
        self.ctx.check(lib().dock_object_export_grid(self.ctx.h, self.h, G.ctypes.data_as(_fp), o.ctypes.data_as(_dp)))
        return G, o

    def rotated(self, quats):
        """(O_R, o_R) per quaternion: the grid rotated and resampled by trilinear
        interpolation, as the rotated-object search builds it."""
        q, qp = _d(quats)
        q = q.reshape(-1, 4)
        n, N = len(q), self.N
        G = np.empty((n, N, N, N), dtype=np.float32)
        o = np.empty((n, 3))
        self.ctx.check(lib().dock_object_rotated(self.ctx.h, self.h, qp, n, G.ctypes.data_as(_fp),
                                                 o.ctypes.data_as(_dp)))
        return G, o

    def close(self):
        # a handle is freed before its context (Context.close frees it first)
        if self.h and self.ctx.h:
            lib().dock_object_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DockSweep:
    def __init__(self, ctx, poses, radius, length, h, N, contact=None):
        self.ctx = ctx
        P, Pp = _d(poses)
        P = P.reshape(-1, 7)
        cp = None
        if contact is not None:
            contact = np.ascontiguousarray(contact, dtype=np.uint8)
            cp = contact.ctypes.data_as(_u8p)
        pr = Probe(0, radius, length)
        h_ = _vp()
        ctx.check(lib().dock_sweep_grid(ctx.h, ctypes.byref(pr), Pp, cp, len(P), h, N, ctypes.byref(h_)))
        self.h = h_
        ctx._children.add(self)
        self.N = N
        self.P = len(P)

    def voxelise(self, quats):
        q, qp = _d(quats)
        q = q.reshape(-1, 4)
        n = len(q)
        N = self.N
        bits = np.empty((n, N, N, N), dtype=np.uint8)
        orig = np.empty((n, 3))
        self.ctx.check(lib().dock_sweep_voxelise(self.ctx.h, self.h, qp, n, bits.ctypes.data_as(_u8p),
                                                 orig.ctypes.data_as(_dp)))
        return bits, orig

    def set_label_aware(self, on=True):
        """Score contact poses with O and non-contact poses with min(O, 0)."""
        self.ctx.check(lib().dock_sweep_set_label_aware(self.ctx.h, self.h, int(bool(on))))

    def set_rotate_object(self, on=True):
        """Rotate and resample the object grid per sample (S fixed) instead of
        voxelising the rotated sweep."""
        self.ctx.check(lib().dock_sweep_set_rotate_object(self.ctx.h, self.h, int(bool(on))))

    def voxelise_labels(self, quats):
        """(S_c, S_n, origins): voxels swept by contact poses, voxels swept
        only by non-contact poses."""
        q, qp = _d(quats)
        q = q.reshape(-1, 4)
        n = len(q)
        N = self.N
        bc = np.empty((n, N, N, N), dtype=np.uint8)
        bn = np.empty((n, N, N, N), dtype=np.uint8)
        orig = np.empty((n, 3))
        self.ctx.check(lib().dock_sweep_voxelise_labels(self.ctx.h, self.h, qp, n, bc.ctypes.data_as(_u8p),
                                                        bn.ctypes.data_as(_u8p), orig.ctypes.data_as(_dp)))
        return bc, bn, orig

    def close(self):
        if self.h and self.ctx.h:
            lib().dock_sweep_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sample_so3(n, sampler=SAMPLER_SF, q0=None, theta=0.0, gamma=0.0, quats=None):
    d = SearchDesc()
    d.sampler = sampler
    d.n = n
    keep = None
    if quats is not None:
        keep, d.quats = _d(quats)
    if q0 is not None:
        for i in range(4):
            d.q0[i] = float(q0[i])
    d.theta = theta
    d.gamma = gamma
    d.top_k = 1
    out = np.empty((n, 4))
    st = lib().dock_sample_so3(ctypes.byref(d), out.ctypes.data_as(_dp))
    del keep
    if st != OK:
        raise DockError(st, "dock_sample_so3 failed")
    return out
