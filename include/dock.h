/*
 * dock.h - C ABI of the GB300 (sm_103a) docking-registration library.
 *
 * Probe-aware contact registration by complementary-shape docking
 * (arxiv 2605.21398).  Given an object mesh, a probe shape and a trajectory of
 * probe poses {T_i} (Sec. III: "a sequence of probe poses ... in which a rigid
 * probe attempts to touch the surface"), the library estimates the object
 * pose T = (R, t) in SE(3) that "best aligns the object with the observed
 * trajectory":
 *   1. global docking search (Sec. IV): for every orientation sample, the
 *      probe's swept volume is voxelised on a lattice rotated by that sample
 *      and correlated over all translations with the object grid by 3-D FFT
 *      (Eq. (5)-(9)); the best peaks survive;
 *   2. local search in a geodesic ball around the best orientation
 *      (Sec. IV-C/D, Algorithm 1);
 *   3. continuous refinement on SE(3) (Sec. V, Eq. (13)-(28)).
 *
 * Conventions
 *   - Units are mm and rad.  A pose is 7 doubles (qw, qx, qy, qz, tx, ty, tz);
 *     probe poses map probe-local points to world points; the returned object
 *     pose maps object-frame points to world points.
 *   - The probe is a flat-ended cylinder: tip face centred at the local
 *     origin, body along +z, z in [0, length], radius `radius`.
 *   - Lattice arrays are indexed (k_z * N + k_y) * N + k_x.
 *   - Host arrays passed in are borrowed for the duration of the call and
 *     copied; they may be freed when the call returns.  Handles are owned by
 *     the caller and released with the matching *_free call.
 *   - Every call returns a dock_status.  A negative status leaves outputs
 *     untouched and sets the context's last-error string.  No C++ exception
 *     crosses this interface.
 *   - Work is issued on the context's CUDA stream; calls that return host
 *     results synchronise that stream before returning.
 */
#ifndef DOCK_H
#define DOCK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#ifndef DOCK_API
#define DOCK_API __attribute__((visibility("default")))
#endif

typedef int32_t dock_status;
#define DOCK_OK            0
#define DOCK_PENDING       1
#define DOCK_E_INVALID    -1   /* bad argument: NaN/Inf, non-unit quaternion, empty input, size out of range */
#define DOCK_E_NOMEM      -2   /* device or host allocation failed */
#define DOCK_E_TOO_LARGE  -3   /* request can never fit the context's HBM budget */
#define DOCK_E_CUDA       -4   /* a CUDA call failed; the context remains usable */
#define DOCK_E_CUDA_FATAL -5   /* sticky CUDA error: the context is dead */
#define DOCK_E_TIMEOUT    -6
#define DOCK_E_CANCELLED  -7
#define DOCK_E_BUSY       -8
#define DOCK_E_OVERFLOW   -9   /* a fixed-capacity device list overflowed (reported, result not trusted) */

typedef struct dock_ctx dock_ctx;
typedef struct dock_object dock_object;
typedef struct dock_sweep dock_sweep;

/* Parameters.  Defaults (dock_params_default) are Table I of Sec. VI plus the
 * readings noted beside each field. */
typedef struct dock_params {
    double tau_out1;     /* Eq. (1)-(2) outer band, mm (Table I: 0.5) */
    double tau_in1;      /* Eq. (1) inner band, mm (Table I: 0.2) */
    double deep_value;   /* Eq. (1) value for f <= -tau_in1 (Table I rho = -50, taken as the value) */
    double tau_out2;     /* Eq. (18) outer threshold, mm (Table I: 0.2); also the Eq. (21) cutoff */
    double tau_in2;      /* Eq. (18) inner threshold, mm (Table I: 0.03); r = tau_in2 / tau_out2 */
    double k_slope;      /* Eq. (18) penalty slope k (15) */
    double lambda;       /* Eq. (19) Tikhonov weight (Table I "10e-4", read as 1e-3) */
    double mu;           /* Gauss-Newton damping added to the normal matrix, mm^-2 (1e-6) */
    double b_t, b_r;     /* Eq. (20) box bounds: |u|_inf <= b_t mm, |w|_inf <= b_r rad (1.0, 5 deg) */
    double step_t, step_r; /* per-iteration trust region on the Gauss-Newton step (0.05 mm, 0.5 deg) */
    int32_t iters;       /* refinement iterations (20); with L-BFGS-B the most accepted steps */
    int32_t tri_iters;   /* inner bisection steps of the per-triangle search (outer golden steps: 1.5x);
                            default 20: u and v to ~1e-6 of the triangle */
    int32_t solver;      /* DOCK_SOLVER_GAUSS_NEWTON (default) or DOCK_SOLVER_LBFGSB (Sec. V-C as printed) */
    int32_t lbfgs_evals; /* L-BFGS-B: most evaluations of J and grad J per candidate (100) */
    double lbfgs_pgtol;  /* L-BFGS-B: stop when the largest projected-gradient component is below (1e-5) */
    double lbfgs_ftol;   /* L-BFGS-B: stop when the relative decrease of J is below (2.2e-9) */
} dock_params;

/*
 * Refinement solvers.  GAUSS_NEWTON: `iters` projected Gauss-Newton steps
 * (FP64 6x6 Cholesky, trust region step_t / step_r, the box of Eq. (20)).
 * LBFGSB: limited-memory BFGS with the box of Eq. (20), from xi_0 = 0 with
 * the analytic gradient of Eq. (28) (Sec. V-C): 8 stored pairs, two-loop
 * direction on the variables not held at a bound, projected Armijo
 * backtracking (safeguarded quadratic interpolation); a candidate stops on lbfgs_pgtol, lbfgs_ftol, `iters`
 * accepted steps, lbfgs_evals evaluations or a failed line search (the
 * objective has kinks where the witness triangle changes), keeping its last
 * accepted twist.  dock_refined.iters reports the accepted steps.
 */
#define DOCK_SOLVER_GAUSS_NEWTON 0
#define DOCK_SOLVER_LBFGSB 1

typedef struct dock_probe {
    int32_t kind;        /* 0 = flat-ended cylinder (the paper's bur, Sec. VI) */
    double radius;       /* mm */
    double length;       /* mm */
} dock_probe;

/* One surviving docking peak (Sec. IV-B/D, Eq. (8)). */
typedef struct dock_candidate {
    double q[4];         /* sampled orientation (w, x, y, z) */
    double t[3];         /* translation R (h dk + o_s - o_o) */
    float score;         /* correlation peak C[dk] (Eq. (7)) */
    int32_t rot;         /* index of the orientation sample */
    int32_t dk[3];       /* voxel shift (x, y, z), each in [-N, N-1] */
    int32_t canvas_idx;  /* (c_z * M + c_y) * M + c_x on the M^3 canvas */
} dock_candidate;

/* Per-rotation peak (test and sharding hook). */
typedef struct dock_peak {
    float score;
    int32_t canvas_idx;
} dock_peak;

enum { DOCK_SAMPLER_SF = 0, DOCK_SAMPLER_HOPF = 1, DOCK_SAMPLER_GEOBALL = 2, DOCK_SAMPLER_EXPLICIT = 3 };

typedef struct dock_search_desc {
    int32_t sampler;     /* DOCK_SAMPLER_* */
    int32_t n;           /* number of orientation samples */
    const double *quats; /* EXPLICIT: n x 4 unit quaternions (host), else NULL */
    double q0[4];        /* GEOBALL: ball centre */
    double theta;        /* GEOBALL: ball radius, quaternion half-angle (Eq. (10); Table I: 5 deg) */
    double gamma;        /* GEOBALL: Algorithm 1 constant gamma (0 = n, the default reading) */
    int32_t top_k;       /* candidates kept, 1..1024 */
    int32_t rot_begin;   /* shard: evaluate samples [rot_begin, rot_end); rot_end = 0 means n */
    int32_t rot_end;
    int32_t batch;       /* rotations per pipeline batch (0 = automatic) */
} dock_search_desc;

/* Refined pose (Sec. V). */
typedef struct dock_refined {
    double q[4];         /* refined object orientation */
    double t[3];         /* refined object translation */
    double xi[6];        /* final twist (u, w) of Eq. (13) relative to the candidate */
    double J;            /* Eq. (19) at xi */
    int32_t cand;        /* index of the candidate it started from */
    int32_t iters;
} dock_refined;

typedef struct dock_register_desc {
    int32_t n_global;    /* global SF samples (Table I n_g) */
    int32_t n_local;     /* local GeoBall-SF samples (Table I n_l; 0 = no local stage) */
    double theta;        /* local ball radius (quaternion half-angle) */
    int32_t top_k;       /* candidates refined */
    int32_t sampler;     /* global sampler: DOCK_SAMPLER_SF or DOCK_SAMPLER_HOPF */
} dock_register_desc;

typedef struct dock_result {
    double q[4], t[3];   /* final object pose (object -> world) */
    double J;            /* objective at the final pose */
    int32_t best_cand;   /* candidate index that won the refinement */
    int32_t n_evals;     /* orientation samples evaluated */
    dock_candidate best_search; /* best candidate of the search stages */
    double latency_ms;   /* submission (or call) to completion, host clock */
    int64_t first_pass;  /* engine search passes (counted per context) that this request */
    int64_t last_pass;   /* first and last took part in */
} dock_result;

/* ---------------------------------------------------------------- context */

/* Create a context on `device`.  hbm_budget_bytes bounds the device memory
 * the context may hold (0 = no bound).  cuda_stream is a cudaStream_t or NULL
 * for a stream the context creates and owns. */
DOCK_API dock_status dock_create(dock_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream);
/* Device memory (bytes) the context and its handles hold now, the most they
 * have held at any time since dock_create, and the budget (0 = none); any
 * pointer may be NULL.  Systems form (serving admission); the paper has no
 * counterpart. */
DOCK_API dock_status dock_memory_stats(dock_ctx *ctx, size_t *held, size_t *peak, size_t *budget);
/* Fault injection on the host: the n-th device allocation the context makes
 * from now on fails as if cudaMalloc had answered out of memory (the call
 * that makes it returns DOCK_E_NOMEM and the context stays usable); n = 0
 * turns it off.  No device fault is involved.  DOCK_E_INVALID for n < 0. */
DOCK_API dock_status dock_fail_allocation(dock_ctx *ctx, int32_t n);
DOCK_API void dock_destroy(dock_ctx *ctx);
/* Last error message of the context (valid until the next call on ctx). */
DOCK_API const char *dock_last_error(const dock_ctx *ctx);
DOCK_API void dock_params_default(dock_params *p);
/* Library version string. */
DOCK_API const char *dock_version(void);

/* ----------------------------------------------------------------- object */

/*
 * Object grid O[k] = min(O_t, O_m)(h k + o_o) of Sec. IV-A.1, Eq. (1)-(4),
 * and its canvas spectrum conj(F(O)) for Eq. (9), kept resident on the device.
 *   verts    V x 3 doubles (object frame, mm); tris T x 3 int32 (watertight,
 *            any orientation); touchable: T bytes marking the touchable
 *            sub-mesh of Eq. (2), or NULL for all triangles.
 *   h, N     voxel size and lattice side; N in {32, 64, 96, 128}.  The
 *            canvas side is M = 2 N (Sec. IV-B: n_o + n_s - 1 <= M).
 *   o_o      = h round(c / h) - (N/2) h, c = the mesh AABB centre.
 * The SDF is the exact point-triangle distance with the sign from the parity
 * of +x ray crossings.  Returns DOCK_E_INVALID when the mesh AABB widened by
 * tau_out1 does not fit the lattice.  Also builds the BVH used by the
 * refinement (Sec. V-B) and sets the anchor a = AABB centre (Sec. V-A).
 */
DOCK_API dock_status dock_object_grid(dock_ctx *ctx, const double *verts, int64_t V, const int32_t *tris, int64_t T,
                             const uint8_t *touchable, double h, int32_t N, const dock_params *params,
                             dock_object **out);
DOCK_API void dock_object_free(dock_object *obj);   /* before dock_destroy of its context */
/* Copy O (N^3 floats) and o_o (3 doubles) to host memory (test hook). */
DOCK_API dock_status dock_object_export_grid(dock_ctx *ctx, const dock_object *obj, float *grid, double *origin);

/* ------------------------------------------------------------------ sweep */

/*
 * Probe + trajectory of Sec. IV-A.2 (Eq. (5)-(6)), resident on the device.
 *   poses    P x 7 doubles, probe -> world; quaternions must be unit (1e-6).
 *   contact  P labels (1 = contact, 0 = non-contact) or NULL (all contact).
 *            Eq. (5) takes the max over all poses, so the labels do not change
 *            the search unless dock_sweep_set_label_aware switches it on.
 *   h, N     must equal the object's when used together.
 * The swept lattice for an orientation sample R has origin
 * o_s,R = h round(R^T c_s / h) - (N/2) h, c_s = mean tip position.
 */
DOCK_API dock_status dock_sweep_grid(dock_ctx *ctx, const dock_probe *probe, const double *poses, const uint8_t *contact,
                            int64_t P, double h, int32_t N, dock_sweep **out);
DOCK_API void dock_sweep_free(dock_sweep *sw);
/* Voxelise S_R for `n` quaternions (host n x 4) into host `bits`
 * (n x N^3 bytes, 0/1) and their origins (n x 3 doubles).  Test hook. */
DOCK_API dock_status dock_sweep_voxelise(dock_ctx *ctx, const dock_sweep *sw, const double *quats, int32_t n,
                                uint8_t *bits, double *origins);

/*
 * Label-aware score (a use of the trajectory's contact labels; Sec. I and
 * Sec. IV-A: a trajectory holds contact and non-contact evidence).  With
 * on = 1, searches and registrations of this sweep that start after the call
 * (a submitted request keeps the mode it was submitted with) correlate
 *     C[dk] = sum_k O[k] S_c[k + dk] + sum_k min(O[k], 0) S_n[k + dk],
 * S_c = the voxels swept by contact poses, S_n = the voxels swept only by
 * non-contact poses (S_c + S_n = the plain S of Eq. (5)-(6), on the same
 * lattice o_s,R of all poses): a pose that did not touch the object may not
 * overlap its interior but earns nothing near its surface.  A sweep whose
 * poses are all contact scores as before.  The refinement (Sec. V) is
 * unchanged.  The first label-aware search of an object computes and keeps
 * conj(F(min(O, 0))) beside its spectrum (the same size).  Default 0 (Eq. (7)
 * over all poses).  dock_search_peaks_noalloc rejects a label-aware sweep
 * (DOCK_E_INVALID).  Returns DOCK_E_INVALID for on outside {0, 1} and for
 * on = 1 while dock_sweep_set_rotate_object is on.
 */
DOCK_API dock_status dock_sweep_set_label_aware(dock_ctx *ctx, dock_sweep *sw, int32_t on);

/*
 * The rotation mechanism as Sec. IV-D prints it.  With on = 1, searches and
 * registrations of this sweep that start after the call rotate the object
 * grid instead of the swept volume: S is voxelised once, on the
 * world-aligned lattice o_s = h round(c_s / h) - (N/2) h, and for each
 * orientation sample R
 *     O_R[k] = trilinear interpolant of O at R^T (h k + o_R) (zero outside
 *              O's lattice), o_R = h round(R c_o / h) - (N/2) h,
 *              c_o = o_o + (N/2) h;
 *     C[dk] = sum_k O_R[k] S[k + dk]  (Eq. (7));
 *     pose T = (R, h dk + o_s - o_R).
 * The first such search of a sweep computes and keeps F(S) / M^3 (the size
 * of an object spectrum).  Interpolation blends the -50 interior into the
 * contact band by up to a voxel, so scores differ from the default (which
 * voxelises the rotated sweep exactly); at rotations that map the lattice
 * onto itself the two agree.  Default 0.  Excludes the label-aware score
 * (DOCK_E_INVALID while it is on); dock_search_peaks_noalloc rejects such a
 * sweep.  Returns DOCK_E_INVALID for on outside {0, 1}.
 */
DOCK_API dock_status dock_sweep_set_rotate_object(dock_ctx *ctx, dock_sweep *sw, int32_t on);
/* O_R and o_R above for `n` quaternions into host grids (n x N^3 floats) and
 * origins (n x 3 doubles, nullable).  Test hook. */
DOCK_API dock_status dock_object_rotated(dock_ctx *ctx, const dock_object *obj, const double *quats, int32_t n,
                                         float *grids, double *origins);
/* S_c and S_n above for `n` quaternions into host bits_c, bits_n (n x N^3
 * bytes each, 0/1) and the origins (n x 3 doubles, nullable).  Test hook. */
DOCK_API dock_status dock_sweep_voxelise_labels(dock_ctx *ctx, const dock_sweep *sw, const double *quats, int32_t n,
                                                uint8_t *bits_c, uint8_t *bits_n, double *origins);

/* ----------------------------------------------------------------- search */

/*
 * Docking search over orientation samples (Sec. IV-B..D): for each sample the
 * rotated swept grid is correlated with O over all M^3 canvas shifts
 * (Eq. (7), by FFT per Eq. (9)), the per-rotation argmax (ties: lowest
 * linear index) is kept, and the top_k peaks over rotations (score
 * descending, rotation index ascending) are written to `out` with their
 * poses (Eq. (8) composed with the sample's rotation).  per_rot (host,
 * n entries, nullable) receives every evaluated rotation's peak; entries
 * outside [rot_begin, rot_end) are left untouched.
 */
DOCK_API dock_status dock_search_so3(dock_ctx *ctx, const dock_object *obj, const dock_sweep *sw,
                            const dock_search_desc *desc, dock_candidate *out, dock_peak *per_rot);

/* Full correlation field C (M^3 floats, host) for one quaternion (the
 * label-aware field when the sweep is label-aware).  Test hook. */
DOCK_API dock_status dock_search_scores(dock_ctx *ctx, const dock_object *obj, const dock_sweep *sw, const double *quat,
                               float *C);

/* Orientation samples as the search generates them (host n x 4).  Test hook. */
DOCK_API dock_status dock_sample_so3(const dock_search_desc *desc, double *quats);

/* ------------------------------------------------------------- refinement */

/*
 * Continuous refinement of Sec. V for K candidates: twist xi (Eq. (13)),
 * left perturbation about the anchor (Eq. (14)-(17)), proximity score
 * (Eq. (18), C^1 coefficients), objective (Eq. (19)) under the box
 * (Eq. (20)); per-pose distances by BVH pruning (Eq. (21)) and per-triangle
 * minimisation of f_p (Eq. (22)-(23)); sensitivities (Eq. (24)-(28)).  The
 * solver is a fixed-iteration projected Gauss-Newton step with an FP64 6x6
 * Cholesky solve per candidate (replacing L-BFGS-B).  out[c] is the refined
 * pose of in[c].
 */
DOCK_API dock_status dock_refine_se3(dock_ctx *ctx, const dock_object *obj, const dock_sweep *sw, const dock_candidate *in,
                            int32_t K, const dock_params *params, dock_refined *out);

/*
 * Differentiable form of the refinement objective for B base poses.
 * base_poses: B x 7 host doubles (object -> world), read before the call
 * returns.  xi (B x 6 floats), J (B floats) and grad (B x 6 floats, nullable)
 * are device pointers used on `stream` (a cudaStream_t; NULL = the context
 * stream, cudaStreamLegacy = the legacy default stream); the call returns
 * without synchronising it.  J[b] = Eq. (19) at
 * twist xi[b] about base pose b (anchor a = the object's AABB centre),
 * grad[b] = Eq. (28).
 */
DOCK_API dock_status dock_objective_fwd(dock_ctx *ctx, const dock_object *obj, const dock_sweep *sw,
                                        const double *base_poses, const float *xi, int32_t B,
                                        const dock_params *params, float *J, float *grad, void *stream);

/* Adjoint of dock_objective_fwd: gxi[b] = gJ[b] * grad J(xi[b]) (Eq. (24)-(28)),
 * recomputed by the sensitivity kernel.  gJ, gxi: device pointers. */
DOCK_API dock_status dock_objective_bwd(dock_ctx *ctx, const dock_object *obj, const dock_sweep *sw,
                                        const double *base_poses, const float *xi, int32_t B,
                                        const dock_params *params, const float *gJ, float *gxi, void *stream);

/* Per-pose distances d_i, world witnesses and normals for B object poses
 * (host B x 7) into host arrays (B x P, B x P x 3, B x P x 3).  Test hook. */
DOCK_API dock_status dock_distances(dock_ctx *ctx, const dock_object *obj, const dock_sweep *sw, const double *obj_poses,
                           int32_t B, const dock_params *params, float *d, float *witness, float *normal);

/* ------------------------------------------------------------ registration */

/* The three-stage pipeline of Fig. 2: global search, local search around the
 * best orientation, refinement of the top_k candidates; the lowest-J refined
 * pose wins (ties: lower candidate index). */
DOCK_API dock_status dock_register(dock_ctx *ctx, const dock_object *obj, const dock_sweep *sw, const dock_register_desc *desc,
                          const dock_params *params, dock_result *out);

/* A registration request: object and sweep handles plus its search sizes. */
typedef struct dock_request {
    const dock_object *obj;
    const dock_sweep *sweep;
    dock_register_desc desc;
} dock_request;

/*
 * Batched registration of uneven requests (different lattice sides, trajectory
 * lengths, probes and sample counts; Fig. 2 per request).  Up to 64 requests
 * are in flight at once; requests with the same lattice side N share every
 * search pass: one launch of each fused search kernel takes rotations of
 * several requests, each rotation carrying its request's trajectory, probe
 * and object spectrum, and lattice sides take turns.  Each result equals the
 * request registered alone by dock_register (the arithmetic per rotation is
 * the same).  out receives n results in request order; on an error the call
 * returns the first failing request's status.
 */
DOCK_API dock_status dock_register_batch(dock_ctx *ctx, const dock_request *reqs, int32_t n, const dock_params *params,
                                         dock_result *out);

/*
 * Per-rotation peaks of the docking search for explicit rotations, computed
 * without allocating: for callers that cannot call cudaMalloc (a host
 * framework that owns every device allocation through its own pool, or code
 * that runs where the memory layout has been planned and fixed).  The paper
 * has no counterpart; this is a systems entry point around the same search
 * kernels as dock_search_so3, and each peak equals that call's per-rotation
 * peak for the same quaternion.
 *
 * quats: host, n x 4 unit quaternions (w, x, y, z); peaks: host, n entries
 * out (score, canvas index; -inf and -1 for an empty sweep).  obj and sweep
 * are handles made beforehand by dock_object_grid / dock_sweep_grid on ctx.
 *
 * Scratch: one fixed device array inside the library, about 14 MB, which
 * every GPU that loads the library holds until the process exits.  Limits:
 * lattice side N <= 64 and 1 <= n <= 4096; larger sizes return
 * DOCK_E_INVALID with a message.  The call allocates no device memory (no
 * cudaMalloc, cudaFree or allocating library routine): dock_create looks up
 * the scratch's device address on its device (once per device), which is
 * where a lazily loaded library places the scratch on the GPU.  The call
 * copies from pageable host memory and synchronises ctx's stream, so it
 * returns DOCK_E_INVALID when that stream is being captured.  All calls share
 * the scratch, which keeps the last call's contents: calls that overlap on the
 * GPU (from several threads or contexts on one device) race.  The call runs
 * on ctx's stream and returns after the peaks are on the host.
 */
DOCK_API dock_status dock_search_peaks_noalloc(dock_ctx *ctx, const dock_object *obj, const dock_sweep *sweep,
                                               const double *quats, int32_t n, dock_peak *peaks);

/*
 * Serving (continuous batching).  dock_submit queues a registration and
 * returns at once with a ticket; a serving thread of the context (started by
 * the first submission) admits queued requests between search passes while
 * one of its 64 request slots is free and the context's HBM budget holds the
 * request's device state (quaternions, rotation records, peak keys and
 * candidates: about 200 bytes per orientation sample, plus the shared search
 * scratch of its lattice side).  Admitted requests of the same lattice side
 * share every search pass, each taking an equal share of the pass's
 * rotations, so a request that arrives while others run starts with the next
 * pass.  Results equal dock_register on the same request.
 *
 * The object and sweep handles must stay alive until the request completes.
 * dock_poll waits up to timeout_us (0: no wait, < 0: until done) and returns
 * DOCK_PENDING, or the request's status; a completed ticket is collected by
 * the dock_poll that returns it and is unknown afterwards.  dock_cancel marks
 * a request: a queued one never starts, an admitted one stops at the next
 * pass boundary; its dock_poll returns DOCK_E_CANCELLED.  While the serving
 * thread runs, every other call on the context waits for the pass in flight.
 * dock_destroy cancels what is left.
 */
DOCK_API dock_status dock_submit(dock_ctx *ctx, const dock_request *req, const dock_params *params, uint64_t *ticket);
DOCK_API dock_status dock_poll(dock_ctx *ctx, uint64_t ticket, dock_result *out, int64_t timeout_us);
DOCK_API dock_status dock_cancel(dock_ctx *ctx, uint64_t ticket);

/* ---------------------------------------------------------------- tuning */

/* Launch shape of the search kernels for one lattice side. */
typedef struct dock_tuning {
    int32_t N;               /* lattice side */
    int32_t batch;           /* rotations per launch of the four search kernels */
    int32_t group;           /* rotations per z-pass block sharing one spectrum read (0 = heuristic) */
    int32_t vox_blocks;      /* voxeliser register target: 3 or 4 resident blocks per SM */
    int32_t plane_cl;        /* CTAs per plane of the inverse plane pass (canvas 256 only: 2, 4 or 8;
                                0 = the default; other canvases use one fixed shape) */
    int32_t zpass_cols;      /* columns per z-pass block (canvas 256 only: 16 or 32; 0 = the default) */
    int32_t vox_overlap;     /* 1: the voxeliser of the next launch runs on a second stream, overlapped
                                with the FFT passes of the current one (plain score); 0: in order */
    int32_t zpass_tc;        /* 1: the z pass's radix-16 DFT stages run as 3 x TF32 products on the
                                tensor cores (canvas 256, zpass_cols 16, plain score); 0: FP32
                                butterflies on the CUDA cores */
    int32_t plane_tma;       /* 1 (canvas 256, plane_cl 4 or 8): the plane pass as persistent clusters that
                                load the next plane's columns with the tensor-memory-access unit
                                during the current plane's C2R; 0: one cluster per plane */
    int32_t fwd_runs;        /* 1 (canvas 256): the forward x and y passes of binary slabs from their
                                run lists, 16 kx columns per round (three blocks per SM); 0: all
                                columns of a slab at once (one block per SM) */
    int32_t fft_plan;        /* radix plan of the FFT passes at canvases 64 and 128 (lattice sides 32
                                and 64): 0: 8 x 8 and 16 x 8; 1: 16 x 4 and 8 x 8 x 2 (other canvases:
                                0 only) */
    double us_per_rotation;  /* measured device time per rotation of this shape (0 = not measured) */
} dock_tuning;

/*
 * Autotuner (systems form; the paper has no counterpart).  Times the search
 * kernels on n_rot SF rotations of (obj, sweep) under candidate launch shapes
 * -- the voxeliser's register target, the rotations per launch, the
 * rotations per z-pass block, at canvases 64 and 128 the FFTs' radix plan,
 * and at canvas 256 the FFT passes' variants (plane-pass cluster size and
 * persistent form, z-pass width and tensor-core stages, forward pass from
 * run lists) -- one knob at a time, with CUDA events on the context's
 * stream, and keeps the fastest for obj's lattice side on ctx (all later
 * searches, registrations and serving passes of that side use it).  Results
 * do not depend on the shape beyond FP32 rounding.  With cache_path non-NULL
 * the context's tuned shapes are written there as JSON (with the device
 * name).  Takes about 13 to 18 timed searches of n_rot rotations; n_rot in
 * [16, 65536].
 */
DOCK_API dock_status dock_autotune(dock_ctx *ctx, const dock_object *obj, const dock_sweep *sweep, int32_t n_rot,
                                   const char *cache_path, dock_tuning *out);
/* Loads shapes written by dock_autotune for this device (entries of other
 * devices are skipped); returns the number loaded in *n_loaded. */
DOCK_API dock_status dock_load_tuning(dock_ctx *ctx, const char *cache_path, int32_t *n_loaded);
/* The shape in use for lattice side N (tuned or default). */
DOCK_API dock_status dock_get_tuning(dock_ctx *ctx, int32_t N, dock_tuning *out);
/* Sets the shape for lattice side t->N (batch 1..256, group 0..256,
 * vox_blocks 3 or 4, plane_cl 0, 2, 4 or 8, zpass_cols 0, 16 or 32,
 * vox_overlap 0 or 1, zpass_tc 0 or 1, plane_tma 0 or 1, fwd_runs 0 or 1,
 * fft_plan 0, or 1 for N 32 or 64); results do not depend on it beyond
 * rounding (zpass_tc, fwd_runs and fft_plan change the order of FP32
 * operations, within the error of the transforms).
 * DOCK_E_INVALID for values out of range. */
DOCK_API dock_status dock_set_tuning(dock_ctx *ctx, const dock_tuning *t);

/* Test hook of failure detection (systems form; the paper has no
 * counterpart): dock_search_scores with the cluster plane pass (canvas 256,
 * plane_cl 4 or 8; the persistent form when plane_tma is set) launched so
 * that no CTA receives its peers' blocks.  Every CTA's wait for them is
 * bounded (about a second of clock cycles); it runs out, the kernel records
 * DOCK_E_TIMEOUT in the context's error word (a persistent cluster stops at
 * its next cluster barrier, every CTA told through its shared memory) and
 * returns, and the call returns DOCK_E_TIMEOUT with C undefined.  No copy is
 * in flight when a CTA gives up and the context stays usable.  quat: one
 * unit quaternion; C: host, M^3 floats.  DOCK_E_INVALID for other canvases
 * or plane shapes. */
DOCK_API dock_status dock_test_plane_timeout(dock_ctx *ctx, const dock_object *obj, const dock_sweep *sweep,
                                             const double *quat, float *C);

/* --------------------------------------------------------------- profiling */

/* Per-kernel CUDA-event timing on the context stream (off by default). */
DOCK_API dock_status dock_set_profiling(dock_ctx *ctx, int enable);
/* Copies up to `cap` entries: kernel name (<= 31 chars), launches, total ms. */
typedef struct dock_kernel_stat {
    char name[32];
    int64_t launches;
    double total_ms;
} dock_kernel_stat;
DOCK_API int32_t dock_get_kernel_stats(dock_ctx *ctx, dock_kernel_stat *stats, int32_t cap);
DOCK_API void dock_reset_kernel_stats(dock_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* DOCK_H */
