// Host runtime and C ABI of the docking library (include/dock.h).
//
// Compiled with -ffp-contract=off: the FP64 set-up arithmetic below (probe
// rotation matrices, the trajectory centroid, lattice origins) is rounded
// exactly as written, matching a plain evaluation of the definitions.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <new>
#include <string>
#include <vector>

#include "dock_internal.h"

using namespace dock;

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct ProfEntry {
    std::string name;
    cudaEvent_t a, b;
};

struct KStat {
    int64_t launches = 0;
    double ms = 0.0;
};

struct Engine;

// Device buffers of one refinement launch sequence (grown on demand).
struct RefBufs {
    double *state = nullptr, *acc = nullptr, *prm = nullptr;
    size_t state_n = 0, acc_n = 0, prm_n = 0;
    void *cands = nullptr;
    size_t cands_n = 0;
    RefineDev *dev = nullptr;   // per-request refinement tables of a launch
    size_t dev_n = 0;
    int32_t *hint = nullptr;    // per-query witness triangle of the previous evaluation
    size_t hint_n = 0;
    int32_t *grp = nullptr;     // candidate -> request
    size_t grp_n = 0;
    double *lb = nullptr;       // L-BFGS-B state per candidate (LB_ST doubles)
    size_t lb_n = 0;
    int32_t *active = nullptr;  // L-BFGS-B: candidates still iterating
    size_t active_n = 0;
};

static void free_refbufs(RefBufs &b)
{
    cudaFree(b.state);
    cudaFree(b.acc);
    cudaFree(b.prm);
    cudaFree(b.cands);
    cudaFree(b.dev);
    cudaFree(b.grp);
    cudaFree(b.hint);
    cudaFree(b.lb);
    cudaFree(b.active);
    b = RefBufs();
}

struct dock_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;        // 0 = unbounded
    size_t held = 0;          // bytes currently held by this context and its handles
    size_t peak_held = 0;     // the most held at any time since creation
    std::atomic<int> fail_alloc{0};   // host fault injection: the n-th allocation from now fails (0 = off)
    std::string err;
    std::mutex err_mu;        // err is written by the serving thread too
    bool dead = false;
    // search scratch (grown on demand)
    float2 *Y = nullptr, *Z = nullptr;
    size_t yz_bytes = 0;
    uint32_t *bits = nullptr;
    size_t bits_n = 0;
    float *ogr = nullptr;     // rotated object grids of a launch's rotate_object rotations
    size_t ogr_n = 0;
    unsigned long long *keys = nullptr;
    size_t keys_n = 0;
    RotRec *rots = nullptr;
    size_t rots_n = 0;
    double *quats = nullptr;
    size_t quats_n = 0;
    int *errflag = nullptr;
    // the voxeliser of the next launch overlapped with the FFT passes of the
    // current one: its own stream, double-buffered bits, ordering events
    cudaStream_t vstream = nullptr;
    cudaEvent_t vev[5] = {};   // 0, 1: bits[k] written; 2, 3: bits[k] read by fwd2d; 4: entry
    dock_candidate *cands = nullptr;
    size_t cands_n = 0;
    ReqDev *reqs = nullptr;   // request table of the current search launches
    size_t reqs_n = 0;
    RotRec *phase = nullptr;  // rotations of several requests gathered for one pipeline pass
    size_t phase_n = 0;
    // refinement buffers
    RefBufs ref;
    // twiddle tables per canvas size
    std::map<int, float2 *> tw, qt;
    std::map<int, double2 *> twd;
    // profiling
    bool prof = false;
    std::vector<ProfEntry> pending;
    std::map<std::string, KStat> stats;
    std::vector<cudaEvent_t> ev_pool;
    // registration engine (created by the first registration or submission)
    std::map<int, dock_tuning> tune;   // per lattice side (autotuner or cache)
    Engine *eng = nullptr;
    std::atomic<bool> eng_ready{false};
    std::recursive_mutex dev_mu;   // serialises device work of API calls and the serving thread
    std::atomic<int> dev_want{0};  // API calls waiting for dev_mu
};

// Lock of ctx->dev_mu for an API call.  The waiter is announced so that the
// serving thread steps aside between passes instead of re-taking the lock
// at once (a plain mutex would let it starve the caller).
struct DevLock {
    dock_ctx *c;
    explicit DevLock(dock_ctx *ctx) : c(ctx)
    {
        c->dev_want.fetch_add(1);
        c->dev_mu.lock();
        c->dev_want.fetch_sub(1);
    }
    ~DevLock() { c->dev_mu.unlock(); }
    DevLock(const DevLock &) = delete;
    DevLock &operator=(const DevLock &) = delete;
};

struct dock_object {
    dock_ctx *ctx;
    int N, M, P;
    double h;
    double o[3];
    double anchor[3];
    float *O = nullptr;       // N^3
    float2 *spec = nullptr;   // tiled conj(F(O)) / M^3
    float2 *spec_pen = nullptr;   // tiled conj(F(min(O, 0))) / M^3, made by the first label-aware use
    float4 *cells = nullptr;      // corner cells of O for the rotated-object search, made on first use
    double *o_dev = nullptr;
    // mesh for the refinement
    int64_t nv = 0, nt = 0;
    float *Vf = nullptr;
    int32_t *T = nullptr;
    float *tri_sphere = nullptr;
    int32_t *tri_order = nullptr;
    BvhNode *nodes = nullptr;
    int n_nodes = 0;
    size_t bytes = 0;
};

struct dock_sweep {
    dock_ctx *ctx;
    int64_t P;
    int N;
    double h, r, L;
    double cs[3];
    double *cs_dev = nullptr;
    PoseRec *poses = nullptr;
    uint8_t *labels = nullptr;
    std::vector<double> host_poses;
    size_t bytes = 0;
    // label-aware score: the poses again, contact ones first (P_c of them),
    // each group in trajectory order; nullptr when every pose is contact
    PoseRec *poses_lab = nullptr;
    int64_t P_c = 0;
    // scoring mode bits, read and changed as one word so that the two
    // exclusive options can never both be on: SCORE_LABEL_AWARE, SCORE_ROTATE_OBJECT
    std::atomic<int> mode{0};
    // rotating the object (Sec. IV-D as printed): S on the world-aligned
    // lattice of the mean tip, its spectrum F(S) / M^3 and origin o_s, made
    // on first use
    float2 *spec_S = nullptr;
    double *os_dev = nullptr;
};

static dock_status fail(dock_ctx *ctx, dock_status st, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        std::lock_guard<std::mutex> lk(ctx->err_mu);
        ctx->err = buf;
    }
    return st;
}

static dock_status cuda_fail(dock_ctx *ctx, cudaError_t e, const char *what)
{
    // errors that poison the context are sticky
    bool sticky = (e == cudaErrorIllegalAddress || e == cudaErrorLaunchFailure || e == cudaErrorIllegalInstruction ||
                   e == cudaErrorMisalignedAddress || e == cudaErrorHardwareStackError ||
                   e == cudaErrorInvalidAddressSpace || e == cudaErrorInvalidPc || e == cudaErrorAssert ||
                   e == cudaErrorLaunchTimeout);
    if (sticky && ctx) ctx->dead = true;
    return fail(ctx, sticky ? DOCK_E_CUDA_FATAL : DOCK_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(ctx, call)                                                  \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);     \
    } while (0)

static dock_status dalloc(dock_ctx *ctx, void **p, size_t bytes, size_t *acct)
{
    if (ctx->budget && ctx->held + bytes > ctx->budget)
        return fail(ctx, DOCK_E_TOO_LARGE, "device allocation of %zu bytes exceeds the HBM budget (%zu held of %zu)",
                    bytes, ctx->held, ctx->budget);
    // injected failure (dock_fail_allocation): taken as an out-of-memory answer
    // of cudaMalloc, before any device memory is touched
    int n = ctx->fail_alloc.load();
    while (n > 0 && !ctx->fail_alloc.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 1) return fail(ctx, DOCK_E_NOMEM, "cudaMalloc(%zu): injected allocation failure", bytes);
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, DOCK_E_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    ctx->held += bytes;
    if (ctx->held > ctx->peak_held) ctx->peak_held = ctx->held;
    if (acct) *acct += bytes;
    return DOCK_OK;
}

static void dfree(dock_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    cudaFree(p);
    if (ctx) ctx->held = ctx->held >= bytes ? ctx->held - bytes : 0;
}

// ---------------------------------------------------------------------------
// profiling: CUDA events around every kernel launch on the context stream
// ---------------------------------------------------------------------------
struct Prof {
    dock_ctx *ctx;
    const char *name;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    Prof(dock_ctx *c, const char *n, cudaStream_t s = nullptr) : ctx(c), name(n), st(s ? s : c->stream)
    {
        if (!ctx->prof) return;
        a = get();
        b = get();
        cudaEventRecord(a, st);
    }
    cudaEvent_t get()
    {
        if (!ctx->ev_pool.empty()) {
            cudaEvent_t e = ctx->ev_pool.back();
            ctx->ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    ~Prof()
    {
        if (!ctx->prof) return;
        cudaEventRecord(b, st);
        ctx->pending.push_back({name, a, b});
    }
};

static void prof_resolve(dock_ctx *ctx)
{
    if (ctx->pending.empty()) return;
    for (auto &p : ctx->pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);   // recorded on the context's or the engine's refinement stream
        cudaEventElapsedTime(&ms, p.a, p.b);
        KStat &s = ctx->stats[p.name];
        s.launches += 1;
        s.ms += ms;
        ctx->ev_pool.push_back(p.a);
        ctx->ev_pool.push_back(p.b);
    }
    ctx->pending.clear();
}

// ---------------------------------------------------------------------------
// small host math (FP64, same expressions as the definitions)
// ---------------------------------------------------------------------------
static void quat_to_mat(const double *q, double *R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

static void quat_mul(const double *a, const double *b, double *o)
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

static double lattice_origin(double c, double h, int N) { return h * round(c / h) - (double)(N / 2) * h; }

// ---------------------------------------------------------------------------
// orientation samplers (Sec. IV-C)
// ---------------------------------------------------------------------------
static const double kPhi = 1.4142135623730951;              // sqrt(2)
static const double kPsi = 1.533751168755204288118041;      // psi^4 = psi + 4

// Super-Fibonacci spiral (Alexa 2022): s = i + 1/2, t = s/n, r = sqrt t,
// R = sqrt(1 - t), alpha = 2 pi s / phi, beta = 2 pi s / psi.
static void sampler_sf(int n, double *q)
{
    for (int i = 0; i < n; ++i) {
        double s = i + 0.5, t = s / n, r = sqrt(t), R = sqrt(1.0 - t);
        double al = 2.0 * M_PI * s / kPhi, be = 2.0 * M_PI * s / kPsi;
        q[4 * i + 0] = r * sin(al);
        q[4 * i + 1] = r * cos(al);
        q[4 * i + 2] = R * sin(be);
        q[4 * i + 3] = R * cos(be);
    }
}

static double radical_inverse(long long i, int base)
{
    double f = 1.0, x = 0.0;
    while (i > 0) {
        f /= base;
        x += f * (double)(i % base);
        i /= base;
    }
    return x;
}

// Hopf coordinates (Yershova et al. 2010) of a Halton (2,3,5) sequence.
static void sampler_hopf(int n, double *q)
{
    for (int i = 0; i < n; ++i) {
        double u1 = radical_inverse(i + 1, 2), u2 = radical_inverse(i + 1, 3), u3 = radical_inverse(i + 1, 5);
        double th = acos(1.0 - 2.0 * u1), ph = 2.0 * M_PI * u2, ps = 2.0 * M_PI * u3;
        q[4 * i + 0] = cos(th / 2) * cos(ps / 2);
        q[4 * i + 1] = cos(th / 2) * sin(ps / 2);
        q[4 * i + 2] = sin(th / 2) * cos(ph + ps / 2);
        q[4 * i + 3] = sin(th / 2) * sin(ph + ps / 2);
    }
}

// GeoBall-SF (Algorithm 1): radial law by the tabulated inverse of the CDF
// of rho(r) ~ r L(r), L(r) = 2 acos(cos theta / sqrt(1 - r^2)) (Eq. (11)-(12)),
// r in [0, sin theta], 4097 nodes, trapezoid rule, linear interpolation.
static void sampler_geoball(int n, const double *q0, double theta, double gamma, double *q)
{
    const int nodes = 4097;
    std::vector<double> rt(nodes), F(nodes);
    double rmax = sin(theta);
    for (int k = 0; k < nodes; ++k) rt[k] = rmax * (double)k / (double)(nodes - 1);
    std::vector<double> rho(nodes);
    for (int k = 0; k < nodes; ++k) {
        double arg = cos(theta) / sqrt(1.0 - rt[k] * rt[k]);
        if (arg > 1.0) arg = 1.0;
        rho[k] = rt[k] * 2.0 * acos(arg);
    }
    F[0] = 0.0;
    for (int k = 1; k < nodes; ++k) F[k] = F[k - 1] + 0.5 * (rho[k] + rho[k - 1]) * (rt[k] - rt[k - 1]);
    double tot = F[nodes - 1];
    for (int k = 0; k < nodes; ++k) F[k] /= tot;
    double g = gamma > 0 ? gamma : (double)n;
    for (int i = 0; i < n; ++i) {
        double s = i + 0.5;
        double u1 = fmod(s / g, 1.0), u2 = fmod(s / kPhi, 1.0), u3 = fmod(s / kPsi, 1.0);
        // inverse CDF by linear interpolation on the table
        int k = (int)(std::upper_bound(F.begin(), F.end(), u1) - F.begin());
        double r;
        if (k <= 0) r = rt[0];
        else if (k >= nodes) r = rt[nodes - 1];
        else {
            double w = (F[k] == F[k - 1]) ? 0.0 : (u1 - F[k - 1]) / (F[k] - F[k - 1]);
            r = rt[k - 1] + w * (rt[k] - rt[k - 1]);
        }
        double R = sqrt(1.0 - r * r);
        double arg = cos(theta) / R;
        if (arg > 1.0) arg = 1.0;
        double L = 2.0 * acos(arg);
        double al = (u2 - 0.5) * L, be = 2.0 * M_PI * u3;
        double ql[4] = {R * cos(al), R * sin(al), r * cos(be), r * sin(be)};
        quat_mul(q0, ql, q + 4 * i);
    }
}

static dock_status gen_samples(dock_ctx *ctx, const dock_search_desc *d, std::vector<double> &q)
{
    if (d->n <= 0) return fail(ctx, DOCK_E_INVALID, "sample count must be positive");
    q.resize((size_t)d->n * 4);
    switch (d->sampler) {
    case DOCK_SAMPLER_SF: sampler_sf(d->n, q.data()); break;
    case DOCK_SAMPLER_HOPF: sampler_hopf(d->n, q.data()); break;
    case DOCK_SAMPLER_GEOBALL: {
        if (!(d->theta > 0.0 && d->theta < M_PI / 2)) return fail(ctx, DOCK_E_INVALID, "theta out of range");
        double nq = sqrt(d->q0[0] * d->q0[0] + d->q0[1] * d->q0[1] + d->q0[2] * d->q0[2] + d->q0[3] * d->q0[3]);
        if (!(fabs(nq - 1.0) <= 1e-6)) return fail(ctx, DOCK_E_INVALID, "q0 is not a unit quaternion");
        sampler_geoball(d->n, d->q0, d->theta, d->gamma, q.data());
        break;
    }
    case DOCK_SAMPLER_EXPLICIT:
        if (!d->quats) return fail(ctx, DOCK_E_INVALID, "explicit sampler without quaternions");
        for (int i = 0; i < d->n; ++i) {
            const double *a = d->quats + 4 * i;
            double nq = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
            if (!(fabs(nq - 1.0) <= 1e-6)) return fail(ctx, DOCK_E_INVALID, "quaternion %d is not unit", i);
        }
        memcpy(q.data(), d->quats, sizeof(double) * 4 * d->n);
        break;
    default: return fail(ctx, DOCK_E_INVALID, "unknown sampler %d", d->sampler);
    }
    return DOCK_OK;
}

static void engine_shutdown(dock_ctx *ctx);
static void engine_drop_handle(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw);

// ---------------------------------------------------------------------------
// context API
// ---------------------------------------------------------------------------
extern "C" {

const char *dock_version(void) { return "dock-gb300 0.1 (sm_103a)"; }

void dock_params_default(dock_params *p)
{
    p->tau_out1 = 0.5;
    p->tau_in1 = 0.2;
    p->deep_value = -50.0;
    p->tau_out2 = 0.2;
    p->tau_in2 = 0.03;
    p->k_slope = 15.0;
    p->lambda = 1e-3;
    p->mu = 1e-6;
    p->b_t = 1.0;
    p->b_r = 5.0 * M_PI / 180.0;
    p->step_t = 0.05;
    p->step_r = 0.5 * M_PI / 180.0;
    p->iters = 20;
    p->tri_iters = 20;
    p->solver = DOCK_SOLVER_GAUSS_NEWTON;
    p->lbfgs_evals = 100;
    p->lbfgs_pgtol = 1e-5;
    p->lbfgs_ftol = 2.220446049250313e-09;
}

dock_status dock_create(dock_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream)
{
    if (!out) return DOCK_E_INVALID;
    *out = nullptr;
    dock_ctx *c = new (std::nothrow) dock_ctx();
    if (!c) return DOCK_E_NOMEM;
    c->device = device;
    c->budget = hbm_budget_bytes;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete c;
        return DOCK_E_CUDA;
    }
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return DOCK_E_CUDA;
        }
        c->own_stream = true;
    }
    e = cudaMalloc(&c->errflag, sizeof(int));
    if (e != cudaSuccess) {
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return DOCK_E_NOMEM;
    }
    cudaMemset(c->errflag, 0, sizeof(int));
    // the allocation-free search's scratch is placed on this device now (its
    // module is loaded by the address lookup), not inside that call
    e = noalloc_prepare(device);
    if (e != cudaSuccess) {
        cudaFree(c->errflag);
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return DOCK_E_CUDA;
    }
    *out = c;
    return DOCK_OK;
}

void dock_destroy(dock_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    engine_shutdown(c);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->Y);
    cudaFree(c->bits);
    cudaFree(c->ogr);
    cudaFree(c->keys);
    cudaFree(c->rots);
    cudaFree(c->quats);
    cudaFree(c->errflag);
    cudaFree(c->cands);
    cudaFree(c->reqs);
    cudaFree(c->phase);
    for (auto e : c->vev)
        if (e) cudaEventDestroy(e);
    if (c->vstream) cudaStreamDestroy(c->vstream);
    free_refbufs(c->ref);
    for (auto &kv : c->tw) cudaFree(kv.second);
    for (auto &kv : c->qt) cudaFree(kv.second);
    for (auto &kv : c->twd) cudaFree(kv.second);
    for (auto &p : c->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *dock_last_error(const dock_ctx *c)
{
    // a per-thread copy: the serving thread may record errors meanwhile
    static thread_local std::string copy;
    if (!c) return "null context";
    std::lock_guard<std::mutex> lk(const_cast<dock_ctx *>(c)->err_mu);
    copy = c->err;
    return copy.c_str();
}

dock_status dock_set_profiling(dock_ctx *c, int enable)
{
    if (!c) return DOCK_E_INVALID;
    DevLock dev_lock_(c);
    if (!enable) prof_resolve(c);
    c->prof = enable != 0;
    return DOCK_OK;
}

int32_t dock_get_kernel_stats(dock_ctx *c, dock_kernel_stat *st, int32_t cap)
{
    if (!c) return 0;
    DevLock dev_lock_(c);
    prof_resolve(c);
    int32_t n = 0;
    for (auto &kv : c->stats) {
        if (n >= cap) break;
        memset(&st[n], 0, sizeof(st[n]));
        strncpy(st[n].name, kv.first.c_str(), sizeof(st[n].name) - 1);
        st[n].launches = kv.second.launches;
        st[n].total_ms = kv.second.ms;
        ++n;
    }
    return n;
}

void dock_reset_kernel_stats(dock_ctx *c)
{
    if (!c) return;
    DevLock dev_lock_(c);
    prof_resolve(c);
    c->stats.clear();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------
static dock_status tables(dock_ctx *ctx, int M, float2 **tw, float2 **qt, double2 **twd)
{
    if (!ctx->tw.count(M)) {
        std::vector<float2> t(M), q(M / 2);
        std::vector<double2> td(M);
        for (int m = 0; m < M; ++m) {
            double a = 2.0 * M_PI * (double)m / (double)M;
            double c = cos(a), s = -sin(a);
            td[m] = make_double2(c, s);
            t[m] = make_float2((float)c, (float)s);
        }
        for (int k = 0; k < M / 2; ++k) {
            // 1 / (1 - w^k), w = exp(-2 pi i / M); unused for k = 0
            if (k == 0) { q[k] = make_float2(0.f, 0.f); continue; }
            double re = 1.0 - td[k].x, im = -td[k].y;
            double den = re * re + im * im;
            q[k] = make_float2((float)(re / den), (float)(-im / den));
        }
        float2 *dt = nullptr, *dq = nullptr;
        double2 *dd = nullptr;
        // a failure part way releases what this call allocated
        auto release = [&] {
            dfree(ctx, dt, sizeof(float2) * M);
            dfree(ctx, dq, sizeof(float2) * (M / 2));
            dfree(ctx, dd, sizeof(double2) * M);
        };
        dock_status s = dalloc(ctx, (void **)&dt, sizeof(float2) * M, nullptr);
        if (s == DOCK_OK) s = dalloc(ctx, (void **)&dq, sizeof(float2) * (M / 2), nullptr);
        if (s == DOCK_OK) s = dalloc(ctx, (void **)&dd, sizeof(double2) * M, nullptr);
        if (s != DOCK_OK) {
            release();
            return s;
        }
        cudaError_t e = cudaMemcpy(dt, t.data(), sizeof(float2) * M, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dq, q.data(), sizeof(float2) * (M / 2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dd, td.data(), sizeof(double2) * M, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            release();
            return cuda_fail(ctx, e, "uploading the twiddle tables");
        }
        ctx->tw[M] = dt;
        ctx->qt[M] = dq;
        ctx->twd[M] = dd;
    }
    *tw = ctx->tw[M];
    *qt = ctx->qt[M];
    *twd = ctx->twd[M];
    return DOCK_OK;
}

static bool valid_N(int N) { return N == 32 || N == 64 || N == 96 || N == 128; }

// ---------------------------------------------------------------------------
// object
// ---------------------------------------------------------------------------
static void build_bins3(const double *V, const int32_t *T, int64_t nt, const double *o, double cs, const int *d,
                        double pad, std::vector<int32_t> &start, std::vector<int32_t> &items)
{
    int64_t nc = (int64_t)d[0] * d[1] * d[2];
    std::vector<int32_t> cnt(nc + 1, 0);
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            start.assign(nc + 1, 0);
            for (int64_t c = 0; c < nc; ++c) start[c + 1] = start[c] + cnt[c];
            items.assign(start[nc] > 0 ? start[nc] : 1, 0);
            std::fill(cnt.begin(), cnt.end(), 0);
        }
        for (int64_t t = 0; t < nt; ++t) {
            int lo[3], hi[3];
            bool ok = true;
            for (int a = 0; a < 3; ++a) {
                double x0 = V[3 * T[3 * t] + a], x1 = V[3 * T[3 * t + 1] + a], x2 = V[3 * T[3 * t + 2] + a];
                double mn = std::min(x0, std::min(x1, x2)) - pad, mx = std::max(x0, std::max(x1, x2)) + pad;
                lo[a] = std::max(0, (int)floor((mn - o[a]) / cs));
                hi[a] = std::min(d[a] - 1, (int)floor((mx - o[a]) / cs));
                if (lo[a] > hi[a]) ok = false;
            }
            if (!ok) continue;
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x) {
                        int64_t c = ((int64_t)z * d[1] + y) * d[0] + x;
                        if (pass == 0) cnt[c]++;
                        else items[start[c] + cnt[c]++] = (int32_t)t;
                    }
        }
    }
}

static void build_bins2(const double *V, const int32_t *T, int64_t nt, const double *o, double cs, const int *d,
                        std::vector<int32_t> &start, std::vector<int32_t> &items)
{
    int64_t nc = (int64_t)d[0] * d[1];
    std::vector<int32_t> cnt(nc + 1, 0);
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            start.assign(nc + 1, 0);
            for (int64_t c = 0; c < nc; ++c) start[c + 1] = start[c] + cnt[c];
            items.assign(start[nc] > 0 ? start[nc] : 1, 0);
            std::fill(cnt.begin(), cnt.end(), 0);
        }
        for (int64_t t = 0; t < nt; ++t) {
            int lo[2], hi[2];
            bool ok = true;
            for (int k = 0; k < 2; ++k) {
                int a = k + 1;
                double x0 = V[3 * T[3 * t] + a], x1 = V[3 * T[3 * t + 1] + a], x2 = V[3 * T[3 * t + 2] + a];
                double mn = std::min(x0, std::min(x1, x2)), mx = std::max(x0, std::max(x1, x2));
                lo[k] = std::max(0, (int)floor((mn - o[a]) / cs));
                hi[k] = std::min(d[k] - 1, (int)floor((mx - o[a]) / cs));
                if (lo[k] > hi[k]) ok = false;
            }
            if (!ok) continue;
            for (int z = lo[1]; z <= hi[1]; ++z)
                for (int y = lo[0]; y <= hi[0]; ++y) {
                    int64_t c = (int64_t)z * d[0] + y;
                    if (pass == 0) cnt[c]++;
                    else items[start[c] + cnt[c]++] = (int32_t)t;
                }
        }
    }
}

// BVH over triangles (object frame): median split on the longest centroid
// axis, leaves of <= 4 triangles; node spheres enclose their triangles.
static void build_bvh(const double *V, const int32_t *T, int64_t nt, std::vector<BvhNode> &nodes,
                      std::vector<int32_t> &order, std::vector<float> &tri_sphere)
{
    order.resize(nt);
    std::vector<double> cen(nt * 3);
    tri_sphere.resize(nt * 4);
    for (int64_t t = 0; t < nt; ++t) {
        order[t] = (int32_t)t;
        double lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            double x0 = V[3 * T[3 * t] + a], x1 = V[3 * T[3 * t + 1] + a], x2 = V[3 * T[3 * t + 2] + a];
            lo[a] = std::min(x0, std::min(x1, x2));
            hi[a] = std::max(x0, std::max(x1, x2));
            cen[3 * t + a] = 0.5 * (lo[a] + hi[a]);
        }
        double rad = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double *v = V + 3 * T[3 * t + k];
            double dx = v[0] - cen[3 * t], dy = v[1] - cen[3 * t + 1], dz = v[2] - cen[3 * t + 2];
            rad = std::max(rad, sqrt(dx * dx + dy * dy + dz * dz));
        }
        for (int a = 0; a < 3; ++a) tri_sphere[4 * t + a] = (float)cen[3 * t + a];
        tri_sphere[4 * t + 3] = (float)(rad * (1.0 + 1e-6) + 1e-6);
    }
    nodes.clear();
    nodes.reserve(2 * nt / 2 + 8);
    struct Item { int node, lo, hi; };
    std::vector<Item> stack;
    nodes.push_back(BvhNode());
    stack.push_back({0, 0, (int)nt});
    while (!stack.empty()) {
        Item it = stack.back();
        stack.pop_back();
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int i = it.lo; i < it.hi; ++i) {
            int t = order[i];
            for (int k = 0; k < 3; ++k) {
                const double *v = V + 3 * T[3 * t + k];
                for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], v[a]); hi[a] = std::max(hi[a], v[a]); }
            }
        }
        double c[3] = {0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2])};
        double rad = 0.0;
        for (int i = it.lo; i < it.hi; ++i) {
            int t = order[i];
            for (int k = 0; k < 3; ++k) {
                const double *v = V + 3 * T[3 * t + k];
                double dx = v[0] - c[0], dy = v[1] - c[1], dz = v[2] - c[2];
                rad = std::max(rad, sqrt(dx * dx + dy * dy + dz * dz));
            }
        }
        BvhNode &nd = nodes[it.node];
        for (int a = 0; a < 3; ++a) nd.c[a] = (float)c[a];
        nd.rad = (float)(rad * (1.0 + 1e-6) + 1e-6);
        nd.pad = 0;
        int n = it.hi - it.lo;
        if (n <= 4) {
            nd.left = -1;
            nd.right = it.lo;
            nd.count = n;
            continue;
        }
        int ax = 0;
        double ext = -1;
        double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
        for (int i = it.lo; i < it.hi; ++i)
            for (int a = 0; a < 3; ++a) {
                clo[a] = std::min(clo[a], cen[3 * order[i] + a]);
                chi[a] = std::max(chi[a], cen[3 * order[i] + a]);
            }
        for (int a = 0; a < 3; ++a) if (chi[a] - clo[a] > ext) { ext = chi[a] - clo[a]; ax = a; }
        int mid = (it.lo + it.hi) / 2;
        std::nth_element(order.begin() + it.lo, order.begin() + mid, order.begin() + it.hi,
                         [&](int a, int b) { return cen[3 * a + ax] < cen[3 * b + ax] ||
                                                   (cen[3 * a + ax] == cen[3 * b + ax] && a < b); });
        int l = (int)nodes.size();
        nodes.push_back(BvhNode());
        int r = (int)nodes.size();
        nodes.push_back(BvhNode());
        nodes[it.node].left = l;
        nodes[it.node].right = r;
        nodes[it.node].count = 0;
        stack.push_back({r, mid, it.hi});
        stack.push_back({l, it.lo, mid});
    }
}

extern "C" dock_status dock_object_grid(dock_ctx *ctx, const double *verts, int64_t V, const int32_t *tris, int64_t T,
                                        const uint8_t *touchable, double h, int32_t N, const dock_params *params,
                                        dock_object **out)
{
    if (!ctx || !out) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    *out = nullptr;
    if (!verts || !tris || V < 3 || T < 1) return fail(ctx, DOCK_E_INVALID, "empty mesh");
    if (!valid_N(N)) return fail(ctx, DOCK_E_INVALID, "N must be one of 32, 64, 96, 128 (got %d)", N);
    if (!(h > 0.0) || !isfinite(h)) return fail(ctx, DOCK_E_INVALID, "voxel size must be positive");
    dock_params pd;
    dock_params_default(&pd);
    const dock_params *p = params ? params : &pd;
    for (int64_t i = 0; i < 3 * V; ++i)
        if (!isfinite(verts[i])) return fail(ctx, DOCK_E_INVALID, "vertex coordinate %lld is not finite", (long long)i);
    for (int64_t i = 0; i < 3 * T; ++i)
        if (tris[i] < 0 || tris[i] >= V) return fail(ctx, DOCK_E_INVALID, "triangle index out of range");
    cudaSetDevice(ctx->device);
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = 0; i < V; ++i)
        for (int a = 0; a < 3; ++a) { mn[a] = std::min(mn[a], verts[3 * i + a]); mx[a] = std::max(mx[a], verts[3 * i + a]); }
    dock_object *ob = new (std::nothrow) dock_object();
    if (!ob) return fail(ctx, DOCK_E_NOMEM, "host allocation");
    ob->ctx = ctx;
    ob->N = N;
    ob->M = 2 * N;
    ob->P = N + 2;
    ob->h = h;
    for (int a = 0; a < 3; ++a) {
        double c = (mn[a] + mx[a]) * 0.5;
        ob->o[a] = lattice_origin(c, h, N);
        ob->anchor[a] = c;
        if (mn[a] - p->tau_out1 < ob->o[a] || mx[a] + p->tau_out1 > ob->o[a] + (double)(N - 1) * h) {
            delete ob;
            return fail(ctx, DOCK_E_INVALID, "mesh (widened by tau_out1) does not fit the %d^3 lattice at h = %g", N, h);
        }
    }
    dock_status s;
    const int M = ob->M, P = ob->P;
    float2 *tw, *qt;
    double2 *twd;
    if ((s = tables(ctx, M, &tw, &qt, &twd)) != DOCK_OK) { delete ob; return s; }
    // bins
    double cut = std::max(p->tau_out1, p->tau_in1);
    double cs = std::max(cut, h);
    int d3[3], d2[2];
    for (int a = 0; a < 3; ++a) d3[a] = (int)ceil(((double)(N - 1) * h) / cs) + 1;
    d2[0] = d3[1];
    d2[1] = d3[2];
    std::vector<int32_t> s3, i3, s2, i2;
    build_bins3(verts, tris, T, ob->o, cs, d3, cut, s3, i3);
    build_bins2(verts, tris, T, ob->o, cs, d2, s2, i2);
    // device buffers
    double *dV = nullptr, *dcen = nullptr;
    int32_t *dT = nullptr, *ds3 = nullptr, *di3 = nullptr, *ds2 = nullptr, *di2 = nullptr;
    uint8_t *dtouch = nullptr;
    double2 *w1 = nullptr, *w2 = nullptr;
    size_t tmp_bytes = 0;
    auto cleanup_tmp = [&]() {
        dfree(ctx, dV, sizeof(double) * 3 * V);
        dfree(ctx, ds3, sizeof(int32_t) * s3.size());
        dfree(ctx, di3, sizeof(int32_t) * i3.size());
        dfree(ctx, ds2, sizeof(int32_t) * s2.size());
        dfree(ctx, di2, sizeof(int32_t) * i2.size());
        dfree(ctx, dtouch, (size_t)T);
        dfree(ctx, w1, sizeof(double2) * (size_t)N * N * (N + 1));
        dfree(ctx, w2, sizeof(double2) * (size_t)N * M * (N + 1));
        (void)dcen;
    };
    auto bail = [&](dock_status st) {
        cleanup_tmp();
        dock_object_free(ob);
        return st;
    };
    if ((s = dalloc(ctx, (void **)&dV, sizeof(double) * 3 * V, &tmp_bytes)) != DOCK_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&dT, sizeof(int32_t) * 3 * T, &ob->bytes)) != DOCK_OK) return bail(s);
    ob->T = dT;
    if ((s = dalloc(ctx, (void **)&ds3, sizeof(int32_t) * s3.size(), &tmp_bytes)) != DOCK_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&di3, sizeof(int32_t) * i3.size(), &tmp_bytes)) != DOCK_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&ds2, sizeof(int32_t) * s2.size(), &tmp_bytes)) != DOCK_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&di2, sizeof(int32_t) * i2.size(), &tmp_bytes)) != DOCK_OK) return bail(s);
    if (touchable && (s = dalloc(ctx, (void **)&dtouch, (size_t)T, &tmp_bytes)) != DOCK_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&ob->O, sizeof(float) * (size_t)N * N * N, &ob->bytes)) != DOCK_OK) return bail(s);
    size_t spec_n = (size_t)M * P / 32 * M * 32;
    if ((s = dalloc(ctx, (void **)&ob->spec, sizeof(float2) * spec_n, &ob->bytes)) != DOCK_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&ob->o_dev, sizeof(double) * 3, &ob->bytes)) != DOCK_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&w1, sizeof(double2) * (size_t)N * N * (N + 1), &tmp_bytes)) != DOCK_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&w2, sizeof(double2) * (size_t)N * M * (N + 1), &tmp_bytes)) != DOCK_OK) return bail(s);
    cudaStream_t st = ctx->stream;
#define CKB(call)                                                   \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return bail(cuda_fail(ctx, e_, #call)); \
    } while (0)
    CKB(cudaMemcpyAsync(dV, verts, sizeof(double) * 3 * V, cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(dT, tris, sizeof(int32_t) * 3 * T, cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(ds3, s3.data(), sizeof(int32_t) * s3.size(), cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(di3, i3.data(), sizeof(int32_t) * i3.size(), cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(ds2, s2.data(), sizeof(int32_t) * s2.size(), cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(di2, i2.data(), sizeof(int32_t) * i2.size(), cudaMemcpyHostToDevice, st));
    if (dtouch) CKB(cudaMemcpyAsync(dtouch, touchable, (size_t)T, cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(ob->o_dev, ob->o, sizeof(double) * 3, cudaMemcpyHostToDevice, st));
    CKB(cudaMemsetAsync(ctx->errflag, 0, sizeof(int), st));
    ObjBins bins;
    bins.cell3_start = ds3;
    bins.cell3_items = di3;
    bins.cell2_start = ds2;
    bins.cell2_items = di2;
    for (int a = 0; a < 3; ++a) bins.d3[a] = d3[a];
    bins.d2[0] = d2[0];
    bins.d2[1] = d2[1];
    bins.cs = cs;
    {
        Prof pr(ctx, "object_grid");
        CKB(launch_object_grid(dV, dT, dtouch, bins, N, h, ob->o, p->tau_out1, p->tau_in1, p->deep_value, ob->O,
                               nullptr, ctx->errflag, st));
    }
    {
        Prof pr(ctx, "object_spectrum");
        CKB(launch_spectrum(ob->O, N, M, P, w1, w2, twd, ob->spec, st));
    }
    // mesh + BVH for the refinement
    std::vector<BvhNode> nodes;
    std::vector<int32_t> order;
    std::vector<float> tsph;
    build_bvh(verts, tris, T, nodes, order, tsph);
    std::vector<float> vf(3 * V);
    for (int64_t i = 0; i < 3 * V; ++i) vf[i] = (float)verts[i];
    ob->nv = V;
    ob->nt = T;
    ob->n_nodes = (int)nodes.size();
    if ((s = dalloc(ctx, (void **)&ob->Vf, sizeof(float) * 3 * V, &ob->bytes)) != DOCK_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&ob->tri_sphere, sizeof(float) * 4 * T, &ob->bytes)) != DOCK_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&ob->tri_order, sizeof(int32_t) * T, &ob->bytes)) != DOCK_OK) return bail(s);
    if ((s = dalloc(ctx, (void **)&ob->nodes, sizeof(BvhNode) * nodes.size(), &ob->bytes)) != DOCK_OK) return bail(s);
    CKB(cudaMemcpyAsync(ob->Vf, vf.data(), sizeof(float) * 3 * V, cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(ob->tri_sphere, tsph.data(), sizeof(float) * 4 * T, cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(ob->tri_order, order.data(), sizeof(int32_t) * T, cudaMemcpyHostToDevice, st));
    CKB(cudaMemcpyAsync(ob->nodes, nodes.data(), sizeof(BvhNode) * nodes.size(), cudaMemcpyHostToDevice, st));
    int herr = 0;
    CKB(cudaMemcpyAsync(&herr, ctx->errflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKB(cudaStreamSynchronize(st));
#undef CKB
    cleanup_tmp();
    if (herr) {
        dock_object_free(ob);
        return fail(ctx, DOCK_E_OVERFLOW, "a lattice row crosses the mesh more than 1024 times");
    }
    *out = ob;
    return DOCK_OK;
}

extern "C" void dock_object_free(dock_object *ob)
{
    if (!ob) return;
    DevLock dev_lock_(ob->ctx);
    dock_ctx *ctx = ob->ctx;
    cudaSetDevice(ctx->device);
    engine_drop_handle(ctx, ob, nullptr);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ob->O);
    cudaFree(ob->spec);
    cudaFree(ob->spec_pen);
    cudaFree(ob->cells);
    cudaFree(ob->o_dev);
    cudaFree(ob->Vf);
    cudaFree(ob->T);
    cudaFree(ob->tri_sphere);
    cudaFree(ob->tri_order);
    cudaFree(ob->nodes);
    ctx->held = ctx->held >= ob->bytes ? ctx->held - ob->bytes : 0;
    delete ob;
}

extern "C" dock_status dock_object_export_grid(dock_ctx *ctx, const dock_object *ob, float *grid, double *origin)
{
    if (!ctx || !ob) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (grid) CK(ctx, cudaMemcpy(grid, ob->O, sizeof(float) * (size_t)ob->N * ob->N * ob->N, cudaMemcpyDeviceToHost));
    if (origin) memcpy(origin, ob->o, sizeof(double) * 3);
    return DOCK_OK;
}

// ---------------------------------------------------------------------------
// sweep
// ---------------------------------------------------------------------------
extern "C" dock_status dock_sweep_grid(dock_ctx *ctx, const dock_probe *probe, const double *poses,
                                       const uint8_t *contact, int64_t P, double h, int32_t N, dock_sweep **out)
{
    if (!ctx || !out || !probe) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    *out = nullptr;
    if (!poses || P <= 0) return fail(ctx, DOCK_E_INVALID, "empty trajectory");
    if (P > (1 << 24)) return fail(ctx, DOCK_E_INVALID, "trajectory too long");
    if (!valid_N(N)) return fail(ctx, DOCK_E_INVALID, "N must be one of 32, 64, 96, 128 (got %d)", N);
    if (probe->kind != 0) return fail(ctx, DOCK_E_INVALID, "only the flat-ended cylinder probe is supported");
    if (!(probe->radius > 0) || !(probe->length > 0) || !isfinite(probe->radius) || !isfinite(probe->length))
        return fail(ctx, DOCK_E_INVALID, "probe radius and length must be positive");
    if (!(h > 0.0) || !isfinite(h)) return fail(ctx, DOCK_E_INVALID, "voxel size must be positive");
    std::vector<PoseRec> pr(P);
    double c[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < P; ++i) {
        const double *q = poses + 7 * i;
        for (int k = 0; k < 7; ++k)
            if (!isfinite(q[k])) return fail(ctx, DOCK_E_INVALID, "pose %lld is not finite", (long long)i);
        double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        if (!(fabs(nq - 1.0) <= 1e-6)) return fail(ctx, DOCK_E_INVALID, "pose %lld has a non-unit quaternion", (long long)i);
        quat_to_mat(q, pr[i].R);
        for (int a = 0; a < 3; ++a) pr[i].t[a] = q[4 + a];
        for (int k = 0; k < 9; ++k) pr[i].Rf[k] = (float)pr[i].R[k];
        for (int a = 0; a < 3; ++a) pr[i].tf[a] = (float)pr[i].t[a];
        c[0] += q[4];
        c[1] += q[5];
        c[2] += q[6];
    }
    for (int a = 0; a < 3; ++a) c[a] = c[a] / (double)P;
    cudaSetDevice(ctx->device);
    dock_sweep *sw = new (std::nothrow) dock_sweep();
    if (!sw) return fail(ctx, DOCK_E_NOMEM, "host allocation");
    sw->ctx = ctx;
    sw->P = P;
    sw->N = N;
    sw->h = h;
    sw->r = probe->radius;
    sw->L = probe->length;
    memcpy(sw->cs, c, sizeof(c));
    sw->host_poses.assign(poses, poses + 7 * P);
    dock_status s;
    if ((s = dalloc(ctx, (void **)&sw->poses, sizeof(PoseRec) * P, &sw->bytes)) != DOCK_OK) { delete sw; return s; }
    if ((s = dalloc(ctx, (void **)&sw->cs_dev, sizeof(double) * 3, &sw->bytes)) != DOCK_OK) { dock_sweep_free(sw); return s; }
    if ((s = dalloc(ctx, (void **)&sw->labels, (size_t)P, &sw->bytes)) != DOCK_OK) { dock_sweep_free(sw); return s; }
    cudaError_t e = cudaMemcpyAsync(sw->poses, pr.data(), sizeof(PoseRec) * P, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sw->cs_dev, c, sizeof(double) * 3, cudaMemcpyHostToDevice, ctx->stream);
    std::vector<uint8_t> lab(P, 1);
    if (contact) for (int64_t i = 0; i < P; ++i) lab[i] = contact[i] ? 1 : 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(sw->labels, lab.data(), (size_t)P, cudaMemcpyHostToDevice, ctx->stream);
    std::vector<PoseRec> prl;
    prl.reserve(P);
    for (int64_t i = 0; i < P; ++i)
        if (lab[i]) prl.push_back(pr[i]);
    sw->P_c = (int64_t)prl.size();
    for (int64_t i = 0; i < P; ++i)
        if (!lab[i]) prl.push_back(pr[i]);
    if (e == cudaSuccess && sw->P_c < P) {
        if ((s = dalloc(ctx, (void **)&sw->poses_lab, sizeof(PoseRec) * P, &sw->bytes)) != DOCK_OK) {
            cudaStreamSynchronize(ctx->stream);
            dock_sweep_free(sw);
            return s;
        }
        e = cudaMemcpyAsync(sw->poses_lab, prl.data(), sizeof(PoseRec) * P, cudaMemcpyHostToDevice, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        dock_sweep_free(sw);
        return cuda_fail(ctx, e, "sweep upload");
    }
    *out = sw;
    return DOCK_OK;
}

extern "C" void dock_sweep_free(dock_sweep *sw)
{
    if (!sw) return;
    DevLock dev_lock_(sw->ctx);
    dock_ctx *ctx = sw->ctx;
    cudaSetDevice(ctx->device);
    engine_drop_handle(ctx, nullptr, sw);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(sw->poses);
    cudaFree(sw->cs_dev);
    cudaFree(sw->labels);
    cudaFree(sw->poses_lab);
    cudaFree(sw->spec_S);
    cudaFree(sw->os_dev);
    ctx->held = ctx->held >= sw->bytes ? ctx->held - sw->bytes : 0;
    delete sw;
}

static Geo make_geo(const dock_sweep *sw)
{
    Geo g;
    g.N = sw->N;
    g.M = 2 * sw->N;
    g.P = sw->N + 2;
    g.h = sw->h;
    g.inv_h = (float)(1.0 / sw->h);
    g.rv = (float)(sw->r / sw->h);
    g.lv = (float)(sw->L / sw->h);
    g.r = sw->r;
    g.L = sw->L;
    return g;
}

// grow-only device scratch owned by the context
static dock_status ensure(dock_ctx *ctx, void **p, size_t *have, size_t need, size_t elem)
{
    if (*have >= need) return DOCK_OK;
    if (*p) {
        cudaStreamSynchronize(ctx->stream);
        dfree(ctx, *p, *have * elem);
        *p = nullptr;
        *have = 0;
    }
    dock_status s = dalloc(ctx, p, need * elem, nullptr);
    if (s == DOCK_OK) *have = need;
    return s;
}

// Upload `count` quaternions (host q) to slots [base, base + count) of the
// context's rotation arrays (capacity `cap`) and build their lattice set-up
// records: sample indices rot0.., request index `req`.
// o_o (nullable, device): rotate the object instead of the sweep.
static dock_status upload_rots(dock_ctx *ctx, const dock_sweep *sw, const double *q, size_t cap, size_t base, int count,
                               int rot0, int req, const double *o_o = nullptr)
{
    dock_status s;
    if ((s = ensure(ctx, (void **)&ctx->quats, &ctx->quats_n, cap * 4, sizeof(double))) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->rots, &ctx->rots_n, cap, sizeof(RotRec))) != DOCK_OK) return s;
    if (count <= 0) return DOCK_OK;
    CK(ctx, cudaMemcpyAsync(ctx->quats + 4 * base, q, sizeof(double) * 4 * count, cudaMemcpyHostToDevice, ctx->stream));
    Prof pr(ctx, "rot_setup");
    CK(ctx, launch_rot_setup(ctx->quats + 4 * base, count, rot0, req, sw->cs_dev, sw->h, sw->N, ctx->rots + base,
                             ctx->stream, o_o));
    return DOCK_OK;
}

// la: the label-aware score (contact poses as pose set 0, non-contact poses
// as pose set 1); a sweep whose poses are all contact has no set 1 and
// scores as a plain one.  For a search, ob->spec_pen must exist
// (ensure_spec_pen) before a label-aware table is used.
// ro: rotate the object; spec is then the sweep's F(S) / M^3 (ensure_spec_S
// first) and Og the object grid.
static ReqDev make_reqdev(const dock_object *ob, const dock_sweep *sw, unsigned long long *keys, bool la,
                          bool ro = false)
{
    ReqDev q;
    q.poses = sw->poses;
    q.P = (int)sw->P;
    q.poses_nc = nullptr;
    q.P_nc = 0;
    q.spec_pen = nullptr;
    if (la && sw->poses_lab) {
        q.poses = sw->poses_lab;
        q.P = (int)sw->P_c;
        q.poses_nc = sw->poses_lab + sw->P_c;
        q.P_nc = (int)(sw->P - sw->P_c);
        q.spec_pen = ob ? ob->spec_pen : nullptr;
    }
    q.h = sw->h;
    q.r = sw->r;
    q.L = sw->L;
    q.inv_h = (float)(1.0 / sw->h);
    q.rv = (float)(sw->r / sw->h);
    q.lv = (float)(sw->L / sw->h);
    q.spec = ob ? ob->spec : nullptr;
    q.keys = keys;
    q.Og4 = nullptr;
    q.rotate_object = 0;
    if (ro) {
        q.spec = sw->spec_S;
        q.Og4 = ob ? ob->cells : nullptr;
        q.rotate_object = 1;
    }
    return q;
}

static dock_status upload_reqs(dock_ctx *ctx, const std::vector<ReqDev> &r)
{
    dock_status s;
    if ((s = ensure(ctx, (void **)&ctx->reqs, &ctx->reqs_n, r.size(), sizeof(ReqDev))) != DOCK_OK) return s;
    CK(ctx, cudaMemcpyAsync(ctx->reqs, r.data(), sizeof(ReqDev) * r.size(), cudaMemcpyHostToDevice, ctx->stream));
    return DOCK_OK;
}

extern "C" dock_status dock_sweep_voxelise(dock_ctx *ctx, const dock_sweep *sw, const double *quats, int32_t n,
                                           uint8_t *bits, double *origins)
{
    if (!ctx || !sw || !quats || n <= 0) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    cudaSetDevice(ctx->device);
    dock_search_desc d = {};
    d.sampler = DOCK_SAMPLER_EXPLICIT;
    d.n = n;
    d.quats = quats;
    std::vector<double> q;
    dock_status s;
    if ((s = gen_samples(ctx, &d, q)) != DOCK_OK) return s;
    if ((s = upload_rots(ctx, sw, q.data(), n, 0, n, 0, 0)) != DOCK_OK) return s;
    std::vector<ReqDev> rq(1, make_reqdev(nullptr, sw, nullptr, false));
    if ((s = upload_reqs(ctx, rq)) != DOCK_OK) return s;
    Geo g = make_geo(sw);
    size_t per = (size_t)g.N * g.N * g.N;
    uint8_t *dbits = nullptr;
    if ((s = dalloc(ctx, (void **)&dbits, per * n, nullptr)) != DOCK_OK) return s;
    cudaError_t e;
    {
        Prof pr(ctx, "vox_export");
        e = launch_vox_export(g, ctx->reqs, ctx->rots, n, dbits, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(bits, dbits, per * n, cudaMemcpyDeviceToHost, ctx->stream);
    std::vector<RotRec> rr(n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rr.data(), ctx->rots, sizeof(RotRec) * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, dbits, per * n);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "voxelise");
    if (origins)
        for (int i = 0; i < n; ++i) memcpy(origins + 3 * i, rr[i].o, sizeof(double) * 3);
    return DOCK_OK;
}

enum { SCORE_LABEL_AWARE = 1, SCORE_ROTATE_OBJECT = 2 };

// Sets or clears `bit` of the sweep's mode; setting fails while `other` is set.
static bool set_mode_bit(dock_sweep *sw, int bit, int other, bool on)
{
    int cur = sw->mode.load();
    for (;;) {
        if (on && (cur & other)) return false;
        const int want = on ? (cur | bit) : (cur & ~bit);
        if (sw->mode.compare_exchange_weak(cur, want)) return true;
    }
}

extern "C" dock_status dock_sweep_set_label_aware(dock_ctx *ctx, dock_sweep *sw, int32_t on)
{
    if (!ctx || !sw || sw->ctx != ctx) return DOCK_E_INVALID;
    if (on != 0 && on != 1) return fail(ctx, DOCK_E_INVALID, "label_aware must be 0 or 1");
    if (!set_mode_bit(sw, SCORE_LABEL_AWARE, SCORE_ROTATE_OBJECT, on != 0))
        return fail(ctx, DOCK_E_INVALID, "the label-aware score needs the rotated sweep (rotate_object is on)");
    return DOCK_OK;
}

extern "C" dock_status dock_sweep_set_rotate_object(dock_ctx *ctx, dock_sweep *sw, int32_t on)
{
    if (!ctx || !sw || sw->ctx != ctx) return DOCK_E_INVALID;
    if (on != 0 && on != 1) return fail(ctx, DOCK_E_INVALID, "rotate_object must be 0 or 1");
    if (!set_mode_bit(sw, SCORE_ROTATE_OBJECT, SCORE_LABEL_AWARE, on != 0))
        return fail(ctx, DOCK_E_INVALID, "rotating the object excludes the label-aware score (label_aware is on)");
    return DOCK_OK;
}

extern "C" dock_status dock_sweep_voxelise_labels(dock_ctx *ctx, const dock_sweep *sw, const double *quats, int32_t n,
                                                  uint8_t *bits_c, uint8_t *bits_n, double *origins)
{
    if (!ctx || !sw || !quats || n <= 0 || !bits_c || !bits_n) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    cudaSetDevice(ctx->device);
    dock_search_desc d = {};
    d.sampler = DOCK_SAMPLER_EXPLICIT;
    d.n = n;
    d.quats = quats;
    std::vector<double> q;
    dock_status s;
    if ((s = gen_samples(ctx, &d, q)) != DOCK_OK) return s;
    if ((s = upload_rots(ctx, sw, q.data(), n, 0, n, 0, 0)) != DOCK_OK) return s;
    std::vector<ReqDev> rq(1, make_reqdev(nullptr, sw, nullptr, true));
    if ((s = upload_reqs(ctx, rq)) != DOCK_OK) return s;
    Geo g = make_geo(sw);
    const size_t per = (size_t)g.N * g.N * g.N;
    uint8_t *dbits = nullptr;
    if ((s = dalloc(ctx, (void **)&dbits, 2 * per * n, nullptr)) != DOCK_OK) return s;
    cudaError_t e;
    {
        Prof pr(ctx, "vox_export");
        e = launch_vox_export(g, ctx->reqs, ctx->rots, n, dbits, ctx->stream, 0);
        if (e == cudaSuccess && sw->poses_lab)
            e = launch_vox_export(g, ctx->reqs, ctx->rots, n, dbits + per * n, ctx->stream, 1);
        else if (e == cudaSuccess)
            e = cudaMemsetAsync(dbits + per * n, 0, per * n, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(bits_c, dbits, per * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bits_n, dbits + per * n, per * n, cudaMemcpyDeviceToHost, ctx->stream);
    std::vector<RotRec> rr(n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rr.data(), ctx->rots, sizeof(RotRec) * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, dbits, 2 * per * n);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "voxelise_labels");
    // the scored non-contact grid is the part that no contact pose covers
    for (size_t i = 0; i < per * n; ++i) bits_n[i] = bits_n[i] && !bits_c[i];
    if (origins)
        for (int i = 0; i < n; ++i) memcpy(origins + 3 * i, rr[i].o, sizeof(double) * 3);
    return DOCK_OK;
}

static dock_status ensure_cells(dock_ctx *ctx, const dock_object *obc);

extern "C" dock_status dock_object_rotated(dock_ctx *ctx, const dock_object *ob, const double *quats, int32_t n,
                                           float *grids, double *origins)
{
    if (!ctx || !ob || !quats || n <= 0 || !grids) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    cudaSetDevice(ctx->device);
    dock_search_desc d = {};
    d.sampler = DOCK_SAMPLER_EXPLICIT;
    d.n = n;
    d.quats = quats;
    std::vector<double> q;
    dock_status s;
    if ((s = gen_samples(ctx, &d, q)) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->quats, &ctx->quats_n, (size_t)n * 4, sizeof(double))) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->rots, &ctx->rots_n, (size_t)n, sizeof(RotRec))) != DOCK_OK) return s;
    CK(ctx, cudaMemcpyAsync(ctx->quats, q.data(), sizeof(double) * 4 * n, cudaMemcpyHostToDevice, ctx->stream));
    // the object's origin drives the set-up (no sweep mean is read)
    CK(ctx, launch_rot_setup(ctx->quats, n, 0, 0, nullptr, ob->h, ob->N, ctx->rots, ctx->stream, ob->o_dev));
    if ((s = ensure_cells(ctx, ob)) != DOCK_OK) return s;
    ReqDev r = {};
    r.Og4 = ob->cells;
    r.rotate_object = 1;
    std::vector<ReqDev> rq(1, r);
    if ((s = upload_reqs(ctx, rq)) != DOCK_OK) return s;
    Geo g = {};
    g.N = ob->N;
    g.M = ob->M;
    g.P = ob->P;
    g.h = ob->h;
    const size_t per = (size_t)g.N * g.N * g.N;
    float *dg = nullptr;
    if ((s = dalloc(ctx, (void **)&dg, sizeof(float) * per * n, nullptr)) != DOCK_OK) return s;
    cudaError_t e;
    {
        Prof pr(ctx, "rot_export");
        e = launch_rot_export(g, ctx->reqs, ctx->rots, n, dg, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(grids, dg, sizeof(float) * per * n, cudaMemcpyDeviceToHost, ctx->stream);
    std::vector<RotRec> rr(n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rr.data(), ctx->rots, sizeof(RotRec) * n, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, dg, sizeof(float) * per * n);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "object_rotated");
    if (origins)
        for (int i = 0; i < n; ++i) memcpy(origins + 3 * i, rr[i].o, sizeof(double) * 3);
    return DOCK_OK;
}

// ---------------------------------------------------------------------------
// search
// ---------------------------------------------------------------------------
static int auto_batch(const Geo &g)
{
    size_t per = (size_t)(g.N + g.M) * g.M * g.P * sizeof(float2);
    // Y and Z of a batch: 12 GiB (126 rotations at 128^3; 2.6 % faster than 42, the
    // launches' tail waves amortised; HBM holds 280 GB)
    size_t lim = (size_t)12 << 30;
    size_t b = lim / per;
    if (b < 1) b = 1;
    if (b > 256) b = 256;
    return (int)b;
}

static dock_status check_pair(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw)
{
    if (ob->N != sw->N || ob->h != sw->h)
        return fail(ctx, DOCK_E_INVALID, "object and sweep lattices differ (N %d vs %d, h %g vs %g)", ob->N, sw->N,
                    ob->h, sw->h);
    return DOCK_OK;
}

// The launch shape of the search kernels for lattice side N: the tuned one
// when the autotuner (or its cache) has one, else the defaults.
// CTAs per plane of the inverse plane pass and columns per z-pass block at
// canvas 256 when untuned.
static const int PLANE_CL_DEFAULT = 8;
static const int ZPASS_COLS_DEFAULT = 16;
// Off by default: overlapped, the voxeliser and the FFT passes slow each other
// (both fill the register file), 1 % faster in all at 128^3, and per-kernel
// event times then overlap.
static const int VOX_OVERLAP_DEFAULT = 0;
static const int ZPASS_TC_DEFAULT = 0;
static const int PLANE_TMA_DEFAULT = 1;
static const int FWD_RUNS_DEFAULT = 1;
static const int FFT_PLAN_DEFAULT = 0;

static dock_tuning tuning_for(dock_ctx *ctx, const Geo &g)
{
    auto it = ctx->tune.find(g.N);
    if (it != ctx->tune.end()) return it->second;
    dock_tuning t = {};
    t.N = g.N;
    t.batch = auto_batch(g);
    t.group = 0;
    t.vox_blocks = 4;
    t.plane_cl = g.M == 256 ? PLANE_CL_DEFAULT : 0;
    t.zpass_cols = g.M == 256 ? ZPASS_COLS_DEFAULT : 0;
    t.vox_overlap = VOX_OVERLAP_DEFAULT;
    t.zpass_tc = g.M == 256 ? ZPASS_TC_DEFAULT : 0;
    t.plane_tma = g.M == 256 ? PLANE_TMA_DEFAULT : 0;
    t.fwd_runs = g.M == 256 ? FWD_RUNS_DEFAULT : 0;
    t.fft_plan = FFT_PLAN_DEFAULT;
    return t;
}

static bool valid_tuning(const dock_tuning &t)
{
    return valid_N(t.N) && t.batch >= 1 && t.batch <= 256 && t.group >= 0 && t.group <= 256 &&
           (t.vox_blocks == 3 || t.vox_blocks == 4) &&
           (t.plane_cl == 0 || t.plane_cl == 2 || t.plane_cl == 4 || t.plane_cl == 8) &&
           (t.zpass_cols == 0 || t.zpass_cols == 16 || t.zpass_cols == 32) &&
           (t.vox_overlap == 0 || t.vox_overlap == 1) && (t.zpass_tc == 0 || t.zpass_tc == 1) &&
           (t.plane_tma == 0 || t.plane_tma == 1) && (t.fwd_runs == 0 || t.fwd_runs == 1) &&
           (t.fft_plan == 0 || (t.fft_plan == 1 && (t.N == 32 || t.N == 64)));
}

// The forward x and y passes of a batch: the run-list kernel at canvas 256
// when the shape asks for it and no request of the batch rotates its object
// (those transform the resampled object grid), else k_fwd2d.
static cudaError_t fwd_pass(const dock_tuning &tc, const Geo &g, int B, const uint32_t *bits, float2 *Y,
                            const float2 *tw, const float2 *qt, cudaStream_t st, const uint32_t *mask,
                            const RotRec *rots, const ReqDev *reqs, const float *ogrids, bool ro_any)
{
    if (g.M == 256 && tc.fwd_runs && !ro_any) return launch_fwd2d_runs(g, B, bits, Y, qt, mask, st);
    return launch_fwd2d(g, B, bits, Y, tw, qt, st, mask, rots, reqs, ogrids, tc.fft_plan);
}

// Runs records [r0, r1) of rots through the search pipeline; every
// rotation's peak key lands in its request's key array (reqs[rot.req]).  All
// requests of the call share the lattice side of g.  dual: some request of
// the table is label-aware; each batch then also voxelises pose set 1, takes
// the voxels that set 0 leaves uncovered and adds their correlation with
// min(O, 0) in the z pass (requests without a set 1 are unaffected).
static dock_status run_pipeline_rots(dock_ctx *ctx, const Geo &g, const ReqDev *reqs, const RotRec *rots, size_t r0,
                                     size_t r1, int batch, bool dual = false, bool ro_any = false)
{
    float2 *tw, *qt;
    double2 *twd;
    dock_status s;
    if ((s = tables(ctx, g.M, &tw, &qt, &twd)) != DOCK_OK) return s;
    const dock_tuning tc = tuning_for(ctx, g);
    int B = batch > 0 ? batch : tc.batch;
    size_t ysz = (size_t)B * g.N * g.M * g.P, zsz = (size_t)B * g.M * g.M * g.P;
    size_t need = ysz + zsz + (dual ? ysz : 0);
    if (ctx->yz_bytes < need) {
        if (ctx->Y) {
            cudaStreamSynchronize(ctx->stream);
            dfree(ctx, ctx->Y, ctx->yz_bytes * sizeof(float2));
            ctx->Y = ctx->Z = nullptr;
            ctx->yz_bytes = 0;
        }
        if ((s = dalloc(ctx, (void **)&ctx->Y, need * sizeof(float2), nullptr)) != DOCK_OK) return s;
        ctx->yz_bytes = need;
    }
    float2 *Y = ctx->Y, *Z = ctx->Y + ysz, *Y2 = dual ? ctx->Y + ysz + zsz : nullptr;
    const size_t bsz = (size_t)B * g.N * g.N * (g.N / 32);
    // Overlap: the voxeliser of batch k + 1 runs on a second stream while the
    // FFT passes of batch k run (the voxeliser moves no data and is bound by
    // instruction issue, the FFT passes by latency); bits double-buffered,
    // batch k's bits released once its fwd2d has read them.
    const int nbatch = (int)((r1 - r0 + B - 1) / B);
    const bool ovl = tc.vox_overlap && !dual && nbatch > 1;
    if ((s = ensure(ctx, (void **)&ctx->bits, &ctx->bits_n, (dual || ovl) ? 2 * bsz : bsz, sizeof(uint32_t))) !=
        DOCK_OK)
        return s;
    uint32_t *bits2 = dual ? ctx->bits + bsz : nullptr;
    if (ovl) {
        if (!ctx->vstream) CK(ctx, cudaStreamCreateWithFlags(&ctx->vstream, cudaStreamNonBlocking));
        for (auto &e : ctx->vev)
            if (!e) CK(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        // everything enqueued before (rotation records, request table, the
        // previous users of the bits) precedes this call's voxelisations
        CK(ctx, cudaEventRecord(ctx->vev[4], ctx->stream));
        CK(ctx, cudaStreamWaitEvent(ctx->vstream, ctx->vev[4], 0));
    }
    if (ro_any &&
        (s = ensure(ctx, (void **)&ctx->ogr, &ctx->ogr_n, (size_t)B * g.N * g.N * g.N, sizeof(float))) != DOCK_OK)
        return s;
    int chunks = g.M * g.P / 32;
    int k = 0;
    for (size_t b0 = r0; b0 < r1; b0 += B, ++k) {
        int nb = (int)std::min<size_t>(B, r1 - b0);
        int groups_needed = (2 * 152 + chunks - 1) / chunks;
        int group = tc.group > 0 ? std::min(tc.group, nb) : std::max(1, nb / groups_needed);
        const RotRec *rb = rots + b0;
        const int kb = k & 1;
        uint32_t *bk = ovl ? ctx->bits + kb * bsz : ctx->bits;
        if (ovl) {
            if (k >= 2) CK(ctx, cudaStreamWaitEvent(ctx->vstream, ctx->vev[2 + kb], 0));   // fwd2d(k - 2) read bk
            {
                Prof pr(ctx, "voxelise", ctx->vstream);
                CK(ctx, launch_voxelise(g, reqs, rb, nb, bk, ctx->vstream, tc.vox_blocks));
            }
            CK(ctx, cudaEventRecord(ctx->vev[kb], ctx->vstream));
            CK(ctx, cudaStreamWaitEvent(ctx->stream, ctx->vev[kb], 0));
        } else {
            Prof pr(ctx, "voxelise");
            CK(ctx, launch_voxelise(g, reqs, rb, nb, bk, ctx->stream, tc.vox_blocks));
        }
        if (dual) {
            Prof pr(ctx, "voxelise_nc");
            CK(ctx, launch_voxelise(g, reqs, rb, nb, bits2, ctx->stream, tc.vox_blocks, 1));
        }
        if (ro_any) {
            Prof pr(ctx, "resample");
            CK(ctx, launch_resample(g, reqs, rb, nb, ctx->ogr, ctx->stream));
        }
        {
            Prof pr(ctx, "fwd2d");
            CK(ctx, fwd_pass(tc, g, nb, bk, Y, tw, qt, ctx->stream, nullptr, rb, reqs, ro_any ? ctx->ogr : nullptr, ro_any));
        }
        if (ovl) CK(ctx, cudaEventRecord(ctx->vev[2 + kb], ctx->stream));
        if (dual) {
            Prof pr(ctx, "fwd2d_nc");
            CK(ctx, fwd_pass(tc, g, nb, bits2, Y2, tw, qt, ctx->stream, ctx->bits, rb, reqs, nullptr, ro_any));
        }
        {
            Prof pr(ctx, dual ? "zpass_dual" : "zpass");
            if (g.M == 256 && tc.zpass_cols == 16 && tc.zpass_tc && !dual)
                CK(ctx, launch_zpass_tc(g, nb, group, Y, rb, reqs, Z, ctx->errflag, ctx->stream));
            else if (g.M == 256 && tc.zpass_cols == 16 && !dual)
                CK(ctx, launch_zpass16(g, nb, group, Y, rb, reqs, Z, ctx->stream));
            else if (g.M == 256 && tc.zpass_cols == 16)
                CK(ctx, launch_zpass16_dual(g, nb, group, Y, Y2, rb, reqs, Z, ctx->stream));
            else
                CK(ctx, launch_zpass(g, nb, group, Y, rb, reqs, Z, tw, ctx->stream, Y2, tc.fft_plan));
        }
        {
            Prof pr(ctx, "plane");
            CK(ctx, launch_plane(g, nb, Z, tw, rb, reqs, ctx->stream, tc.plane_cl, ctx->errflag, tc.plane_tma, tc.fft_plan));
        }
    }
    return DOCK_OK;
}

static dock_status run_pipeline(dock_ctx *ctx, const Geo &g, size_t r0, size_t r1, int batch, bool dual, bool ro)
{
    return run_pipeline_rots(ctx, g, ctx->reqs, ctx->rots, r0, r1, batch, dual, ro);
}

// The label-aware score of a sweep in `mode` (one read of dock_sweep::mode)
// is in force and differs from the plain one.
static bool dual_scoring(const dock_sweep *sw, int mode) { return (mode & SCORE_LABEL_AWARE) && sw->poses_lab != nullptr; }

// conj(F(min(O, 0))) / M^3 of the object, made on first use and kept with it.
static dock_status ensure_spec_pen(dock_ctx *ctx, const dock_object *obc)
{
    dock_object *ob = const_cast<dock_object *>(obc);
    if (ob->spec_pen) return DOCK_OK;
    const int N = ob->N, M = ob->M, P = ob->P;
    float2 *tw, *qt;
    double2 *twd;
    dock_status s;
    if ((s = tables(ctx, M, &tw, &qt, &twd)) != DOCK_OK) return s;
    const size_t spec_n = (size_t)M * P / 32 * M * 32;
    const size_t b1 = sizeof(double2) * (size_t)N * N * (N + 1), b2 = sizeof(double2) * (size_t)N * M * (N + 1);
    float2 *sp = nullptr;
    double2 *w1 = nullptr, *w2 = nullptr;
    size_t held = 0;
    if ((s = dalloc(ctx, (void **)&sp, sizeof(float2) * spec_n, &held)) != DOCK_OK) return s;
    if ((s = dalloc(ctx, (void **)&w1, b1, nullptr)) != DOCK_OK) { dfree(ctx, sp, sizeof(float2) * spec_n); return s; }
    if ((s = dalloc(ctx, (void **)&w2, b2, nullptr)) != DOCK_OK) {
        dfree(ctx, sp, sizeof(float2) * spec_n);
        dfree(ctx, w1, b1);
        return s;
    }
    cudaError_t e;
    {
        Prof pr(ctx, "object_spectrum_pen");
        e = launch_spectrum(ob->O, N, M, P, w1, w2, twd, sp, ctx->stream, true);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, w1, b1);
    dfree(ctx, w2, b2);
    if (e != cudaSuccess) {
        dfree(ctx, sp, sizeof(float2) * spec_n);
        return cuda_fail(ctx, e, "penetration spectrum");
    }
    ob->spec_pen = sp;
    ob->bytes += held;
    return DOCK_OK;
}

// Corner cells of the object grid for the rotated-object search (4 (N+1)^3
// floats), made on first use and kept with the object.
static dock_status ensure_cells(dock_ctx *ctx, const dock_object *obc)
{
    dock_object *ob = const_cast<dock_object *>(obc);
    if (ob->cells) return DOCK_OK;
    const size_t n = (size_t)(ob->N + 1) * (ob->N + 1) * (ob->N + 1);
    float4 *c = nullptr;
    size_t held = 0;
    dock_status s;
    if ((s = dalloc(ctx, (void **)&c, sizeof(float4) * n, &held)) != DOCK_OK) return s;
    cudaError_t e = launch_corner_cells(ob->O, ob->N, c, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        dfree(ctx, c, sizeof(float4) * n);
        return cuda_fail(ctx, e, "corner cells");
    }
    ob->cells = c;
    ob->bytes += held;
    return DOCK_OK;
}

// The fixed swept grid of the rotated-object search: S voxelised on the
// lattice of the identity rotation (origin o_s = h round(c_s / h) - (N/2) h),
// its spectrum F(S) / M^3 and o_s, made on first use and kept with the sweep.
static dock_status ensure_spec_S(dock_ctx *ctx, const dock_sweep *swc)
{
    dock_sweep *sw = const_cast<dock_sweep *>(swc);
    if (sw->spec_S) return DOCK_OK;
    const Geo g = make_geo(sw);
    const int N = g.N, M = g.M, P = g.P;
    float2 *tw, *qt;
    double2 *twd;
    dock_status s;
    if ((s = tables(ctx, M, &tw, &qt, &twd)) != DOCK_OK) return s;
    const double qi[4] = {1.0, 0.0, 0.0, 0.0};
    if ((s = upload_rots(ctx, sw, qi, 1, 0, 1, 0, 0)) != DOCK_OK) return s;
    std::vector<ReqDev> rq(1, make_reqdev(nullptr, sw, nullptr, false));
    if ((s = upload_reqs(ctx, rq)) != DOCK_OK) return s;
    const size_t spec_n = (size_t)M * P / 32 * M * 32;
    const size_t bS = sizeof(float) * (size_t)N * N * N;
    const size_t b1 = sizeof(double2) * (size_t)N * N * (N + 1), b2 = sizeof(double2) * (size_t)N * M * (N + 1);
    float2 *sp = nullptr;
    double *os = nullptr;
    float *Sg = nullptr;
    double2 *w1 = nullptr, *w2 = nullptr;
    size_t held = 0;
    auto release = [&](bool keep) {
        dfree(ctx, Sg, bS);
        dfree(ctx, w1, b1);
        dfree(ctx, w2, b2);
        if (!keep) {
            dfree(ctx, sp, sizeof(float2) * spec_n);
            dfree(ctx, os, sizeof(double) * 3);
        }
    };
    if ((s = dalloc(ctx, (void **)&sp, sizeof(float2) * spec_n, &held)) != DOCK_OK) return s;
    if ((s = dalloc(ctx, (void **)&os, sizeof(double) * 3, &held)) != DOCK_OK) { release(false); return s; }
    if ((s = dalloc(ctx, (void **)&Sg, bS, nullptr)) != DOCK_OK) { release(false); return s; }
    if ((s = dalloc(ctx, (void **)&w1, b1, nullptr)) != DOCK_OK) { release(false); return s; }
    if ((s = dalloc(ctx, (void **)&w2, b2, nullptr)) != DOCK_OK) { release(false); return s; }
    cudaError_t e;
    {
        Prof pr(ctx, "sweep_spectrum");
        e = launch_vox_float(g, ctx->reqs, ctx->rots, Sg, ctx->stream);
        if (e == cudaSuccess) e = launch_spectrum(Sg, N, M, P, w1, w2, twd, sp, ctx->stream, false, false);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(os, reinterpret_cast<const char *>(ctx->rots) + offsetof(RotRec, o), sizeof(double) * 3,
                            cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        release(false);
        return cuda_fail(ctx, e, "swept-grid spectrum");
    }
    release(true);
    sw->spec_S = sp;
    sw->os_dev = os;
    sw->bytes += held;
    return DOCK_OK;
}

// The search of this sweep rotates the object grid.
static bool rotates_object(int mode) { return (mode & SCORE_ROTATE_OBJECT) != 0; }

static dock_status search_impl(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw, const dock_search_desc *d,
                               const std::vector<double> &q, int r0, int r1, dock_candidate *out, dock_peak *per_rot)
{
    const int n = d->n;
    dock_status s;
    const int mode = sw->mode.load();   // one read: the two options are exclusive
    const bool ro = rotates_object(mode);
    if (ro && ((s = ensure_spec_S(ctx, sw)) != DOCK_OK || (s = ensure_cells(ctx, ob)) != DOCK_OK)) return s;
    if ((s = upload_rots(ctx, sw, q.data(), n, 0, n, 0, 0, ro ? ob->o_dev : nullptr)) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->keys, &ctx->keys_n, (size_t)n, sizeof(unsigned long long))) != DOCK_OK) return s;
    CK(ctx, cudaMemsetAsync(ctx->keys, 0, sizeof(unsigned long long) * n, ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->errflag, 0, sizeof(int), ctx->stream));
    const bool dual = dual_scoring(sw, mode);
    if (dual && (s = ensure_spec_pen(ctx, ob)) != DOCK_OK) return s;
    std::vector<ReqDev> rq(1, make_reqdev(ob, sw, ctx->keys, dual, ro));
    if ((s = upload_reqs(ctx, rq)) != DOCK_OK) return s;
    if ((s = run_pipeline(ctx, make_geo(sw), r0, r1, d->batch, dual, ro)) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->cands, &ctx->cands_n, (size_t)d->top_k, sizeof(dock_candidate))) != DOCK_OK) return s;
    {
        Prof pr(ctx, "topk");
        CK(ctx, launch_topk(ctx->keys, n, d->top_k, ob->N, ob->M, ob->h, ob->o_dev, ctx->quats, ctx->rots, ctx->cands,
                            ctx->stream, ro ? sw->os_dev : nullptr));
    }
    CK(ctx, cudaMemcpyAsync(out, ctx->cands, sizeof(dock_candidate) * d->top_k, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<unsigned long long> keys;
    if (per_rot) {
        keys.resize(n);
        CK(ctx, cudaMemcpyAsync(keys.data(), ctx->keys, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, ctx->stream));
    }
    int herr = 0;
    CK(ctx, cudaMemcpyAsync(&herr, ctx->errflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (herr) return fail(ctx, herr, "device reported error %d during the search", herr);
    if (per_rot) {
        for (int i = r0; i < r1; ++i) {
            unsigned long long k = keys[i];
            uint32_t sk = (uint32_t)(k >> 32);
            uint32_t u = (sk & 0x80000000u) ? (sk & 0x7FFFFFFFu) : ~sk;
            float f;
            memcpy(&f, &u, 4);
            per_rot[i].score = k ? f : -INFINITY;
            per_rot[i].canvas_idx = k ? (int32_t)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull)) : -1;
        }
    }
    return DOCK_OK;
}

extern "C" dock_status dock_search_so3(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                       const dock_search_desc *d, dock_candidate *out, dock_peak *per_rot)
{
    if (!ctx || !ob || !sw || !d || !out) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    dock_status s;
    if ((s = check_pair(ctx, ob, sw)) != DOCK_OK) return s;
    if (d->top_k < 1 || d->top_k > 1024) return fail(ctx, DOCK_E_INVALID, "top_k must be in [1, 1024]");
    int r0 = d->rot_begin, r1 = d->rot_end > 0 ? d->rot_end : d->n;
    if (r0 < 0 || r1 > d->n || r0 >= r1) return fail(ctx, DOCK_E_INVALID, "bad rotation range [%d, %d) of %d", r0, r1, d->n);
    cudaSetDevice(ctx->device);
    std::vector<double> q;
    if ((s = gen_samples(ctx, d, q)) != DOCK_OK) return s;
    return search_impl(ctx, ob, sw, d, q, r0, r1, out, per_rot);
}

extern "C" dock_status dock_search_peaks_noalloc(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                                 const double *quats, int32_t n, dock_peak *peaks)
{
    if (!ctx || !ob || !sw || !quats || !peaks) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    dock_status s;
    if ((s = check_pair(ctx, ob, sw)) != DOCK_OK) return s;
    if (ob->N > NOALLOC_MAX_N)
        return fail(ctx, DOCK_E_INVALID, "lattice side %d exceeds the scratch limit %d of dock_search_peaks_noalloc",
                    ob->N, NOALLOC_MAX_N);
    if (n < 1 || n > NOALLOC_MAX_ROT)
        return fail(ctx, DOCK_E_INVALID, "rotation count %d outside [1, %d] of dock_search_peaks_noalloc", n,
                    NOALLOC_MAX_ROT);
    if (sw->mode.load() != 0)
        return fail(ctx, DOCK_E_INVALID,
                    "dock_search_peaks_noalloc rotates the sweep and scores plainly; the sweep asks otherwise");
    {
        // its copies come from pageable host memory and it synchronises the
        // stream: neither can be recorded into a graph
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaError_t ce = cudaStreamIsCapturing(ctx->stream, &cs);
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamIsCapturing");
        if (cs != cudaStreamCaptureStatusNone)
            return fail(ctx, DOCK_E_INVALID, "dock_search_peaks_noalloc must not be called on a capturing stream");
    }
    for (int i = 0; i < n; ++i) {
        const double *a = quats + 4 * (size_t)i;
        double nq = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2] + a[3] * a[3]);
        if (!(fabs(nq - 1.0) <= 1e-6)) return fail(ctx, DOCK_E_INVALID, "quaternion %d is not unit", i);
    }
    // the twiddle tables of this canvas side were made with the object
    auto it = ctx->tw.find(ob->M);
    auto iq = ctx->qt.find(ob->M);
    if (it == ctx->tw.end() || iq == ctx->qt.end()) return fail(ctx, DOCK_E_INVALID, "no twiddle tables for M = %d", ob->M);
    cudaSetDevice(ctx->device);
    NoallocJob j;
    j.device = ctx->device;
    j.g = make_geo(sw);
    j.req = make_reqdev(ob, sw, nullptr, false);
    j.c_s = sw->cs_dev;
    j.quats = quats;
    j.n = n;
    j.tw = it->second;
    j.qt = iq->second;
    j.stream = ctx->stream;
    j.peaks = peaks;
    CK(ctx, noalloc_search_peaks(j));
    return DOCK_OK;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
static dock_status time_shape(dock_ctx *ctx, const Geo &g, int n, const dock_tuning &t, double *us)
{
    ctx->tune[g.N] = t;
    dock_status s;
    // every run starts from cleared peak keys, as a search does (the plane
    // passes skip work for rows below a rotation's best score so far)
    CK(ctx, cudaMemsetAsync(ctx->keys, 0, sizeof(unsigned long long) * n, ctx->stream));
    if ((s = run_pipeline_rots(ctx, g, ctx->reqs, ctx->rots, 0, n, 0)) != DOCK_OK) return s;   // warm-up
    CK(ctx, cudaMemsetAsync(ctx->keys, 0, sizeof(unsigned long long) * n, ctx->stream));
    cudaEvent_t a = nullptr, b = nullptr;
    CK(ctx, cudaEventCreate(&a));
    cudaError_t e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        return cuda_fail(ctx, e, "cudaEventCreate");
    }
    e = cudaEventRecord(a, ctx->stream);
    if (e == cudaSuccess) s = run_pipeline_rots(ctx, g, ctx->reqs, ctx->rots, 0, n, 0);
    if (e == cudaSuccess && s == DOCK_OK) e = cudaEventRecord(b, ctx->stream);
    if (e == cudaSuccess && s == DOCK_OK) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess && s == DOCK_OK) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (s != DOCK_OK) return s;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "timing a launch shape");
    *us = 1000.0 * ms / n;
    return DOCK_OK;
}

static std::string device_name(int dev)
{
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "unknown";
    std::string n = pr.name;
    for (auto &ch : n)
        if (ch == '"' || ch == '\\') ch = '_';
    return n;
}

static dock_status write_tuning(dock_ctx *ctx, const char *path)
{
    FILE *f = fopen(path, "w");
    if (!f) return fail(ctx, DOCK_E_INVALID, "cannot write the tuning cache %s", path);
    fprintf(f, "{\"device\": \"%s\", \"entries\": [", device_name(ctx->device).c_str());
    bool first = true;
    for (auto &kv : ctx->tune) {
        const dock_tuning &t = kv.second;
        fprintf(f,
                "%s\n  {\"N\": %d, \"batch\": %d, \"group\": %d, \"vox_blocks\": %d, \"plane_cl\": %d, "
                "\"zpass_cols\": %d, \"vox_overlap\": %d, \"zpass_tc\": %d, \"plane_tma\": %d, \"fwd_runs\": %d, \"fft_plan\": %d, \"us_per_rotation\": %.3f}",
                first ? "" : ",", t.N, t.batch, t.group, t.vox_blocks, t.plane_cl, t.zpass_cols, t.vox_overlap,
                t.zpass_tc, t.plane_tma, t.fwd_runs, t.fft_plan, t.us_per_rotation);
        first = false;
    }
    fprintf(f, "\n]}\n");
    bool ok = ferror(f) == 0;
    ok = (fclose(f) == 0) && ok;
    return ok ? DOCK_OK : fail(ctx, DOCK_E_INVALID, "cannot write the tuning cache %s", path);
}

extern "C" dock_status dock_autotune(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw, int32_t n_rot,
                                     const char *cache_path, dock_tuning *out)
{
    if (!ctx || !ob || !sw) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    dock_status s;
    if ((s = check_pair(ctx, ob, sw)) != DOCK_OK) return s;
    if (n_rot < 16 || n_rot > 65536) return fail(ctx, DOCK_E_INVALID, "n_rot must be in [16, 65536]");
    cudaSetDevice(ctx->device);
    dock_search_desc d = {};
    d.sampler = DOCK_SAMPLER_SF;
    d.n = n_rot;
    std::vector<double> q;
    if ((s = gen_samples(ctx, &d, q)) != DOCK_OK) return s;
    if ((s = upload_rots(ctx, sw, q.data(), n_rot, 0, n_rot, 0, 0)) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->keys, &ctx->keys_n, (size_t)n_rot, sizeof(unsigned long long))) != DOCK_OK)
        return s;
    CK(ctx, cudaMemsetAsync(ctx->keys, 0, sizeof(unsigned long long) * n_rot, ctx->stream));
    std::vector<ReqDev> rq(1, make_reqdev(ob, sw, ctx->keys, false));   // plain score: its launch shape
    if ((s = upload_reqs(ctx, rq)) != DOCK_OK) return s;
    const Geo g = make_geo(sw);
    const bool had = ctx->tune.count(g.N) != 0;
    const dock_tuning prev = had ? ctx->tune[g.N] : dock_tuning{};
    ctx->tune.erase(g.N);
    dock_tuning best = tuning_for(ctx, g);
    const int bmax = std::min(auto_batch(g), n_rot);
    best.batch = std::min(best.batch, bmax);
    double best_us = 0.0;
    auto restore = [&] {
        if (had) ctx->tune[g.N] = prev;
        else ctx->tune.erase(g.N);
    };
    if ((s = time_shape(ctx, g, n_rot, best, &best_us)) != DOCK_OK) { restore(); return s; }
    auto trial = [&](dock_tuning t) -> dock_status {
        double us = 0.0;
        dock_status st = time_shape(ctx, g, n_rot, t, &us);
        if (st != DOCK_OK) return st;
        if (us < best_us) {
            best = t;
            best_us = us;
        }
        return DOCK_OK;
    };
    {
        dock_tuning t = best;
        t.vox_blocks = best.vox_blocks == 4 ? 3 : 4;
        if ((s = trial(t)) != DOCK_OK) { restore(); return s; }
    }
    for (int b : {8, 16, 32, 64, 128, 256}) {
        if (b > bmax || b == best.batch) continue;
        dock_tuning t = best;
        t.batch = b;
        if ((s = trial(t)) != DOCK_OK) { restore(); return s; }
    }
    for (int gr : {1, 2, 4, 8, 16}) {
        if (gr > best.batch) continue;
        dock_tuning t = best;
        t.group = gr;
        if ((s = trial(t)) != DOCK_OK) { restore(); return s; }
    }
    if (g.M == 64 || g.M == 128) {   // the alternative radix plan of the FFTs
        dock_tuning t = best;
        t.fft_plan = best.fft_plan ? 0 : 1;
        if ((s = trial(t)) != DOCK_OK) { restore(); return s; }
    }
    if (g.M == 256) {
        for (int cl : {2, 4, 8}) {
            if (cl == best.plane_cl) continue;
            dock_tuning t = best;
            t.plane_cl = cl;
            if ((s = trial(t)) != DOCK_OK) { restore(); return s; }
        }
        if (best.plane_cl == 4 || best.plane_cl == 8) {
            dock_tuning t = best;
            t.plane_tma = best.plane_tma ? 0 : 1;
            if ((s = trial(t)) != DOCK_OK) { restore(); return s; }
        }
        {
            dock_tuning t = best;
            t.fwd_runs = best.fwd_runs ? 0 : 1;
            if ((s = trial(t)) != DOCK_OK) { restore(); return s; }
        }
        {
            dock_tuning t = best;
            t.zpass_cols = best.zpass_cols == 16 ? 32 : 16;
            t.zpass_tc = 0;
            if ((s = trial(t)) != DOCK_OK) { restore(); return s; }
        }
        if (best.zpass_cols == 16) {
            dock_tuning t = best;
            t.zpass_tc = best.zpass_tc ? 0 : 1;
            if ((s = trial(t)) != DOCK_OK) { restore(); return s; }
        }
    }
    best.us_per_rotation = best_us;
    ctx->tune[g.N] = best;
    if (out) *out = best;
    if (cache_path && (s = write_tuning(ctx, cache_path)) != DOCK_OK) return s;
    return DOCK_OK;
}

static bool json_int(const char *p, const char *key, long *v)
{
    const char *k = strstr(p, key);
    if (!k) return false;
    k = strchr(k, ':');
    return k && sscanf(k + 1, "%ld", v) == 1;
}

extern "C" dock_status dock_load_tuning(dock_ctx *ctx, const char *path, int32_t *n_loaded)
{
    if (!ctx || !path) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (n_loaded) *n_loaded = 0;
    FILE *f = fopen(path, "r");
    if (!f) return fail(ctx, DOCK_E_INVALID, "cannot read the tuning cache %s", path);
    std::string txt;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, got);
    fclose(f);
    const std::string want = "\"device\": \"" + device_name(ctx->device) + "\"";
    if (txt.find(want) == std::string::npos) return DOCK_OK;   // tuned on another device
    int n = 0;
    size_t pos = 0;
    while ((pos = txt.find("{\"N\":", pos)) != std::string::npos) {
        size_t end = txt.find('}', pos);
        if (end == std::string::npos) break;
        std::string e = txt.substr(pos, end - pos);
        long N, b, gr, vb, pc = -1;
        if (json_int(e.c_str(), "\"N\"", &N) && json_int(e.c_str(), "\"batch\"", &b) &&
            json_int(e.c_str(), "\"group\"", &gr) && json_int(e.c_str(), "\"vox_blocks\"", &vb)) {
            dock_tuning t = {};
            t.N = (int)N;
            t.batch = (int)b;
            t.group = (int)gr;
            t.vox_blocks = (int)vb;
            Geo gt = {};
            gt.M = 2 * t.N;
            t.plane_cl = json_int(e.c_str(), "\"plane_cl\"", &pc) ? (int)pc : (gt.M == 256 ? PLANE_CL_DEFAULT : 0);
            long zc = 0;
            t.zpass_cols =
                json_int(e.c_str(), "\"zpass_cols\"", &zc) ? (int)zc : (gt.M == 256 ? ZPASS_COLS_DEFAULT : 0);
            long vo = VOX_OVERLAP_DEFAULT;
            json_int(e.c_str(), "\"vox_overlap\"", &vo);
            t.vox_overlap = (int)vo;
            long zt = gt.M == 256 ? ZPASS_TC_DEFAULT : 0;
            json_int(e.c_str(), "\"zpass_tc\"", &zt);
            t.zpass_tc = (int)zt;
            long pt = gt.M == 256 ? PLANE_TMA_DEFAULT : 0;
            json_int(e.c_str(), "\"plane_tma\"", &pt);
            t.plane_tma = (int)pt;
            long fr = gt.M == 256 ? FWD_RUNS_DEFAULT : 0;
            json_int(e.c_str(), "\"fwd_runs\"", &fr);
            t.fwd_runs = (int)fr;
            long fp = FFT_PLAN_DEFAULT;
            json_int(e.c_str(), "\"fft_plan\"", &fp);
            t.fft_plan = (int)fp;
            if (!valid_tuning(t)) {
                pos = end;
                continue;
            }
            const char *u = strstr(e.c_str(), "\"us_per_rotation\"");
            if (u && (u = strchr(u, ':'))) t.us_per_rotation = atof(u + 1);
            ctx->tune[t.N] = t;
            ++n;
        }
        pos = end;
    }
    if (n_loaded) *n_loaded = n;
    return DOCK_OK;
}

extern "C" dock_status dock_get_tuning(dock_ctx *ctx, int32_t N, dock_tuning *out)
{
    if (!ctx || !out) return DOCK_E_INVALID;
    if (!valid_N(N)) return fail(ctx, DOCK_E_INVALID, "lattice side %d not supported", N);
    DevLock dev_lock_(ctx);
    Geo g = {};
    g.N = N;
    g.M = 2 * N;
    g.P = N + 2;
    *out = tuning_for(ctx, g);
    return DOCK_OK;
}

extern "C" dock_status dock_memory_stats(dock_ctx *ctx, size_t *held, size_t *peak, size_t *budget)
{
    if (!ctx) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (held) *held = ctx->held;
    if (peak) *peak = ctx->peak_held;
    if (budget) *budget = ctx->budget;
    return DOCK_OK;
}

extern "C" dock_status dock_fail_allocation(dock_ctx *ctx, int32_t n)
{
    if (!ctx || n < 0) return DOCK_E_INVALID;
    ctx->fail_alloc.store(n);
    return DOCK_OK;
}

extern "C" dock_status dock_set_tuning(dock_ctx *ctx, const dock_tuning *t)
{
    if (!ctx || !t) return DOCK_E_INVALID;
    if (!valid_tuning(*t)) return fail(ctx, DOCK_E_INVALID, "tuning out of range");
    DevLock dev_lock_(ctx);
    ctx->tune[t->N] = *t;
    return DOCK_OK;
}

// The full correlation field of one rotation (the search kernels with the
// plane pass exporting every value).  withhold: the test hook of the bounded
// wait of the cluster plane pass (its peers' blocks are never pushed).
static dock_status search_scores_impl(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw, const double *quat,
                                      float *C, int withhold)
{
    if (!ctx || !ob || !sw || !quat || !C) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    dock_status s;
    if ((s = check_pair(ctx, ob, sw)) != DOCK_OK) return s;
    cudaSetDevice(ctx->device);
    dock_search_desc d = {};
    d.sampler = DOCK_SAMPLER_EXPLICIT;
    d.n = 1;
    d.quats = quat;
    std::vector<double> q;
    if ((s = gen_samples(ctx, &d, q)) != DOCK_OK) return s;
    const int mode = sw->mode.load();   // one read: the two options are exclusive
    const bool ro = rotates_object(mode);
    if (ro && ((s = ensure_spec_S(ctx, sw)) != DOCK_OK || (s = ensure_cells(ctx, ob)) != DOCK_OK)) return s;
    if ((s = upload_rots(ctx, sw, q.data(), 1, 0, 1, 0, 0, ro ? ob->o_dev : nullptr)) != DOCK_OK) return s;
    const bool dual = dual_scoring(sw, mode);
    if (dual && (s = ensure_spec_pen(ctx, ob)) != DOCK_OK) return s;
    std::vector<ReqDev> rq(1, make_reqdev(ob, sw, nullptr, dual, ro));
    if ((s = upload_reqs(ctx, rq)) != DOCK_OK) return s;
    Geo g = make_geo(sw);
    float2 *tw, *qt;
    double2 *twd;
    if ((s = tables(ctx, g.M, &tw, &qt, &twd)) != DOCK_OK) return s;
    size_t ysz = (size_t)g.N * g.M * g.P, zsz = (size_t)g.M * g.M * g.P, csz = (size_t)g.M * g.M * g.M;
    const size_t ybytes = (ysz + zsz + (dual ? ysz : 0)) * sizeof(float2);
    const size_t bsz = (size_t)g.N * g.N * (g.N / 32);
    float2 *Y = nullptr;
    float *dC = nullptr;
    if ((s = ensure(ctx, (void **)&ctx->bits, &ctx->bits_n, 2 * bsz, sizeof(uint32_t))) != DOCK_OK) return s;
    if ((s = dalloc(ctx, (void **)&Y, ybytes, nullptr)) != DOCK_OK) return s;
    if ((s = dalloc(ctx, (void **)&dC, csz * sizeof(float), nullptr)) != DOCK_OK) { dfree(ctx, Y, ybytes); return s; }
    float2 *Y2 = dual ? Y + ysz + zsz : nullptr;
    const dock_tuning tc = tuning_for(ctx, g);
    cudaError_t e = cudaMemsetAsync(ctx->errflag, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = launch_voxelise(g, ctx->reqs, ctx->rots, 1, ctx->bits, ctx->stream);
    if (e == cudaSuccess)
        e = fwd_pass(tc, g, 1, ctx->bits, Y, tw, qt, ctx->stream, nullptr, ctx->rots, ctx->reqs, nullptr, ro);
    if (dual && e == cudaSuccess) e = launch_voxelise(g, ctx->reqs, ctx->rots, 1, ctx->bits + bsz, ctx->stream, 4, 1);
    if (dual && e == cudaSuccess)
        e = fwd_pass(tc, g, 1, ctx->bits + bsz, Y2, tw, qt, ctx->stream, ctx->bits, ctx->rots, ctx->reqs, nullptr, ro);
    if (e == cudaSuccess) {
        if (g.M == 256 && tc.zpass_cols == 16 && tc.zpass_tc && !dual)
            e = launch_zpass_tc(g, 1, 1, Y, ctx->rots, ctx->reqs, Y + ysz, ctx->errflag, ctx->stream);
        else if (g.M == 256 && tc.zpass_cols == 16 && !dual)
            e = launch_zpass16(g, 1, 1, Y, ctx->rots, ctx->reqs, Y + ysz, ctx->stream);
        else if (g.M == 256 && tc.zpass_cols == 16)
            e = launch_zpass16_dual(g, 1, 1, Y, Y2, ctx->rots, ctx->reqs, Y + ysz, ctx->stream);
        else
            e = launch_zpass(g, 1, 1, Y, ctx->rots, ctx->reqs, Y + ysz, tw, ctx->stream, Y2, tc.fft_plan);
    }
    if (e == cudaSuccess)
        e = withhold ? (tc.plane_tma && plane_ps_supported(g.M, tc.plane_cl)
                            ? launch_plane_ps_export(g, tc.plane_cl, Y + ysz, dC, ctx->errflag, ctx->stream, 1)
                            : launch_plane_cl_export(g, tc.plane_cl, Y + ysz, tw, dC, ctx->errflag, ctx->stream, 1))
                     : launch_plane_export(g, Y + ysz, tw, dC, ctx->stream, tc.plane_cl, ctx->errflag, tc.plane_tma, tc.fft_plan);
    if (e == cudaSuccess) e = cudaMemcpyAsync(C, dC, csz * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, ctx->errflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, Y, ybytes);
    dfree(ctx, dC, csz * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "search_scores");
    if (herr) {
        cudaMemsetAsync(ctx->errflag, 0, sizeof(int), ctx->stream);
        return fail(ctx, herr, "device reported error %d during the search", herr);
    }
    return DOCK_OK;
}

extern "C" dock_status dock_search_scores(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw, const double *quat,
                                          float *C)
{
    return search_scores_impl(ctx, ob, sw, quat, C, 0);
}

extern "C" dock_status dock_test_plane_timeout(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                               const double *quat, float *C)
{
    if (!ctx || !ob || !sw) return DOCK_E_INVALID;
    Geo g = make_geo(sw);
    if (!plane_cl_supported(g.M, tuning_for(ctx, g).plane_cl))
        return fail(ctx, DOCK_E_INVALID, "the timeout hook needs the cluster plane pass (canvas 256, plane_cl 4 or 8)");
    return search_scores_impl(ctx, ob, sw, quat, C, 1);
}

extern "C" dock_status dock_sample_so3(const dock_search_desc *d, double *quats)
{
    if (!d || !quats) return DOCK_E_INVALID;
    std::vector<double> q;
    dock_status s = gen_samples(nullptr, d, q);
    if (s != DOCK_OK) return s;
    memcpy(quats, q.data(), sizeof(double) * q.size());
    return DOCK_OK;
}

// ---------------------------------------------------------------------------
// refinement (Sec. V)
// ---------------------------------------------------------------------------
static RefineDev make_refine_dev(const dock_object *ob, const dock_sweep *sw, const dock_params *p)
{
    RefineDev D;
    D.Vf = ob->Vf;
    D.T = ob->T;
    D.tri_sphere = ob->tri_sphere;
    D.tri_order = ob->tri_order;
    D.nodes = ob->nodes;
    D.poses = sw->poses;
    D.P = (int)sw->P;
    D.r = (float)sw->r;
    D.L = (float)sw->L;
    D.tau_out = (float)p->tau_out2;
    D.tau_in = (float)p->tau_in2;
    D.k_slope = (float)p->k_slope;
    // Eq. (18): r = tau_in / tau_out; C^1 at t = -r and t = 0 needs
    // A = k/r^2 - 2/r^3, B = k/r - 3/r^2
    double r = p->tau_in2 / p->tau_out2, k = p->k_slope;
    D.rr = (float)r;
    D.A = (float)(k / (r * r) - 2.0 / (r * r * r));
    D.B = (float)(k / r - 3.0 / (r * r));
    D.tri_iters = p->tri_iters > 0 ? p->tri_iters : 20;
    return D;
}

static dock_status ref_buffers(dock_ctx *ctx, RefBufs &rb, int K, int nblk)
{
    dock_status s;
    if ((s = ensure(ctx, (void **)&rb.state, &rb.state_n, (size_t)K * REF_ST, sizeof(double))) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&rb.acc, &rb.acc_n, (size_t)K * nblk * REF_NACC, sizeof(double))) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&rb.prm, &rb.prm_n, 16, sizeof(double))) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&rb.cands, &rb.cands_n, (size_t)K, cand_bytes())) != DOCK_OK) return s;
    return DOCK_OK;
}

static void state_from_pose(const double *q, const double *t, const double *anchor, double *st)
{
    quat_to_mat(q, st);
    for (int a = 0; a < 3; ++a) { st[9 + a] = t[a]; st[12 + a] = anchor[a]; }
    for (int j = 15; j < REF_ST; ++j) st[j] = 0.0;
}

static void mat_to_quat(const double *m, double *q)
{
    double tr = m[0] + m[4] + m[8];
    if (tr > 0) {
        double s = sqrt(tr + 1.0) * 2;
        q[0] = 0.25 * s; q[1] = (m[7] - m[5]) / s; q[2] = (m[2] - m[6]) / s; q[3] = (m[3] - m[1]) / s;
    } else if (m[0] > m[4] && m[0] > m[8]) {
        double s = sqrt(1.0 + m[0] - m[4] - m[8]) * 2;
        q[0] = (m[7] - m[5]) / s; q[1] = 0.25 * s; q[2] = (m[1] + m[3]) / s; q[3] = (m[2] + m[6]) / s;
    } else if (m[4] > m[8]) {
        double s = sqrt(1.0 + m[4] - m[0] - m[8]) * 2;
        q[0] = (m[2] - m[6]) / s; q[1] = (m[1] + m[3]) / s; q[2] = 0.25 * s; q[3] = (m[5] + m[7]) / s;
    } else {
        double s = sqrt(1.0 + m[8] - m[0] - m[4]) * 2;
        q[0] = (m[3] - m[1]) / s; q[1] = (m[2] + m[6]) / s; q[2] = (m[5] + m[7]) / s; q[3] = 0.25 * s;
    }
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double sg = q[0] < 0 ? -1.0 : 1.0;
    for (int k = 0; k < 4; ++k) q[k] = sg * q[k] / n;
}

// T(xi) of Eq. (14)-(17) in FP64 on the host (final poses)
static void pose_of_state(const double *st, double *R, double *p)
{
    const double *R0 = st, *p0 = st + 9, *an = st + 12, *u = st + 15, *w = st + 18;
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double a, b, sA;
    if (th < 1e-4) {
        double t2 = th * th;
        a = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
        b = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
        sA = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
    } else {
        a = (1.0 - cos(th)) / (th * th);
        b = (th - sin(th)) / (th * th * th);
        sA = sin(th) / th;
    }
    double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0}, K2[9], dR[9], V[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
    for (int k = 0; k < 9; ++k) {
        double I = (k % 4 == 0) ? 1.0 : 0.0;
        dR[k] = I + sA * K[k] + a * K2[k];
        V[k] = I + a * K[k] + b * K2[k];
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[3 * i + j] = dR[3 * i] * R0[j] + dR[3 * i + 1] * R0[3 + j] + dR[3 * i + 2] * R0[6 + j];
    double Ra[3], dRRa[3], Vu[3];
    for (int i = 0; i < 3; ++i) Ra[i] = R0[3 * i] * an[0] + R0[3 * i + 1] * an[1] + R0[3 * i + 2] * an[2];
    for (int i = 0; i < 3; ++i) dRRa[i] = dR[3 * i] * Ra[0] + dR[3 * i + 1] * Ra[1] + dR[3 * i + 2] * Ra[2];
    for (int i = 0; i < 3; ++i) Vu[i] = V[3 * i] * u[0] + V[3 * i + 1] * u[1] + V[3 * i + 2] * u[2];
    for (int i = 0; i < 3; ++i) p[i] = ((p0[i] + Vu[i]) + Ra[i]) - dRRa[i];
}

// Uploads the per-request tables of one refinement launch (staged copies:
// the host vectors may be released once the copies are issued).
static dock_status upload_refdev(dock_ctx *ctx, RefBufs &rb, const std::vector<RefineDev> &Ds,
                                 const std::vector<int32_t> &grp, cudaStream_t st)
{
    dock_status s;
    if ((s = ensure(ctx, (void **)&rb.dev, &rb.dev_n, Ds.size(), sizeof(RefineDev))) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&rb.grp, &rb.grp_n, std::max<size_t>(1, grp.size()), sizeof(int32_t))) != DOCK_OK)
        return s;
    CK(ctx, cudaMemcpyAsync(rb.dev, Ds.data(), sizeof(RefineDev) * Ds.size(), cudaMemcpyHostToDevice, st));
    if (!grp.empty())
        CK(ctx, cudaMemcpyAsync(rb.grp, grp.data(), sizeof(int32_t) * grp.size(), cudaMemcpyHostToDevice, st));
    return DOCK_OK;
}

// Runs `iters` projected Gauss-Newton iterations on the K states in
// rb.state, then a final evaluation that records J at the final twist.
static dock_status refine_loop(dock_ctx *ctx, RefBufs &rb, int K, int nblk, int iters, const dock_params *p,
                               cudaStream_t st)
{
    double prm[9] = {p->lambda, p->mu, p->step_t, p->step_r, p->b_t, p->b_r, p->lbfgs_pgtol, p->lbfgs_ftol,
                     (double)iters};
    CK(ctx, cudaMemcpyAsync(rb.prm, prm, sizeof(prm), cudaMemcpyHostToDevice, st));
    CandF *cf = (CandF *)rb.cands;
    dock_status s;
    if ((s = ensure(ctx, (void **)&rb.hint, &rb.hint_n, (size_t)K * nblk * 128, sizeof(int32_t))) != DOCK_OK) return s;
    CK(ctx, cudaMemsetAsync(rb.hint, 0xFF, sizeof(int32_t) * (size_t)K * nblk * 128, st));   // -1: no hint yet
    if (p->solver == DOCK_SOLVER_LBFGSB) {
        // L-BFGS-B (Sec. V-C as printed): rounds of one evaluation (J and
        // grad J at every active candidate's trial twist) and one solver
        // step; finished candidates skip the evaluation
        if ((s = ensure(ctx, (void **)&rb.lb, &rb.lb_n, (size_t)K * LB_ST, sizeof(double))) != DOCK_OK) return s;
        if ((s = ensure(ctx, (void **)&rb.active, &rb.active_n, (size_t)K, sizeof(int32_t))) != DOCK_OK) return s;
        CK(ctx, launch_lbfgs(K, nblk * REF_WARPS, rb.state, rb.acc, rb.prm, rb.lb, rb.active, cf, 0, st));
        for (int r = 0; r < p->lbfgs_evals; ++r) {
            {
                Prof pr(ctx, "refine_eval", st);
                CK(ctx, launch_refine_eval(rb.dev, rb.grp, K, nblk, cf, rb.acc, true, nullptr, nullptr, nullptr, st,
                                           rb.hint, rb.active));
            }
            Prof pr(ctx, "refine_lbfgs", st);
            CK(ctx, launch_lbfgs(K, nblk * REF_WARPS, rb.state, rb.acc, rb.prm, rb.lb, rb.active, cf, 1, st));
        }
        CK(ctx, launch_lbfgs(K, nblk * REF_WARPS, rb.state, rb.acc, rb.prm, rb.lb, rb.active, cf, 2, st));
        return DOCK_OK;
    }
    CK(ctx, launch_refine_solve(K, nblk * REF_WARPS, rb.state, rb.acc, rb.prm, 0, cf, st));
    for (int it = 0; it < iters; ++it) {
        {
            Prof pr(ctx, "refine_eval", st);
            CK(ctx, launch_refine_eval(rb.dev, rb.grp, K, nblk, cf, rb.acc, true, nullptr, nullptr, nullptr, st,
                                       rb.hint));
        }
        Prof pr(ctx, "refine_solve", st);
        CK(ctx, launch_refine_solve(K, nblk * REF_WARPS, rb.state, rb.acc, rb.prm, 1, cf, st));
    }
    {
        Prof pr(ctx, "refine_eval", st);
        CK(ctx, launch_refine_eval(rb.dev, rb.grp, K, nblk, cf, rb.acc, false, nullptr, nullptr, nullptr, st,
                                   rb.hint));
    }
    CK(ctx, launch_refine_solve(K, nblk * REF_WARPS, rb.state, rb.acc, rb.prm, 2, cf, st));
    return DOCK_OK;
}

// One group of candidates of one request: candidates [c0, c0 + K).
struct RefGroup {
    const dock_object *ob;
    const dock_sweep *sw;
    int c0, K;
};

static int refine_count(const std::vector<RefGroup> &groups)
{
    int K = 0;
    for (auto &gr : groups) K += gr.K;
    return K;
}

// Issues the refinement of the candidates of several requests (same
// parameters) on stream st, in shared launches; each candidate's arithmetic
// is the same as refined alone.  The final states (REF_ST doubles per
// candidate) are copied to host_state, which must stay valid (and, for the
// copy to be asynchronous, be pinned) until st reaches this point.
static dock_status refine_launch(dock_ctx *ctx, RefBufs &rb, const std::vector<RefGroup> &groups,
                                 const dock_candidate *in, const dock_params *p, cudaStream_t st, double *host_state)
{
    int K = refine_count(groups), nblk = 1;
    for (auto &gr : groups) nblk = std::max(nblk, ((int)gr.sw->P + 127) / 128);
    dock_status s;
    if ((s = ref_buffers(ctx, rb, K, nblk * REF_WARPS)) != DOCK_OK) return s;
    std::vector<double> sv((size_t)K * REF_ST);
    std::vector<RefineDev> Ds;
    std::vector<int32_t> grp(K);
    for (size_t g = 0; g < groups.size(); ++g) {
        const RefGroup &gr = groups[g];
        Ds.push_back(make_refine_dev(gr.ob, gr.sw, p));
        for (int c = gr.c0; c < gr.c0 + gr.K; ++c) {
            state_from_pose(in[c].q, in[c].t, gr.ob->anchor, sv.data() + (size_t)c * REF_ST);
            grp[c] = (int32_t)g;
        }
    }
    CK(ctx, cudaMemcpyAsync(rb.state, sv.data(), sizeof(double) * sv.size(), cudaMemcpyHostToDevice, st));
    if ((s = upload_refdev(ctx, rb, Ds, grp, st)) != DOCK_OK) return s;
    if ((s = refine_loop(ctx, rb, K, nblk, p->iters, p, st)) != DOCK_OK) return s;   // iters: the most L-BFGS-B steps
    CK(ctx, cudaMemcpyAsync(host_state, rb.state, sizeof(double) * sv.size(), cudaMemcpyDeviceToHost, st));
    return DOCK_OK;
}

// Poses, twists and J of refined candidates from their final states.
static void refine_results(const std::vector<RefGroup> &groups, const double *host_state, const dock_params *p,
                           dock_refined *out)
{
    for (auto &gr : groups)
        for (int c = gr.c0; c < gr.c0 + gr.K; ++c) {
            const double *x = host_state + (size_t)c * REF_ST;
            double R[9], t[3];
            pose_of_state(x, R, t);
            mat_to_quat(R, out[c].q);
            memcpy(out[c].t, t, sizeof(t));
            memcpy(out[c].xi, x + 15, sizeof(double) * 6);
            out[c].J = x[21];
            out[c].cand = c - gr.c0;
            out[c].iters = p->solver == DOCK_SOLVER_LBFGSB ? (int32_t)x[22] : p->iters;
        }
}

// Synchronous refinement on the context's own buffers and stream.
static dock_status refine_many(dock_ctx *ctx, const std::vector<RefGroup> &groups, const dock_candidate *in,
                               const dock_params *p, dock_refined *out)
{
    std::vector<double> hs((size_t)refine_count(groups) * REF_ST);
    dock_status s;
    if ((s = refine_launch(ctx, ctx->ref, groups, in, p, ctx->stream, hs.data())) != DOCK_OK) return s;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    refine_results(groups, hs.data(), p, out);
    return DOCK_OK;
}

static dock_status refine_impl(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw, const dock_candidate *in,
                               int K, const dock_params *p, dock_refined *out)
{
    std::vector<RefGroup> g(1, RefGroup{ob, sw, 0, K});
    return refine_many(ctx, g, in, p, out);
}

static dock_status check_quat_pose(dock_ctx *ctx, const double *q)
{
    for (int k = 0; k < 7; ++k) if (!isfinite(q[k])) return fail(ctx, DOCK_E_INVALID, "pose is not finite");
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(fabs(nq - 1.0) <= 1e-6)) return fail(ctx, DOCK_E_INVALID, "pose quaternion is not unit");
    return DOCK_OK;
}

static dock_status check_params(dock_ctx *ctx, const dock_params *p)
{
    if (p->iters < 0 || p->iters > 10000) return fail(ctx, DOCK_E_INVALID, "iters out of range");
    if (p->solver != DOCK_SOLVER_GAUSS_NEWTON && p->solver != DOCK_SOLVER_LBFGSB)
        return fail(ctx, DOCK_E_INVALID, "unknown solver %d", p->solver);
    if (p->solver == DOCK_SOLVER_LBFGSB &&
        (p->lbfgs_evals < 1 || p->lbfgs_evals > 10000 || !(p->lbfgs_pgtol >= 0.0) || !(p->lbfgs_ftol >= 0.0)))
        return fail(ctx, DOCK_E_INVALID, "L-BFGS-B limits out of range");
    return DOCK_OK;
}

extern "C" dock_status dock_refine_se3(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                       const dock_candidate *in, int32_t K, const dock_params *params,
                                       dock_refined *out)
{
    if (!ctx || !ob || !sw || !in || !out) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    if (K < 1 || K > 1024) return fail(ctx, DOCK_E_INVALID, "K must be in [1, 1024]");
    dock_status s;
    if ((s = check_pair(ctx, ob, sw)) != DOCK_OK) return s;
    dock_params pd;
    dock_params_default(&pd);
    const dock_params *p = params ? params : &pd;
    if ((s = check_params(ctx, p)) != DOCK_OK) return s;
    for (int c = 0; c < K; ++c) {
        double pose[7] = {in[c].q[0], in[c].q[1], in[c].q[2], in[c].q[3], in[c].t[0], in[c].t[1], in[c].t[2]};
        if ((s = check_quat_pose(ctx, pose)) != DOCK_OK) return s;
    }
    cudaSetDevice(ctx->device);
    return refine_impl(ctx, ob, sw, in, K, p, out);
}

static dock_status objective_impl(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw, const double *base,
                                  const float *xi, int B, const dock_params *params, float *J, float *grad,
                                  const float *gJ, void *stream)
{
    if (!ctx || !ob || !sw || !base || !xi || B < 1) return DOCK_E_INVALID;
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    dock_status s;
    if ((s = check_pair(ctx, ob, sw)) != DOCK_OK) return s;
    for (int b = 0; b < B; ++b)
        if ((s = check_quat_pose(ctx, base + 7 * b)) != DOCK_OK) return s;
    dock_params pd;
    dock_params_default(&pd);
    const dock_params *p = params ? params : &pd;
    cudaSetDevice(ctx->device);
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    int nblk = ((int)sw->P + 127) / 128;
    if ((s = ref_buffers(ctx, ctx->ref, B, nblk * REF_WARPS)) != DOCK_OK) return s;
    std::vector<double> stv((size_t)B * REF_ST);
    for (int b = 0; b < B; ++b) state_from_pose(base + 7 * b, base + 7 * b + 4, ob->anchor, stv.data() + (size_t)b * REF_ST);
    CK(ctx, cudaMemcpyAsync(ctx->ref.state, stv.data(), sizeof(double) * stv.size(), cudaMemcpyHostToDevice, st));
    std::vector<RefineDev> Ds(1, make_refine_dev(ob, sw, p));
    if ((s = upload_refdev(ctx, ctx->ref, Ds, std::vector<int32_t>(), st)) != DOCK_OK) return s;
    CK(ctx, cudaStreamSynchronize(st));   // the host staging vectors are released on return
    CK(ctx, launch_set_xi(B, xi, ctx->ref.state, st));
    CandF *cf = (CandF *)ctx->ref.cands;
    CK(ctx, launch_refine_solve(B, nblk * REF_WARPS, ctx->ref.state, ctx->ref.acc, ctx->ref.prm, 0, cf, st));
    {
        Prof pr(ctx, grad ? "objective_adjoint" : "objective_fwd");
        CK(ctx, launch_refine_eval(ctx->ref.dev, nullptr, B, nblk, cf, ctx->ref.acc, grad != nullptr, nullptr, nullptr,
                                   nullptr, st));
    }
    CK(ctx, launch_finish_objective(B, nblk * REF_WARPS, ctx->ref.state, ctx->ref.acc, p->lambda, J, grad, gJ, st));
    return DOCK_OK;
}

extern "C" dock_status dock_objective_fwd(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                          const double *base_poses, const float *xi, int32_t B,
                                          const dock_params *params, float *J, float *grad, void *stream)
{
    if (!ctx) return DOCK_E_INVALID;
    if (!J) return fail(ctx, DOCK_E_INVALID, "J output is required");
    DevLock dev_lock_(ctx);
    return objective_impl(ctx, ob, sw, base_poses, xi, B, params, J, grad, nullptr, stream);
}

extern "C" dock_status dock_objective_bwd(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                          const double *base_poses, const float *xi, int32_t B,
                                          const dock_params *params, const float *gJ, float *gxi, void *stream)
{
    if (!ctx) return DOCK_E_INVALID;
    if (!gJ || !gxi) return fail(ctx, DOCK_E_INVALID, "gJ and gxi are required");
    DevLock dev_lock_(ctx);
    return objective_impl(ctx, ob, sw, base_poses, xi, B, params, nullptr, gxi, gJ, stream);
}

extern "C" dock_status dock_distances(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                      const double *obj_poses, int32_t B, const dock_params *params, float *d,
                                      float *witness, float *normal)
{
    if (!ctx || !ob || !sw || !obj_poses || B < 1 || !d || !witness || !normal) return DOCK_E_INVALID;
    DevLock dev_lock_(ctx);
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    dock_status s;
    if ((s = check_pair(ctx, ob, sw)) != DOCK_OK) return s;
    dock_params pd;
    dock_params_default(&pd);
    const dock_params *p = params ? params : &pd;
    cudaSetDevice(ctx->device);
    int nblk = ((int)sw->P + 127) / 128;
    if ((s = ref_buffers(ctx, ctx->ref, B, nblk * REF_WARPS)) != DOCK_OK) return s;
    std::vector<double> stv((size_t)B * REF_ST);
    for (int b = 0; b < B; ++b) {
        if ((s = check_quat_pose(ctx, obj_poses + 7 * b)) != DOCK_OK) return s;
        state_from_pose(obj_poses + 7 * b, obj_poses + 7 * b + 4, ob->anchor, stv.data() + (size_t)b * REF_ST);
    }
    size_t n = (size_t)B * sw->P;
    float *buf = nullptr;
    if ((s = dalloc(ctx, (void **)&buf, sizeof(float) * 7 * n, nullptr)) != DOCK_OK) return s;
    cudaStream_t st = ctx->stream;
    CandF *cf = (CandF *)ctx->ref.cands;
    std::vector<RefineDev> Ds(1, make_refine_dev(ob, sw, p));
    if ((s = upload_refdev(ctx, ctx->ref, Ds, std::vector<int32_t>(), st)) != DOCK_OK) {
        dfree(ctx, buf, sizeof(float) * 7 * n);
        return s;
    }
    cudaError_t e = cudaMemcpyAsync(ctx->ref.state, stv.data(), sizeof(double) * stv.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_refine_solve(B, nblk * REF_WARPS, ctx->ref.state, ctx->ref.acc, ctx->ref.prm, 0, cf, st);
    if (e == cudaSuccess)
        e = launch_refine_eval(ctx->ref.dev, nullptr, B, nblk, cf, ctx->ref.acc, false, buf, buf + n, buf + 4 * n, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, buf, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(witness, buf + n, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(normal, buf + 4 * n, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(ctx, buf, sizeof(float) * 7 * n);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "distances");
    return DOCK_OK;
}

// ---------------------------------------------------------------------------
// registration engine: the three stages of Fig. 2 per request, with
// continuous batching across requests
//
// Every registration is a job that moves through the stages of Fig. 2: a
// global SF/Hopf search, a local GeoBall-SF search around the best global
// orientation (Sec. IV-C.2), and the refinement of the top-K candidates
// (Sec. V).  The engine runs in passes.  A pass picks one lattice side (round
// robin over the sides that have work), takes an equal share of rotations
// from every admitted job of that side, gathers their rotation records into
// one array and runs the four search kernels once over all of them.  Each
// record names its job's slot in the device request table, so every rotation
// is correlated with its own object, trajectory and probe, and its peak key
// lands in its own job's key array.  After a pass, jobs whose stage is
// complete move on (top-1 -> local samples; or top-K -> refinement ->
// result).  Queued jobs are admitted between passes while a slot is free and
// the HBM budget allows, so requests that arrive while others run join the
// next pass.  A job's arithmetic is the same whatever it is batched with.
// ---------------------------------------------------------------------------
constexpr int ENGINE_SLOTS = 64;   // jobs admitted at once
constexpr int ENGINE_MIN_SHARE = 16;
constexpr int PASS_BATCHES = 4;    // launch batches per pass (the voxeliser of one overlaps the FFT passes of another)

enum JobStage { JOB_QUEUED, JOB_GLOBAL, JOB_LOCAL, JOB_DONE };

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t ticket = 0;
    const dock_object *ob = nullptr;
    const dock_sweep *sw = nullptr;
    dock_register_desc d{};
    dock_params p{};
    int slot = -1;
    JobStage stage = JOB_QUEUED;
    int s0 = 0, s1 = 0, issued = 0;       // rotation range of the current stage, rotations sent
    std::vector<double> q;                // host quaternions: global, then local
    std::vector<dock_candidate> cands;    // top-K of the search stages
    void *dev = nullptr;                  // one device block: quaternions, records, keys, candidates
    size_t dev_bytes = 0;
    double *dq = nullptr;
    RotRec *drot = nullptr;
    unsigned long long *dkey = nullptr;
    dock_candidate *dcand = nullptr;
    dock_result res{};
    dock_status status = DOCK_PENDING;
    std::string err;
    bool cancel = false;
    bool async = false;                   // submitted by dock_submit (kept until polled)
    bool la = false;                      // label-aware score (the sweep's mode at submission)
    bool ro = false;                      // rotate the object (the sweep's mode at submission)
    Clock::time_point t_submit;
};
using JobP = std::shared_ptr<Job>;

struct Engine {
    std::mutex mu;                        // queue, tickets, job status, flags
    std::condition_variable cv_work, cv_done;
    std::deque<JobP> queue;
    std::vector<JobP> active;             // admitted jobs in admission order (engine thread only)
    std::map<uint64_t, JobP> tickets;     // submitted jobs until collected by dock_poll
    uint64_t next_ticket = 1;
    ReqDev *reqtab = nullptr;             // device request table, ENGINE_SLOTS entries
    std::vector<int> free_slots;
    int last_N = 0;
    int64_t passes = 0;                   // search passes run so far
    std::vector<JobP> refine_wait;        // searches done, refinement pending
    Clock::time_point refine_since;       // when the oldest of them finished its search
    cudaEvent_t pass_ev[2] = {nullptr, nullptr};   // completion of the last two passes
    // one refinement batch at a time runs on its own stream, beside the search
    // passes, with its own buffers and a pinned host copy of its final states
    cudaStream_t rstream = nullptr;
    cudaEvent_t rdone = nullptr;
    RefBufs rb;
    double *rhost = nullptr;
    size_t rhost_n = 0;
    bool rbusy = false;
    std::vector<JobP> rjobs;
    std::vector<RefGroup> rgroups;
    dock_params rparams{};
    std::thread worker;
    bool started = false, stop = false;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static dock_status check_job(dock_ctx *ctx, const Job &j)
{
    if (!j.ob || !j.sw) return fail(ctx, DOCK_E_INVALID, "request without object or sweep");
    dock_status s;
    if ((s = check_pair(ctx, j.ob, j.sw)) != DOCK_OK) return s;
    const dock_register_desc &d = j.d;
    if (d.n_global < 1 || d.n_local < 0 || d.top_k < 1 || d.top_k > 1024)
        return fail(ctx, DOCK_E_INVALID, "bad registration descriptor");
    if (d.sampler != DOCK_SAMPLER_SF && d.sampler != DOCK_SAMPLER_HOPF)
        return fail(ctx, DOCK_E_INVALID, "global sampler must be SF or HOPF");
    if (d.n_local > 0 && !(d.theta > 0.0 && d.theta < M_PI / 2)) return fail(ctx, DOCK_E_INVALID, "theta out of range");
    return check_params(ctx, &j.p);
}

static dock_status engine_init(dock_ctx *ctx)
{
    if (ctx->eng) return DOCK_OK;
    Engine *E = new (std::nothrow) Engine();
    if (!E) return fail(ctx, DOCK_E_NOMEM, "out of host memory");
    dock_status s = dalloc(ctx, (void **)&E->reqtab, sizeof(ReqDev) * ENGINE_SLOTS, nullptr);
    if (s != DOCK_OK) {
        delete E;
        return s;
    }
    for (auto &ev : E->pass_ev) {
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (auto &x : E->pass_ev) if (x) cudaEventDestroy(x);
            dfree(ctx, E->reqtab, sizeof(ReqDev) * ENGINE_SLOTS);
            delete E;
            return cuda_fail(ctx, e, "cudaEventCreate");
        }
    }
    cudaError_t e = cudaStreamCreateWithFlags(&E->rstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&E->rdone, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (E->rstream) cudaStreamDestroy(E->rstream);
        for (auto &x : E->pass_ev) if (x) cudaEventDestroy(x);
        dfree(ctx, E->reqtab, sizeof(ReqDev) * ENGINE_SLOTS);
        delete E;
        return cuda_fail(ctx, e, "creating the refinement stream");
    }
    for (int i = ENGINE_SLOTS - 1; i >= 0; --i) E->free_slots.push_back(i);
    ctx->eng = E;
    return DOCK_OK;
}

static size_t job_bytes(const Job &j)
{
    size_t n = (size_t)j.d.n_global + j.d.n_local;
    return align256(n * 4 * sizeof(double)) + align256(n * sizeof(RotRec)) + align256(n * sizeof(unsigned long long)) +
           align256((size_t)j.d.top_k * sizeof(dock_candidate));
}

// Device bytes the Y/Z scratch must grow by for a pass at lattice side N.
static size_t yz_growth(dock_ctx *ctx, const dock_sweep *sw, bool la)
{
    Geo g = make_geo(sw);
    size_t need = (size_t)tuning_for(ctx, g).batch * (g.N + g.M + (la ? g.N : 0)) * g.M * g.P;
    return need > ctx->yz_bytes ? (need - ctx->yz_bytes) * sizeof(float2) : 0;
}

static void job_release(dock_ctx *ctx, Engine &E, Job &j)
{
    if (j.dev) {
        dfree(ctx, j.dev, j.dev_bytes);
        j.dev = nullptr;
    }
    if (j.slot >= 0) {
        E.free_slots.push_back(j.slot);
        j.slot = -1;
    }
}

static void job_finish(dock_ctx *ctx, Engine &E, const JobP &j, dock_status st)
{
    job_release(ctx, E, *j);
    if (st != DOCK_OK) j->err = ctx->err;
    j->res.latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - j->t_submit).count();
    std::lock_guard<std::mutex> lk(E.mu);
    j->stage = JOB_DONE;
    j->status = st;
    E.cv_done.notify_all();
}

enum { ADMIT_OK = 0, ADMIT_WAIT = 1 };

// Allocate the job's device block, draw its global samples and set up their
// rotation records; the job's slot in the request table points at its
// object spectrum, trajectory and key array.
static dock_status job_admit(dock_ctx *ctx, Engine &E, Job &j, int *wait)
{
    *wait = ADMIT_OK;
    const size_t bytes = job_bytes(j);
    const bool la = j.la && j.sw->poses_lab;
    size_t pen_bytes = la && !j.ob->spec_pen ? sizeof(float2) * (size_t)j.ob->M * j.ob->P * j.ob->M : 0;
    if (j.ro && !j.sw->spec_S) pen_bytes += sizeof(float2) * (size_t)j.ob->M * j.ob->P * j.ob->M;
    if (j.ro && !j.ob->cells) pen_bytes += sizeof(float4) * (size_t)(j.ob->N + 1) * (j.ob->N + 1) * (j.ob->N + 1);
    if (j.ro) {   // the rotated object grids of a launch, if not held yet
        const Geo gj = make_geo(j.sw);
        const size_t need = (size_t)tuning_for(ctx, gj).batch * gj.N * gj.N * gj.N;
        if (need > ctx->ogr_n) pen_bytes += sizeof(float) * need;
    }
    if (ctx->budget && ctx->held + bytes + pen_bytes + yz_growth(ctx, j.sw, la) > ctx->budget) {
        if (!E.active.empty()) {
            *wait = ADMIT_WAIT;
            return DOCK_OK;
        }
        return fail(ctx, DOCK_E_TOO_LARGE, "request needs %zu bytes beyond the HBM budget", bytes);
    }
    dock_status s;
    if (la && (s = ensure_spec_pen(ctx, j.ob)) != DOCK_OK) return s;
    if (j.ro && ((s = ensure_spec_S(ctx, j.sw)) != DOCK_OK || (s = ensure_cells(ctx, j.ob)) != DOCK_OK)) return s;
    if ((s = dalloc(ctx, &j.dev, bytes, nullptr)) != DOCK_OK) return s;
    j.dev_bytes = bytes;
    const size_t n = (size_t)j.d.n_global + j.d.n_local;
    unsigned char *b = (unsigned char *)j.dev;
    j.dq = (double *)b;
    b += align256(n * 4 * sizeof(double));
    j.drot = (RotRec *)b;
    b += align256(n * sizeof(RotRec));
    j.dkey = (unsigned long long *)b;
    b += align256(n * sizeof(unsigned long long));
    j.dcand = (dock_candidate *)b;
    j.slot = E.free_slots.back();
    E.free_slots.pop_back();
    dock_search_desc d = {};
    d.sampler = j.d.sampler;
    d.n = j.d.n_global;
    d.top_k = 1;
    std::vector<double> qg;
    if ((s = gen_samples(ctx, &d, qg)) != DOCK_OK) return s;
    j.q.assign(4 * n, 0.0);
    memcpy(j.q.data(), qg.data(), sizeof(double) * qg.size());
    CK(ctx, cudaMemcpyAsync(j.dq, j.q.data(), sizeof(double) * 4 * j.d.n_global, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, launch_rot_setup(j.dq, j.d.n_global, 0, j.slot, j.sw->cs_dev, j.sw->h, j.sw->N, j.drot, ctx->stream,
                             j.ro ? j.ob->o_dev : nullptr));
    CK(ctx, cudaMemsetAsync(j.dkey, 0, sizeof(unsigned long long) * n, ctx->stream));
    ReqDev r = make_reqdev(j.ob, j.sw, j.dkey, la, j.ro);
    CK(ctx, cudaMemcpyAsync(E.reqtab + j.slot, &r, sizeof(ReqDev), cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));   // r and j.q are host staging of this call
    j.stage = JOB_GLOBAL;
    j.s0 = 0;
    j.s1 = j.d.n_global;
    j.issued = 0;
    return DOCK_OK;
}

// The job's stage is complete: start the local search around the best
// global orientation, or take its top-K candidates (*final set; the
// refinement runs afterwards, batched with other jobs finishing in the same
// pass).
// Synchronises the context stream and reads (and clears) the device error
// word that kernels set when they give up (e.g. a bounded wait that ran out).
static dock_status take_device_error(dock_ctx *ctx)
{
    int herr = 0;
    CK(ctx, cudaMemcpyAsync(&herr, ctx->errflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (!herr) return DOCK_OK;
    CK(ctx, cudaMemsetAsync(ctx->errflag, 0, sizeof(int), ctx->stream));
    return fail(ctx, herr, "device reported error %d during a search pass", herr);
}

static dock_status job_advance(dock_ctx *ctx, Job &j, bool *final)
{
    *final = false;
    dock_status s;
    const dock_object *ob = j.ob;
    const int ng = j.d.n_global, nl = j.d.n_local;
    if (j.stage == JOB_GLOBAL && nl > 0) {
        {
            Prof pr(ctx, "topk");
            CK(ctx, launch_topk(j.dkey, ng, 1, ob->N, ob->M, ob->h, ob->o_dev, j.dq, j.drot, j.dcand, ctx->stream,
                                j.ro ? j.sw->os_dev : nullptr));
        }
        dock_candidate best;
        CK(ctx, cudaMemcpyAsync(&best, j.dcand, sizeof(best), cudaMemcpyDeviceToHost, ctx->stream));
        if ((s = take_device_error(ctx)) != DOCK_OK) return s;
        dock_search_desc dl = {};
        dl.sampler = DOCK_SAMPLER_GEOBALL;
        dl.n = nl;
        memcpy(dl.q0, best.q, sizeof(dl.q0));
        dl.theta = j.d.theta;
        std::vector<double> ql;
        if ((s = gen_samples(ctx, &dl, ql)) != DOCK_OK) return s;
        memcpy(j.q.data() + 4 * (size_t)ng, ql.data(), sizeof(double) * ql.size());
        CK(ctx, cudaMemcpyAsync(j.dq + 4 * (size_t)ng, j.q.data() + 4 * (size_t)ng, sizeof(double) * 4 * nl,
                                cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, launch_rot_setup(j.dq + 4 * (size_t)ng, nl, ng, j.slot, j.sw->cs_dev, j.sw->h, j.sw->N, j.drot + ng,
                                 ctx->stream, j.ro ? ob->o_dev : nullptr));
        j.stage = JOB_LOCAL;
        j.s0 = ng;
        j.s1 = ng + nl;
        j.issued = 0;
        return DOCK_OK;
    }
    const int n = ng + nl, K = j.d.top_k;
    {
        Prof pr(ctx, "topk");
        CK(ctx, launch_topk(j.dkey, n, K, ob->N, ob->M, ob->h, ob->o_dev, j.dq, j.drot, j.dcand, ctx->stream,
                            j.ro ? j.sw->os_dev : nullptr));
    }
    j.cands.assign(K, dock_candidate());
    CK(ctx, cudaMemcpyAsync(j.cands.data(), j.dcand, sizeof(dock_candidate) * K, cudaMemcpyDeviceToHost, ctx->stream));
    if ((s = take_device_error(ctx)) != DOCK_OK) return s;
    int Kv = 0;
    while (Kv < K && j.cands[Kv].rot >= 0) ++Kv;
    if (Kv == 0) return fail(ctx, DOCK_E_INVALID, "the search produced no candidate");
    j.cands.resize(Kv);
    *final = true;
    return DOCK_OK;
}

// Results of the refinement batch in flight once its stream has finished
// it: the lowest J of a job's candidates wins (ties: lower candidate index).
static void engine_refine_collect(dock_ctx *ctx, Engine &E, bool wait)
{
    if (!E.rbusy) return;
    cudaError_t e = wait ? cudaEventSynchronize(E.rdone) : cudaEventQuery(E.rdone);
    if (e == cudaErrorNotReady) return;
    E.rbusy = false;
    std::vector<JobP> jobs;
    jobs.swap(E.rjobs);
    if (e != cudaSuccess) {
        dock_status s = cuda_fail(ctx, e, "refinement");
        for (auto &jp : jobs)
            if (jp->stage != JOB_DONE) job_finish(ctx, E, jp, s);
    } else {
        std::vector<dock_refined> ref(refine_count(E.rgroups));
        refine_results(E.rgroups, E.rhost, &E.rparams, ref.data());
        for (size_t g = 0; g < jobs.size(); ++g) {
            const JobP &jp = jobs[g];
            if (jp->stage == JOB_DONE) continue;   // cancelled meanwhile
            Job &j = *jp;
            const dock_refined *r = ref.data() + E.rgroups[g].c0;
            int bi = 0;
            for (int c = 1; c < E.rgroups[g].K; ++c) if (r[c].J < r[bi].J) bi = c;
            memcpy(j.res.q, r[bi].q, sizeof(j.res.q));
            memcpy(j.res.t, r[bi].t, sizeof(j.res.t));
            j.res.J = r[bi].J;
            j.res.best_cand = bi;
            j.res.n_evals = j.d.n_global + j.d.n_local;
            j.res.best_search = j.cands[0];
            job_finish(ctx, E, jp, DOCK_OK);
        }
    }
    E.rgroups.clear();
    E.active.erase(std::remove_if(E.active.begin(), E.active.end(),
                                  [](const JobP &j) { return j->stage == JOB_DONE; }),
                   E.active.end());
}

// Refinements of several requests share launches, which a single request's
// few candidates cannot fill.  Finished searches wait (in admission order)
// until 16 of them are ready, no search work is left, or the oldest has
// waited 50 ms; the batch (the waiting jobs with the first one's parameters)
// then runs on the refinement stream while search passes go on.
constexpr size_t ENGINE_REFINE_BATCH = 16;
constexpr double ENGINE_REFINE_WAIT_MS = 50.0;

static void engine_refine_now(dock_ctx *ctx, Engine &E)
{
    if (E.rbusy) return;
    std::vector<JobP> batch, rest;
    for (auto &j : E.refine_wait) {
        if (j->stage == JOB_DONE) continue;   // an error may have ended some meanwhile
        if (batch.empty() || memcmp(&j->p, &batch[0]->p, sizeof(dock_params)) == 0) batch.push_back(j);
        else rest.push_back(j);
    }
    E.refine_wait.swap(rest);
    if (!E.refine_wait.empty()) E.refine_since = Clock::now();
    if (batch.empty()) return;
    std::vector<RefGroup> groups;
    std::vector<dock_candidate> cands;
    for (auto &jp : batch) {
        groups.push_back(RefGroup{jp->ob, jp->sw, (int)cands.size(), (int)jp->cands.size()});
        cands.insert(cands.end(), jp->cands.begin(), jp->cands.end());
    }
    const size_t need = cands.size() * REF_ST;
    dock_status s = DOCK_OK;
    if (need > E.rhost_n) {
        if (E.rhost) cudaFreeHost(E.rhost);
        E.rhost = nullptr;
        E.rhost_n = 0;
        cudaError_t e = cudaMallocHost((void **)&E.rhost, need * sizeof(double));
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "pinned host buffer for the refinement");
        else E.rhost_n = need;
    }
    if (s == DOCK_OK) s = refine_launch(ctx, E.rb, groups, cands.data(), &batch[0]->p, E.rstream, E.rhost);
    if (s == DOCK_OK) {
        cudaError_t e = cudaEventRecord(E.rdone, E.rstream);
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "recording the refinement");
    }
    if (s != DOCK_OK) {
        cudaStreamSynchronize(E.rstream);
        for (auto &jp : batch) job_finish(ctx, E, jp, s);
        E.active.erase(std::remove_if(E.active.begin(), E.active.end(),
                                      [](const JobP &j) { return j->stage == JOB_DONE; }),
                       E.active.end());
        return;
    }
    E.rbusy = true;
    E.rjobs = batch;
    E.rgroups = groups;
    E.rparams = batch[0]->p;
}

static void engine_refine_if_due(dock_ctx *ctx, Engine &E)
{
    if (E.refine_wait.empty()) return;
    bool search_left = false;
    for (auto &j : E.active)
        if (j->stage != JOB_DONE && j->issued < j->s1 - j->s0) search_left = true;
    {
        std::lock_guard<std::mutex> lk(E.mu);
        if (!E.queue.empty()) search_left = true;
    }
    const double waited = std::chrono::duration<double, std::milli>(Clock::now() - E.refine_since).count();
    if (!search_left || E.refine_wait.size() >= ENGINE_REFINE_BATCH || waited >= ENGINE_REFINE_WAIT_MS)
        engine_refine_now(ctx, E);
}

// One engine step: admissions, then one search pass.  Returns false when
// there was nothing to run.  Caller holds ctx->dev_mu.
static bool engine_step(dock_ctx *ctx)
{
    Engine &E = *ctx->eng;
    // cancelled jobs leave between passes
    E.refine_wait.erase(std::remove_if(E.refine_wait.begin(), E.refine_wait.end(),
                                       [](const JobP &j) { return j->cancel; }),
                        E.refine_wait.end());
    for (size_t i = 0; i < E.active.size();) {
        if (E.active[i]->cancel) {
            fail(ctx, DOCK_E_CANCELLED, "request cancelled");
            job_finish(ctx, E, E.active[i], DOCK_E_CANCELLED);
            E.active.erase(E.active.begin() + i);
        } else {
            ++i;
        }
    }
    engine_refine_collect(ctx, E, false);
    bool did = false;
    for (;;) {
        JobP j;
        {
            std::lock_guard<std::mutex> lk(E.mu);
            if (E.queue.empty() || E.free_slots.empty()) break;
            j = E.queue.front();
            if (j->cancel) E.queue.pop_front();
        }
        if (j->cancel) {
            fail(ctx, DOCK_E_CANCELLED, "request cancelled");
            job_finish(ctx, E, j, DOCK_E_CANCELLED);
            continue;
        }
        int wait = ADMIT_OK;
        dock_status s = job_admit(ctx, E, *j, &wait);
        if (s == DOCK_OK && wait == ADMIT_WAIT) break;
        {
            std::lock_guard<std::mutex> lk(E.mu);
            E.queue.pop_front();
        }
        did = true;
        if (s != DOCK_OK) {
            job_finish(ctx, E, j, s);
            if (ctx->dead) break;
            continue;
        }
        E.active.push_back(j);
    }
    if (ctx->dead) {
        for (auto &j : E.active) job_finish(ctx, E, j, DOCK_E_CUDA_FATAL);
        E.active.clear();
        E.refine_wait.clear();
        return did;
    }
    // lattice side of this pass: round robin over the sides with work
    int pick = 0;
    for (auto &j : E.active) {
        if (j->issued >= j->s1 - j->s0) continue;
        int N = j->ob->N;
        if (N > E.last_N && (pick == 0 || N < pick)) pick = N;
    }
    if (pick == 0)
        for (auto &j : E.active)
            if (j->issued < j->s1 - j->s0 && (pick == 0 || j->ob->N < pick)) pick = j->ob->N;
    if (pick == 0) {
        // no search work: finish the refinement in flight, refine whatever waits
        if (E.rbusy) {
            engine_refine_collect(ctx, E, true);
            return true;
        }
        if (!E.refine_wait.empty()) {
            engine_refine_now(ctx, E);
            return true;
        }
        return did;
    }
    E.last_N = pick;
    std::vector<Job *> cls;
    for (auto &j : E.active)
        if (j->ob->N == pick && j->issued < j->s1 - j->s0) cls.push_back(j.get());
    const Geo g = make_geo(cls[0]->sw);
    const int B1 = tuning_for(ctx, g).batch;   // rotations per launch
    const int B = B1 * PASS_BATCHES;           // rotations per pass
    dock_status s;
    if ((s = ensure(ctx, (void **)&ctx->phase, &ctx->phase_n, (size_t)B, sizeof(RotRec))) != DOCK_OK) {
        for (auto &j : E.active)
            if (j->ob->N == pick) job_finish(ctx, E, j, s);
        E.active.erase(std::remove_if(E.active.begin(), E.active.end(),
                                      [&](const JobP &j) { return j->stage == JOB_DONE; }),
                       E.active.end());
        return true;
    }
    // At most two passes in flight: without this bound the host would queue
    // every pass of a long request at once, and requests arriving meanwhile
    // would only start after all of them.
    if (E.passes >= 2) {
        cudaError_t e = cudaEventSynchronize(E.pass_ev[E.passes % 2]);
        if (e != cudaSuccess) {
            s = cuda_fail(ctx, e, "waiting for a search pass");
            for (auto &j : E.active) job_finish(ctx, E, j, s);
            E.active.clear();
            E.refine_wait.clear();
            return true;
        }
    }
    // equal shares, then whatever is left in admission order
    const int share = std::max(ENGINE_MIN_SHARE, B / (int)cls.size());
    int taken = 0;
    std::vector<Job *> in_pass;
    cudaError_t ce = cudaSuccess;
    for (int round = 0; round < 2 && taken < B && ce == cudaSuccess; ++round)
        for (auto *jp : cls) {
            int rem = jp->s1 - jp->s0 - jp->issued;
            int take = std::min(rem, B - taken);
            if (round == 0) take = std::min(take, share);
            if (take <= 0) continue;
            ce = cudaMemcpyAsync(ctx->phase + taken, jp->drot + jp->s0 + jp->issued, sizeof(RotRec) * take,
                                 cudaMemcpyDeviceToDevice, ctx->stream);
            if (ce != cudaSuccess) break;
            jp->issued += take;
            taken += take;
            if (jp->res.first_pass < 0) jp->res.first_pass = E.passes;
            jp->res.last_pass = E.passes;
            if (std::find(in_pass.begin(), in_pass.end(), jp) == in_pass.end()) in_pass.push_back(jp);
            if (taken == B) break;
        }
    bool dual = false, ro_any = false;
    for (auto *jp : in_pass) {
        dual = dual || (jp->la && jp->sw->poses_lab);
        ro_any = ro_any || jp->ro;
    }
    if (ce != cudaSuccess) s = cuda_fail(ctx, ce, "gather of rotation records");
    else s = run_pipeline_rots(ctx, g, E.reqtab, ctx->phase, 0, taken, B1, dual, ro_any);
    if (s == DOCK_OK) {
        cudaError_t e = cudaEventRecord(E.pass_ev[E.passes % 2], ctx->stream);
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "recording a search pass");
    }
    ++E.passes;
    std::vector<JobP> &finals = E.refine_wait;
    for (auto *jp : in_pass) {
        JobP j;
        for (auto &x : E.active)
            if (x.get() == jp) j = x;
        if (s != DOCK_OK) {
            job_finish(ctx, E, j, s);
            continue;
        }
        if (jp->issued < jp->s1 - jp->s0) continue;
        bool final = false;
        dock_status sa = job_advance(ctx, *jp, &final);
        if (sa != DOCK_OK) job_finish(ctx, E, j, sa);
        else if (final) {
            finals.push_back(j);
            if (finals.size() == 1) E.refine_since = Clock::now();
        }
    }
    engine_refine_if_due(ctx, E);
    E.active.erase(std::remove_if(E.active.begin(), E.active.end(),
                                  [](const JobP &j) { return j->stage == JOB_DONE; }),
                   E.active.end());
    return true;
}

static void engine_worker(dock_ctx *ctx)
{
    Engine &E = *ctx->eng;
    cudaSetDevice(ctx->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(E.mu);
            E.cv_work.wait(lk, [&] { return E.stop || !E.queue.empty() || !E.active.empty(); });
            if (E.stop) break;
        }
        // let waiting API calls in first (bounded: 100 ms)
        for (int k = 0; k < 2000 && ctx->dev_want.load() > 0; ++k)
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        bool did;
        {
            std::lock_guard<std::recursive_mutex> dl(ctx->dev_mu);
            did = engine_step(ctx);
        }
        if (!did) {
            // queued jobs wait for memory held by nothing that will free it soon
            std::unique_lock<std::mutex> lk(E.mu);
            E.cv_work.wait_for(lk, std::chrono::milliseconds(1));
        }
    }
}

static void engine_shutdown(dock_ctx *ctx)
{
    Engine *E = ctx->eng;
    if (!E) return;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        E->stop = true;
        E->cv_work.notify_all();
    }
    if (E->worker.joinable()) E->worker.join();
    if (E->rbusy) cudaStreamSynchronize(E->rstream);   // its jobs end cancelled below
    fail(ctx, DOCK_E_CANCELLED, "context destroyed");
    for (auto &j : E->active) job_finish(ctx, *E, j, DOCK_E_CANCELLED);
    std::deque<JobP> q;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        q.swap(E->queue);
    }
    for (auto &j : q) job_finish(ctx, *E, j, DOCK_E_CANCELLED);
    dfree(ctx, E->reqtab, sizeof(ReqDev) * ENGINE_SLOTS);
    for (auto &ev : E->pass_ev) if (ev) cudaEventDestroy(ev);
    if (E->rstream) {
        cudaStreamSynchronize(E->rstream);
        cudaStreamDestroy(E->rstream);
    }
    if (E->rdone) cudaEventDestroy(E->rdone);
    if (E->rhost) cudaFreeHost(E->rhost);
    free_refbufs(E->rb);
    delete E;
    ctx->eng = nullptr;
}

// Requests that use a handle being freed are cancelled first (caller holds
// ctx->dev_mu, so no pass is in flight).
static void engine_drop_handle(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw)
{
    Engine *E = ctx->eng;
    if (!E) return;
    engine_refine_collect(ctx, *E, true);   // the batch in flight may read the handle
    auto uses = [&](const JobP &j) { return (ob && j->ob == ob) || (sw && j->sw == sw); };
    std::vector<JobP> drop;
    {
        std::lock_guard<std::mutex> lk(E->mu);
        for (auto it = E->queue.begin(); it != E->queue.end();) {
            if (uses(*it)) {
                drop.push_back(*it);
                it = E->queue.erase(it);
            } else {
                ++it;
            }
        }
    }
    for (auto &j : E->active)
        if (uses(j)) drop.push_back(j);
    E->refine_wait.erase(std::remove_if(E->refine_wait.begin(), E->refine_wait.end(), uses), E->refine_wait.end());
    if (drop.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    fail(ctx, DOCK_E_CANCELLED, "a handle of the request was freed");
    for (auto &j : drop) job_finish(ctx, *E, j, DOCK_E_CANCELLED);
    E->active.erase(std::remove_if(E->active.begin(), E->active.end(),
                                   [](const JobP &j) { return j->stage == JOB_DONE; }),
                    E->active.end());
}

// Run jobs to completion from the calling thread (or let the serving worker
// run them when it is active) and return the first error, if any.
static dock_status run_jobs(dock_ctx *ctx, std::vector<JobP> &js)
{
    for (auto &j : js)
        if (dock_status s = check_job(ctx, *j)) return s;
    dock_status s;
    if (!ctx->eng_ready.load()) {
        DevLock dl(ctx);
        if ((s = engine_init(ctx)) != DOCK_OK) return s;
        ctx->eng_ready.store(true);
    }
    Engine &E = *ctx->eng;
    bool threaded;
    {
        std::lock_guard<std::mutex> lk(E.mu);
        for (auto &j : js) {
            j->t_submit = Clock::now();
            E.queue.push_back(j);
        }
        threaded = E.started;
        E.cv_work.notify_all();
    }
    auto all_done = [&] {
        for (auto &j : js)
            if (j->stage != JOB_DONE) return false;
        return true;
    };
    if (threaded) {
        std::unique_lock<std::mutex> lk(E.mu);
        E.cv_done.wait(lk, all_done);
    } else {
        DevLock dl(ctx);
        for (;;) {
            {
                std::lock_guard<std::mutex> lk(E.mu);
                if (all_done()) break;
            }
            if (!engine_step(ctx)) {
                // nothing could run: a queued job waits for memory no active job holds
                std::lock_guard<std::mutex> lk(E.mu);
                if (!all_done() && E.active.empty()) break;
            }
        }
    }
    for (auto &j : js)
        if (j->status != DOCK_OK) {
            if (j->status == DOCK_PENDING) return fail(ctx, DOCK_E_TOO_LARGE, "request could not be admitted");
            fail(ctx, j->status, "%s", j->err.c_str());
            return j->status;
        }
    return DOCK_OK;
}

static JobP make_job(const dock_object *ob, const dock_sweep *sw, const dock_register_desc *rd, const dock_params *params)
{
    JobP j = std::make_shared<Job>();
    j->res.first_pass = -1;
    j->res.last_pass = -1;
    j->ob = ob;
    j->sw = sw;
    const int mode = sw ? sw->mode.load() : 0;   // one read: the two options are exclusive
    j->la = (mode & SCORE_LABEL_AWARE) != 0;
    j->ro = (mode & SCORE_ROTATE_OBJECT) != 0;
    j->d = *rd;
    if (params) j->p = *params;
    else dock_params_default(&j->p);
    return j;
}

extern "C" dock_status dock_register(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                     const dock_register_desc *rd, const dock_params *params, dock_result *out)
{
    if (!ctx || !ob || !sw || !rd || !out) return DOCK_E_INVALID;
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    cudaSetDevice(ctx->device);
    std::vector<JobP> js(1, make_job(ob, sw, rd, params));
    dock_status s = run_jobs(ctx, js);
    if (s == DOCK_OK) *out = js[0]->res;
    return s;
}

extern "C" dock_status dock_register_batch(dock_ctx *ctx, const dock_request *reqs, int32_t n, const dock_params *params,
                                           dock_result *out)
{
    if (!ctx || !reqs || !out || n < 1) return DOCK_E_INVALID;
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    cudaSetDevice(ctx->device);
    std::vector<JobP> js;
    for (int i = 0; i < n; ++i) js.push_back(make_job(reqs[i].obj, reqs[i].sweep, &reqs[i].desc, params));
    dock_status s = run_jobs(ctx, js);
    if (s == DOCK_OK)
        for (int i = 0; i < n; ++i) out[i] = js[i]->res;
    return s;
}

extern "C" dock_status dock_submit(dock_ctx *ctx, const dock_request *req, const dock_params *params, uint64_t *ticket)
{
    if (!ctx || !req || !ticket) return DOCK_E_INVALID;
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    JobP j = make_job(req->obj, req->sweep, &req->desc, params);
    dock_status s;
    if ((s = check_job(ctx, *j)) != DOCK_OK) return s;
    if (!ctx->eng_ready.load()) {
        DevLock dl(ctx);
        cudaSetDevice(ctx->device);
        if ((s = engine_init(ctx)) != DOCK_OK) return s;
        ctx->eng_ready.store(true);
    }
    Engine &E = *ctx->eng;
    std::lock_guard<std::mutex> lk(E.mu);
    if (!E.started) {
        try {
            E.worker = std::thread(engine_worker, ctx);
        } catch (...) {
            return fail(ctx, DOCK_E_NOMEM, "cannot start the serving thread");
        }
        E.started = true;
    }
    j->async = true;
    j->ticket = E.next_ticket++;
    j->t_submit = Clock::now();
    E.tickets[j->ticket] = j;
    E.queue.push_back(j);
    E.cv_work.notify_all();
    *ticket = j->ticket;
    return DOCK_OK;
}

extern "C" dock_status dock_poll(dock_ctx *ctx, uint64_t ticket, dock_result *out, int64_t timeout_us)
{
    if (!ctx || !out) return DOCK_E_INVALID;
    if (!ctx->eng) return fail(ctx, DOCK_E_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    Engine &E = *ctx->eng;
    std::unique_lock<std::mutex> lk(E.mu);
    auto it = E.tickets.find(ticket);
    if (it == E.tickets.end()) return fail(ctx, DOCK_E_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    JobP j = it->second;
    auto done = [&] { return j->stage == JOB_DONE; };
    if (!done()) {
        if (timeout_us < 0) E.cv_done.wait(lk, done);
        else if (timeout_us > 0) E.cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done);
    }
    if (!done()) return DOCK_PENDING;
    E.tickets.erase(it);
    if (j->status != DOCK_OK) {
        lk.unlock();
        fail(ctx, j->status, "%s", j->err.c_str());
        return j->status;
    }
    *out = j->res;
    return DOCK_OK;
}

extern "C" dock_status dock_cancel(dock_ctx *ctx, uint64_t ticket)
{
    if (!ctx) return DOCK_E_INVALID;
    if (!ctx->eng) return fail(ctx, DOCK_E_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    Engine &E = *ctx->eng;
    std::lock_guard<std::mutex> lk(E.mu);
    auto it = E.tickets.find(ticket);
    if (it == E.tickets.end()) return fail(ctx, DOCK_E_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    it->second->cancel = true;
    E.cv_work.notify_all();
    return DOCK_OK;
}
