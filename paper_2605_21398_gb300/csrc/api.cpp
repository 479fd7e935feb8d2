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
#include <chrono>
#include <mutex>
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

struct dock_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;        // 0 = unbounded
    size_t held = 0;          // bytes currently held by this context and its handles
    std::string err;
    bool dead = false;
    // search scratch (grown on demand)
    float2 *Y = nullptr, *Z = nullptr;
    size_t yz_bytes = 0;
    uint32_t *bits = nullptr;
    size_t bits_n = 0;
    unsigned long long *keys = nullptr;
    size_t keys_n = 0;
    RotRec *rots = nullptr;
    size_t rots_n = 0;
    double *quats = nullptr;
    size_t quats_n = 0;
    int *errflag = nullptr;
    dock_candidate *cands = nullptr;
    size_t cands_n = 0;
    // refinement buffers
    double *ref_state = nullptr, *ref_acc = nullptr, *ref_prm = nullptr;
    size_t ref_state_n = 0, ref_acc_n = 0, ref_prm_n = 0;
    void *ref_cands = nullptr;
    size_t ref_cands_n = 0;
    // twiddle tables per canvas size
    std::map<int, float2 *> tw, qt;
    std::map<int, double2 *> twd;
    // profiling
    bool prof = false;
    std::vector<ProfEntry> pending;
    std::map<std::string, KStat> stats;
    std::vector<cudaEvent_t> ev_pool;
};

struct dock_object {
    dock_ctx *ctx;
    int N, M, P;
    double h;
    double o[3];
    double anchor[3];
    float *O = nullptr;       // N^3
    float2 *spec = nullptr;   // tiled conj(F(O)) / M^3
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
};

static dock_status fail(dock_ctx *ctx, dock_status st, const char *fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
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
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, DOCK_E_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    ctx->held += bytes;
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
    cudaEvent_t a = nullptr, b = nullptr;
    Prof(dock_ctx *c, const char *n) : ctx(c), name(n)
    {
        if (!ctx->prof) return;
        a = get();
        b = get();
        cudaEventRecord(a, ctx->stream);
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
        cudaEventRecord(b, ctx->stream);
        ctx->pending.push_back({name, a, b});
    }
};

static void prof_resolve(dock_ctx *ctx)
{
    if (ctx->pending.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &p : ctx->pending) {
        float ms = 0.f;
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
    p->tri_iters = 24;
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
    *out = c;
    return DOCK_OK;
}

void dock_destroy(dock_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->Y);
    cudaFree(c->bits);
    cudaFree(c->keys);
    cudaFree(c->rots);
    cudaFree(c->quats);
    cudaFree(c->errflag);
    cudaFree(c->cands);
    cudaFree(c->ref_state);
    cudaFree(c->ref_acc);
    cudaFree(c->ref_prm);
    cudaFree(c->ref_cands);
    for (auto &kv : c->tw) cudaFree(kv.second);
    for (auto &kv : c->qt) cudaFree(kv.second);
    for (auto &kv : c->twd) cudaFree(kv.second);
    for (auto &p : c->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *dock_last_error(const dock_ctx *c) { return c ? c->err.c_str() : "null context"; }

dock_status dock_set_profiling(dock_ctx *c, int enable)
{
    if (!c) return DOCK_E_INVALID;
    if (!enable) prof_resolve(c);
    c->prof = enable != 0;
    return DOCK_OK;
}

int32_t dock_get_kernel_stats(dock_ctx *c, dock_kernel_stat *st, int32_t cap)
{
    if (!c) return 0;
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
        dock_status s;
        if ((s = dalloc(ctx, (void **)&dt, sizeof(float2) * M, nullptr)) != DOCK_OK) return s;
        if ((s = dalloc(ctx, (void **)&dq, sizeof(float2) * (M / 2), nullptr)) != DOCK_OK) return s;
        if ((s = dalloc(ctx, (void **)&dd, sizeof(double2) * M, nullptr)) != DOCK_OK) return s;
        CK(ctx, cudaMemcpy(dt, t.data(), sizeof(float2) * M, cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(dq, q.data(), sizeof(float2) * (M / 2), cudaMemcpyHostToDevice));
        CK(ctx, cudaMemcpy(dd, td.data(), sizeof(double2) * M, cudaMemcpyHostToDevice));
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
    dock_ctx *ctx = ob->ctx;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ob->O);
    cudaFree(ob->spec);
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
    dock_ctx *ctx = sw->ctx;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(sw->poses);
    cudaFree(sw->cs_dev);
    cudaFree(sw->labels);
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

// Upload quaternions [begin, begin + count) of a set of n_total and build
// their lattice set-up records at the same global indices.
static dock_status upload_rots(dock_ctx *ctx, const dock_sweep *sw, const double *q, int n_total, int begin, int count)
{
    dock_status s;
    if ((s = ensure(ctx, (void **)&ctx->quats, &ctx->quats_n, (size_t)n_total * 4, sizeof(double))) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->rots, &ctx->rots_n, (size_t)n_total, sizeof(RotRec))) != DOCK_OK) return s;
    if (count <= 0) return DOCK_OK;
    CK(ctx, cudaMemcpyAsync(ctx->quats + 4 * (size_t)begin, q + 4 * (size_t)begin, sizeof(double) * 4 * count,
                            cudaMemcpyHostToDevice, ctx->stream));
    Prof pr(ctx, "rot_setup");
    CK(ctx, launch_rot_setup(ctx->quats + 4 * (size_t)begin, count, begin, sw->cs_dev, sw->h, sw->N, ctx->rots + begin,
                             ctx->stream));
    return DOCK_OK;
}

extern "C" dock_status dock_sweep_voxelise(dock_ctx *ctx, const dock_sweep *sw, const double *quats, int32_t n,
                                           uint8_t *bits, double *origins)
{
    if (!ctx || !sw || !quats || n <= 0) return DOCK_E_INVALID;
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    cudaSetDevice(ctx->device);
    dock_search_desc d = {};
    d.sampler = DOCK_SAMPLER_EXPLICIT;
    d.n = n;
    d.quats = quats;
    std::vector<double> q;
    dock_status s;
    if ((s = gen_samples(ctx, &d, q)) != DOCK_OK) return s;
    if ((s = upload_rots(ctx, sw, q.data(), n, 0, n)) != DOCK_OK) return s;
    Geo g = make_geo(sw);
    size_t per = (size_t)g.N * g.N * g.N;
    uint8_t *dbits = nullptr;
    if ((s = dalloc(ctx, (void **)&dbits, per * n, nullptr)) != DOCK_OK) return s;
    CK(ctx, cudaMemsetAsync(ctx->errflag, 0, sizeof(int), ctx->stream));
    cudaError_t e;
    {
        Prof pr(ctx, "vox_export");
        e = launch_vox_export(g, ctx->rots, n, sw->poses, (int)sw->P, dbits, ctx->stream);
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

// ---------------------------------------------------------------------------
// search
// ---------------------------------------------------------------------------
static int auto_batch(const Geo &g)
{
    size_t per = (size_t)(g.N + g.M) * g.M * g.P * sizeof(float2);
    size_t lim = (size_t)1 << 30;
    size_t b = lim / per;
    if (b < 1) b = 1;
    if (b > 64) b = 64;
    return (int)b;
}

static dock_status check_pair(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw)
{
    if (ob->N != sw->N || ob->h != sw->h)
        return fail(ctx, DOCK_E_INVALID, "object and sweep lattices differ (N %d vs %d, h %g vs %g)", ob->N, sw->N,
                    ob->h, sw->h);
    return DOCK_OK;
}

// Runs rotations [r0, r1) of the uploaded set through the pipeline into ctx->keys.
static dock_status run_pipeline(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw, int r0, int r1, int batch)
{
    Geo g = make_geo(sw);
    float2 *tw, *qt;
    double2 *twd;
    dock_status s;
    if ((s = tables(ctx, g.M, &tw, &qt, &twd)) != DOCK_OK) return s;
    int B = batch > 0 ? batch : auto_batch(g);
    size_t ysz = (size_t)B * g.N * g.M * g.P, zsz = (size_t)B * g.M * g.M * g.P;
    size_t need = ysz + zsz;
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
    float2 *Y = ctx->Y, *Z = ctx->Y + ysz;
    if ((s = ensure(ctx, (void **)&ctx->bits, &ctx->bits_n, (size_t)B * g.N * g.N * (g.N / 32), sizeof(uint32_t))) != DOCK_OK)
        return s;
    int chunks = g.M * g.P / 32;
    for (int b0 = r0; b0 < r1; b0 += B) {
        int nb = std::min(B, r1 - b0);
        int groups_needed = (2 * 152 + chunks - 1) / chunks;
        int group = std::max(1, nb / groups_needed);
        {
            Prof pr(ctx, "voxelise");
            CK(ctx, launch_voxelise(g, ctx->rots + b0, nb, sw->poses, (int)sw->P, ctx->bits, ctx->stream));
        }
        {
            Prof pr(ctx, "fwd2d");
            CK(ctx, launch_fwd2d(g, nb, ctx->bits, Y, tw, qt, ctx->stream));
        }
        {
            Prof pr(ctx, "zpass");
            CK(ctx, launch_zpass(g, nb, group, Y, ob->spec, Z, tw, ctx->stream));
        }
        {
            Prof pr(ctx, "plane");
            CK(ctx, launch_plane(g, nb, Z, tw, ctx->rots + b0, ctx->keys, ctx->stream));
        }
    }
    return DOCK_OK;
}

static dock_status search_impl(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw, const dock_search_desc *d,
                               const std::vector<double> &q, int r0, int r1, dock_candidate *out, dock_peak *per_rot)
{
    const int n = d->n;
    dock_status s;
    if ((s = upload_rots(ctx, sw, q.data(), n, 0, n)) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->keys, &ctx->keys_n, (size_t)n, sizeof(unsigned long long))) != DOCK_OK) return s;
    CK(ctx, cudaMemsetAsync(ctx->keys, 0, sizeof(unsigned long long) * n, ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->errflag, 0, sizeof(int), ctx->stream));
    if ((s = run_pipeline(ctx, ob, sw, r0, r1, d->batch)) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->cands, &ctx->cands_n, (size_t)d->top_k, sizeof(dock_candidate))) != DOCK_OK) return s;
    {
        Prof pr(ctx, "topk");
        CK(ctx, launch_topk(ctx->keys, n, d->top_k, ob->N, ob->M, ob->h, ob->o_dev, ctx->quats, ctx->rots, ctx->cands,
                            ctx->stream));
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

extern "C" dock_status dock_search_scores(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw, const double *quat,
                                          float *C)
{
    if (!ctx || !ob || !sw || !quat || !C) return DOCK_E_INVALID;
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
    if ((s = upload_rots(ctx, sw, q.data(), 1, 0, 1)) != DOCK_OK) return s;
    Geo g = make_geo(sw);
    float2 *tw, *qt;
    double2 *twd;
    if ((s = tables(ctx, g.M, &tw, &qt, &twd)) != DOCK_OK) return s;
    size_t ysz = (size_t)g.N * g.M * g.P, zsz = (size_t)g.M * g.M * g.P, csz = (size_t)g.M * g.M * g.M;
    float2 *Y = nullptr;
    float *dC = nullptr;
    if ((s = ensure(ctx, (void **)&ctx->bits, &ctx->bits_n, (size_t)g.N * g.N * (g.N / 32), sizeof(uint32_t))) != DOCK_OK)
        return s;
    if ((s = dalloc(ctx, (void **)&Y, (ysz + zsz) * sizeof(float2), nullptr)) != DOCK_OK) return s;
    if ((s = dalloc(ctx, (void **)&dC, csz * sizeof(float), nullptr)) != DOCK_OK) { dfree(ctx, Y, (ysz + zsz) * sizeof(float2)); return s; }
    cudaError_t e = cudaMemsetAsync(ctx->errflag, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = launch_voxelise(g, ctx->rots, 1, sw->poses, (int)sw->P, ctx->bits, ctx->stream);
    if (e == cudaSuccess) e = launch_fwd2d(g, 1, ctx->bits, Y, tw, qt, ctx->stream);
    if (e == cudaSuccess) e = launch_zpass(g, 1, 1, Y, ob->spec, Y + ysz, tw, ctx->stream);
    if (e == cudaSuccess) e = launch_plane_export(g, Y + ysz, tw, dC, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(C, dC, csz * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, Y, (ysz + zsz) * sizeof(float2));
    dfree(ctx, dC, csz * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "search_scores");
    return DOCK_OK;
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
    D.tri_iters = p->tri_iters > 0 ? p->tri_iters : 24;
    return D;
}

static dock_status ref_buffers(dock_ctx *ctx, int K, int nblk)
{
    dock_status s;
    if ((s = ensure(ctx, (void **)&ctx->ref_state, &ctx->ref_state_n, (size_t)K * REF_ST, sizeof(double))) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->ref_acc, &ctx->ref_acc_n, (size_t)K * nblk * REF_NACC, sizeof(double))) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->ref_prm, &ctx->ref_prm_n, 8, sizeof(double))) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->ref_cands, &ctx->ref_cands_n, (size_t)K, cand_bytes())) != DOCK_OK) return s;
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

// Runs `iters` projected Gauss-Newton iterations on the K states in
// ctx->ref_state, then a final evaluation that records J at the final twist.
static dock_status refine_loop(dock_ctx *ctx, const RefineDev &D, int K, int iters, const dock_params *p, cudaStream_t st)
{
    int nblk = (D.P + 127) / 128;
    double prm[6] = {p->lambda, p->mu, p->step_t, p->step_r, p->b_t, p->b_r};
    CK(ctx, cudaMemcpyAsync(ctx->ref_prm, prm, sizeof(prm), cudaMemcpyHostToDevice, st));
    CandF *cf = (CandF *)ctx->ref_cands;
    CK(ctx, launch_refine_solve(K, nblk, ctx->ref_state, ctx->ref_acc, ctx->ref_prm, 0, cf, st));
    for (int it = 0; it < iters; ++it) {
        {
            Prof pr(ctx, "refine_eval");
            CK(ctx, launch_refine_eval(D, K, cf, ctx->ref_acc, true, nullptr, nullptr, nullptr, st));
        }
        Prof pr(ctx, "refine_solve");
        CK(ctx, launch_refine_solve(K, nblk, ctx->ref_state, ctx->ref_acc, ctx->ref_prm, 1, cf, st));
    }
    {
        Prof pr(ctx, "refine_eval");
        CK(ctx, launch_refine_eval(D, K, cf, ctx->ref_acc, false, nullptr, nullptr, nullptr, st));
    }
    CK(ctx, launch_refine_solve(K, nblk, ctx->ref_state, ctx->ref_acc, ctx->ref_prm, 2, cf, st));
    return DOCK_OK;
}

static dock_status refine_impl(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw, const dock_candidate *in,
                               int K, const dock_params *p, dock_refined *out)
{
    int nblk = ((int)sw->P + 127) / 128;
    dock_status s;
    if ((s = ref_buffers(ctx, K, nblk)) != DOCK_OK) return s;
    std::vector<double> st((size_t)K * REF_ST);
    for (int c = 0; c < K; ++c) state_from_pose(in[c].q, in[c].t, ob->anchor, st.data() + (size_t)c * REF_ST);
    CK(ctx, cudaMemcpyAsync(ctx->ref_state, st.data(), sizeof(double) * st.size(), cudaMemcpyHostToDevice, ctx->stream));
    RefineDev D = make_refine_dev(ob, sw, p);
    if ((s = refine_loop(ctx, D, K, p->iters, p, ctx->stream)) != DOCK_OK) return s;
    CK(ctx, cudaMemcpyAsync(st.data(), ctx->ref_state, sizeof(double) * st.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < K; ++c) {
        const double *x = st.data() + (size_t)c * REF_ST;
        double R[9], t[3];
        pose_of_state(x, R, t);
        mat_to_quat(R, out[c].q);
        memcpy(out[c].t, t, sizeof(t));
        memcpy(out[c].xi, x + 15, sizeof(double) * 6);
        out[c].J = x[21];
        out[c].cand = c;
        out[c].iters = p->iters;
    }
    return DOCK_OK;
}

static dock_status check_quat_pose(dock_ctx *ctx, const double *q)
{
    for (int k = 0; k < 7; ++k) if (!isfinite(q[k])) return fail(ctx, DOCK_E_INVALID, "pose is not finite");
    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(fabs(nq - 1.0) <= 1e-6)) return fail(ctx, DOCK_E_INVALID, "pose quaternion is not unit");
    return DOCK_OK;
}

extern "C" dock_status dock_refine_se3(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                       const dock_candidate *in, int32_t K, const dock_params *params,
                                       dock_refined *out)
{
    if (!ctx || !ob || !sw || !in || !out) return DOCK_E_INVALID;
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    if (K < 1 || K > 1024) return fail(ctx, DOCK_E_INVALID, "K must be in [1, 1024]");
    dock_status s;
    if ((s = check_pair(ctx, ob, sw)) != DOCK_OK) return s;
    dock_params pd;
    dock_params_default(&pd);
    const dock_params *p = params ? params : &pd;
    if (p->iters < 0 || p->iters > 10000) return fail(ctx, DOCK_E_INVALID, "iters out of range");
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
    if ((s = ref_buffers(ctx, B, nblk)) != DOCK_OK) return s;
    std::vector<double> stv((size_t)B * REF_ST);
    for (int b = 0; b < B; ++b) state_from_pose(base + 7 * b, base + 7 * b + 4, ob->anchor, stv.data() + (size_t)b * REF_ST);
    CK(ctx, cudaMemcpyAsync(ctx->ref_state, stv.data(), sizeof(double) * stv.size(), cudaMemcpyHostToDevice, st));
    CK(ctx, cudaStreamSynchronize(st));   // the host staging vector is released on return
    CK(ctx, launch_set_xi(B, xi, ctx->ref_state, st));
    CandF *cf = (CandF *)ctx->ref_cands;
    CK(ctx, launch_refine_solve(B, nblk, ctx->ref_state, ctx->ref_acc, ctx->ref_prm, 0, cf, st));
    RefineDev D = make_refine_dev(ob, sw, p);
    {
        Prof pr(ctx, grad ? "objective_adjoint" : "objective_fwd");
        CK(ctx, launch_refine_eval(D, B, cf, ctx->ref_acc, grad != nullptr, nullptr, nullptr, nullptr, st));
    }
    CK(ctx, launch_finish_objective(B, nblk, ctx->ref_state, ctx->ref_acc, p->lambda, J, grad, gJ, st));
    return DOCK_OK;
}

extern "C" dock_status dock_objective_fwd(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                          const double *base_poses, const float *xi, int32_t B,
                                          const dock_params *params, float *J, float *grad, void *stream)
{
    if (!J) return fail(ctx, DOCK_E_INVALID, "J output is required");
    return objective_impl(ctx, ob, sw, base_poses, xi, B, params, J, grad, nullptr, stream);
}

extern "C" dock_status dock_objective_bwd(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                          const double *base_poses, const float *xi, int32_t B,
                                          const dock_params *params, const float *gJ, float *gxi, void *stream)
{
    if (!gJ || !gxi) return fail(ctx, DOCK_E_INVALID, "gJ and gxi are required");
    return objective_impl(ctx, ob, sw, base_poses, xi, B, params, nullptr, gxi, gJ, stream);
}

extern "C" dock_status dock_distances(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                      const double *obj_poses, int32_t B, const dock_params *params, float *d,
                                      float *witness, float *normal)
{
    if (!ctx || !ob || !sw || !obj_poses || B < 1 || !d || !witness || !normal) return DOCK_E_INVALID;
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    dock_status s;
    if ((s = check_pair(ctx, ob, sw)) != DOCK_OK) return s;
    dock_params pd;
    dock_params_default(&pd);
    const dock_params *p = params ? params : &pd;
    cudaSetDevice(ctx->device);
    int nblk = ((int)sw->P + 127) / 128;
    if ((s = ref_buffers(ctx, B, nblk)) != DOCK_OK) return s;
    std::vector<double> stv((size_t)B * REF_ST);
    for (int b = 0; b < B; ++b) {
        if ((s = check_quat_pose(ctx, obj_poses + 7 * b)) != DOCK_OK) return s;
        state_from_pose(obj_poses + 7 * b, obj_poses + 7 * b + 4, ob->anchor, stv.data() + (size_t)b * REF_ST);
    }
    size_t n = (size_t)B * sw->P;
    float *buf = nullptr;
    if ((s = dalloc(ctx, (void **)&buf, sizeof(float) * 7 * n, nullptr)) != DOCK_OK) return s;
    cudaStream_t st = ctx->stream;
    CandF *cf = (CandF *)ctx->ref_cands;
    RefineDev D = make_refine_dev(ob, sw, p);
    cudaError_t e = cudaMemcpyAsync(ctx->ref_state, stv.data(), sizeof(double) * stv.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_refine_solve(B, nblk, ctx->ref_state, ctx->ref_acc, ctx->ref_prm, 0, cf, st);
    if (e == cudaSuccess) e = launch_refine_eval(D, B, cf, ctx->ref_acc, false, buf, buf + n, buf + 4 * n, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, buf, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(witness, buf + n, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(normal, buf + 4 * n, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(ctx, buf, sizeof(float) * 7 * n);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "distances");
    return DOCK_OK;
}

// ---------------------------------------------------------------------------
// three-stage registration (Fig. 2)
// ---------------------------------------------------------------------------
extern "C" dock_status dock_register(dock_ctx *ctx, const dock_object *ob, const dock_sweep *sw,
                                     const dock_register_desc *rd, const dock_params *params, dock_result *out)
{
    if (!ctx || !ob || !sw || !rd || !out) return DOCK_E_INVALID;
    if (ctx->dead) return fail(ctx, DOCK_E_CUDA_FATAL, "context is dead after a sticky CUDA error");
    dock_status s;
    if ((s = check_pair(ctx, ob, sw)) != DOCK_OK) return s;
    if (rd->n_global < 1 || rd->n_local < 0 || rd->top_k < 1 || rd->top_k > 1024)
        return fail(ctx, DOCK_E_INVALID, "bad registration descriptor");
    if (rd->sampler != DOCK_SAMPLER_SF && rd->sampler != DOCK_SAMPLER_HOPF)
        return fail(ctx, DOCK_E_INVALID, "global sampler must be SF or HOPF");
    dock_params pd;
    dock_params_default(&pd);
    const dock_params *p = params ? params : &pd;
    cudaSetDevice(ctx->device);
    const int ng = rd->n_global, nl = rd->n_local, n = ng + nl;
    // stage 1: global search
    dock_search_desc d = {};
    d.sampler = rd->sampler;
    d.n = ng;
    d.top_k = 1;
    std::vector<double> qg, q((size_t)n * 4);
    if ((s = gen_samples(ctx, &d, qg)) != DOCK_OK) return s;
    memcpy(q.data(), qg.data(), sizeof(double) * 4 * ng);
    if ((s = upload_rots(ctx, sw, q.data(), n, 0, ng)) != DOCK_OK) return s;
    if ((s = ensure(ctx, (void **)&ctx->keys, &ctx->keys_n, (size_t)n, sizeof(unsigned long long))) != DOCK_OK) return s;
    CK(ctx, cudaMemsetAsync(ctx->keys, 0, sizeof(unsigned long long) * n, ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->errflag, 0, sizeof(int), ctx->stream));
    if ((s = run_pipeline(ctx, ob, sw, 0, ng, 0)) != DOCK_OK) return s;
    int K = rd->top_k;
    if ((s = ensure(ctx, (void **)&ctx->cands, &ctx->cands_n, (size_t)std::max(K, 1), sizeof(dock_candidate))) != DOCK_OK) return s;
    dock_candidate best;
    {
        Prof pr(ctx, "topk");
        CK(ctx, launch_topk(ctx->keys, ng, 1, ob->N, ob->M, ob->h, ob->o_dev, ctx->quats, ctx->rots, ctx->cands,
                            ctx->stream));
    }
    CK(ctx, cudaMemcpyAsync(&best, ctx->cands, sizeof(best), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    // stage 2: local GeoBall-SF search around the best orientation
    if (nl > 0) {
        dock_search_desc dl = {};
        dl.sampler = DOCK_SAMPLER_GEOBALL;
        dl.n = nl;
        memcpy(dl.q0, best.q, sizeof(dl.q0));
        dl.theta = rd->theta;
        std::vector<double> ql;
        if ((s = gen_samples(ctx, &dl, ql)) != DOCK_OK) return s;
        memcpy(q.data() + 4 * (size_t)ng, ql.data(), sizeof(double) * 4 * nl);
        if ((s = upload_rots(ctx, sw, q.data(), n, ng, nl)) != DOCK_OK) return s;
        if ((s = run_pipeline(ctx, ob, sw, ng, n, 0)) != DOCK_OK) return s;
    }
    std::vector<dock_candidate> cands(K);
    {
        Prof pr(ctx, "topk");
        CK(ctx, launch_topk(ctx->keys, n, K, ob->N, ob->M, ob->h, ob->o_dev, ctx->quats, ctx->rots, ctx->cands,
                            ctx->stream));
    }
    int herr = 0;
    CK(ctx, cudaMemcpyAsync(cands.data(), ctx->cands, sizeof(dock_candidate) * K, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaMemcpyAsync(&herr, ctx->errflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (herr) return fail(ctx, herr, "device reported error %d during the search", herr);
    int Kv = 0;
    while (Kv < K && cands[Kv].rot >= 0) ++Kv;
    if (Kv == 0) return fail(ctx, DOCK_E_INVALID, "the search produced no candidate");
    // stage 3: refinement of the surviving candidates; lowest J wins
    std::vector<dock_refined> ref(Kv);
    if ((s = refine_impl(ctx, ob, sw, cands.data(), Kv, p, ref.data())) != DOCK_OK) return s;
    int bi = 0;
    for (int c = 1; c < Kv; ++c) if (ref[c].J < ref[bi].J) bi = c;
    memcpy(out->q, ref[bi].q, sizeof(out->q));
    memcpy(out->t, ref[bi].t, sizeof(out->t));
    out->J = ref[bi].J;
    out->best_cand = bi;
    out->n_evals = n;
    out->best_search = cands[0];
    return DOCK_OK;
}
