// Continuous refinement (Sec. V) on the GPU.
//
// K10/K11 (k_refine_eval): one thread per (candidate, probe pose).  The probe
// pose is expressed in the object frame, the mesh BVH is traversed with the
// Eq. (21) test f_p(c) < r_node + eps (eps = tau_out2, so pruned geometry
// can only have s = s' = 0), and each surviving triangle's minimum of f_p is
// found by golden-section search over one barycentric coordinate with an inner
// bisection on subgradient signs (f_p is convex).  From d*, the witness and
// the SDF normal (Eq. (22)-(23)) the kernel forms the exact sensitivities of
// d w.r.t. the twist (Eq. (24)-(27), rotational term through the left Jacobian
// V(w), coupling term analytic), the score s(d) of Eq. (18) and its
// derivatives, and reduces J, grad J (Eq. (28)) and the Gauss-Newton matrix
// per candidate in FP64, deterministically (per-block partials, fixed order).
// K12 (k_refine_solve): one thread per candidate, FP64: Cholesky 6x6 solve of
// the normal equations, trust-region scaling, box projection (Eq. (20)), and
// the pose data of the next iteration (Eq. (14)-(17)).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dock_internal.h"

namespace dock {

#define KINK_BAND 1e-3f   // distance from the medial surface within which a witness is treated as on it (mm)

// per-candidate data read by the evaluation kernel (FP32)
struct CandF {
    float R[9], p[3];   // object pose T(xi)
    float V[9];         // left Jacobian V(w)
    float Mc[9];        // d(V(w) u)/dw
    float c[3];         // pivot p0 + V u + R0 a
    float pad[3];
};

// state layout (doubles): R0[9] p0[3] a[3] xi[6] -> 21, then J at 21, pad to 24
constexpr int ST = 24;
constexpr int NACC = 28;   // J, G[6], H upper triangle [21]

// f_p of the flat-ended cylinder (tip face z = 0, body z in [0, L]) and, in g,
// the gradient of the active branch (a valid subgradient: the cap branch on
// the inside medial surface dr == dz, +x as the radial direction on the axis).
__device__ __forceinline__ float sdf_cyl(float x, float y, float z, float r, float L, float *g)
{
    float rho = sqrtf(fmaf(x, x, y * y));
    float ux = 1.f, uy = 0.f;
    if (rho > 0.f) { ux = x / rho; uy = y / rho; }
    float dr = rho - r;
    float zlo = -z, zhi = z - L;
    float dz = zlo >= zhi ? zlo : zhi;
    float cz = zlo >= zhi ? -1.f : 1.f;
    float f;
    if (dr <= 0.f && dz <= 0.f) {
        if (dr > dz) { f = dr; if (g) { g[0] = ux; g[1] = uy; g[2] = 0.f; } }
        else { f = dz; if (g) { g[0] = 0.f; g[1] = 0.f; g[2] = cz; } }
    } else if (dr > 0.f && dz > 0.f) {
        f = sqrtf(fmaf(dr, dr, dz * dz));
        if (g) { g[0] = dr * ux / f; g[1] = dr * uy / f; g[2] = dz * cz / f; }
    } else if (dr > 0.f) {
        f = dr;
        if (g) { g[0] = ux; g[1] = uy; g[2] = 0.f; }
    } else {
        f = dz;
        if (g) { g[0] = 0.f; g[1] = 0.f; g[2] = cz; }
    }
    return f;
}

// Contact normal n* (Eq. (23)): the unit gradient; where f_p is not
// differentiable (the medial surface inside, the axis) the gradient of the
// branch sdf_cyl reports (the cap on ties, +x radially on the axis).
__device__ __forceinline__ void sdf_normal(const float *x, float r, float L, float *n)
{
    float g[3];
    sdf_cyl(x[0], x[1], x[2], r, L, g);
    float gn = sqrtf(fmaf(g[0], g[0], fmaf(g[1], g[1], g[2] * g[2])));
    n[0] = g[0] / gn; n[1] = g[1] / gn; n[2] = g[2] / gn;
}

__device__ __forceinline__ float dot3f(const float *a, const float *b) { return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2])); }

// The subgradient of f_p at the witness x (probe frame) of triangle lv that
// gives the derivative of d = min over the triangle of f_p (Sec. V-B,
// Eq. (22)-(24)): the gradient where f_p is differentiable; on the medial
// surface inside the probe, the combination lam a + (1 - lam) b of the
// radial and cap gradients whose component along the witness's face (the
// triangle's plane, or its edge when a barycentric weight is ~0) vanishes,
// the element the minimum over the triangle selects (Danskin); a vertex lies
// on the medial surface only by coincidence, so at a vertex witness the
// gradient of the active branch (sdf_normal).  Not normalised.
__device__ __noinline__ void witness_subgradient(const float *x, const float lv[3][3], float r, float L, float *n)
{
    const float rho = sqrtf(fmaf(x[0], x[0], x[1] * x[1]));
    const float dr = rho - r, zlo = -x[2], zhi = x[2] - L;
    const float dz = zlo >= zhi ? zlo : zhi;
    if (!(dr <= 0.f && dz <= 0.f && fabsf(dr - dz) <= KINK_BAND && rho > 0.f)) {
        sdf_normal(x, r, L, n);
        return;
    }
    float e1[3], e2[3], p[3];
    for (int i = 0; i < 3; ++i) { e1[i] = lv[1][i] - lv[0][i]; e2[i] = lv[2][i] - lv[0][i]; p[i] = x[i] - lv[0][i]; }
    const float d00 = dot3f(e1, e1), d01 = dot3f(e1, e2), d11 = dot3f(e2, e2), d20 = dot3f(p, e1), d21 = dot3f(p, e2);
    const float den = fmaf(d00, d11, -d01 * d01);
    float w[3];
    w[1] = den != 0.f ? fmaf(d11, d20, -d01 * d21) / den : 0.f;
    w[2] = den != 0.f ? fmaf(d00, d21, -d01 * d20) / den : 0.f;
    w[0] = 1.f - w[1] - w[2];
    int nz = 0, zi = -1;
    for (int k = 0; k < 3; ++k)
        if (w[k] <= 1e-4f) { ++nz; zi = k; }
    if (nz >= 2 || den == 0.f) {
        sdf_normal(x, r, L, n);
        return;
    }
    const float a[3] = {x[0] / rho, x[1] / rho, 0.f}, b[3] = {0.f, 0.f, zlo >= zhi ? -1.f : 1.f};
    float Pa[3], Pb[3];
    if (nz == 0) {
        const float nu[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const float nn = dot3f(nu, nu), an = dot3f(a, nu) / nn, bn = dot3f(b, nu) / nn;
        for (int i = 0; i < 3; ++i) { Pa[i] = a[i] - an * nu[i]; Pb[i] = b[i] - bn * nu[i]; }
    } else {
        const float *pp = lv[(zi + 1) % 3], *qq = lv[(zi + 2) % 3];
        const float e[3] = {qq[0] - pp[0], qq[1] - pp[1], qq[2] - pp[2]};
        const float ee = dot3f(e, e), ae = dot3f(a, e) / ee, be = dot3f(b, e) / ee;
        for (int i = 0; i < 3; ++i) { Pa[i] = ae * e[i]; Pb[i] = be * e[i]; }
    }
    const float df[3] = {Pa[0] - Pb[0], Pa[1] - Pb[1], Pa[2] - Pb[2]};
    const float dd = dot3f(df, df);
    const float lm = dd > 0.f ? fminf(1.f, fmaxf(0.f, -dot3f(Pb, df) / dd)) : 0.5f;
    for (int i = 0; i < 3; ++i) n[i] = fmaf(lm, a[i], (1.f - lm) * b[i]);
}

// A number with the sign of g . e, g the subgradient sdf_cyl reports at
// (x, y, z) (same branch rules), without normalising g: the bisections need
// only the sign of the directional derivative.
__device__ __forceinline__ float sdf_slope_sign(float x, float y, float z, float r, float L, const float *e)
{
    const float r2 = fmaf(x, x, y * y);
    const float ri = r2 > 0.f ? rsqrtf(r2) : 0.f;
    const float rho = r2 * ri;
    const float se = r2 > 0.f ? fmaf(x, e[0], y * e[1]) : e[0];   // rho (u . e_xy), u = +x on the axis
    const float dr = rho - r, zlo = -z, zhi = z - L;
    const float dz = zlo >= zhi ? zlo : zhi;
    const float ce = zlo >= zhi ? -e[2] : e[2];                    // cz e_z
    if (dr <= 0.f && dz <= 0.f) return dr > dz ? se : ce;
    if (dr > 0.f && dz > 0.f) return fmaf(dr * se, r2 > 0.f ? ri : 1.f, dz * ce);
    return dr > 0.f ? se : ce;
}

// f_p is differentiable at x: everywhere outside the probe; inside, away
// (by more than 1e-3 mm) from the medial surfaces where two branches meet
// and from the axis.
__device__ __forceinline__ bool sdf_smooth_at(const float *x, float r, float L)
{
    float rho = sqrtf(fmaf(x[0], x[0], x[1] * x[1]));
    float dr = rho - r, zlo = -x[2], zhi = x[2] - L;
    float dz = fmaxf(zlo, zhi);
    if (dr > 0.f || dz > 0.f) return true;
    const float band = 1e-3f;
    return fabsf(dr - dz) > band && fabsf(zlo - zhi) > band && rho > band;
}

// min over v in [0, 1-u] of f(v0 + u e1 + v e2): bisection on df/dv (a
// subgradient sign; the same steps for every call, so the lanes of a warp
// that search together stay converged; an end minimum is approached to
// 2^-iters of the segment)
__device__ __noinline__ float inner_min(const float *v0, const float *e1, const float *e2, float u, float r, float L,
                                        int iters, float *v_out)
{
    const float vmax = fmaxf(0.f, 1.f - u);
    float x[3];
    for (int a = 0; a < 3; ++a) x[a] = fmaf(u, e1[a], v0[a]);
    float lo = 0.f, hi = vmax;
    for (int k = 0; k < iters; ++k) {
        float mid = 0.5f * (lo + hi);
        float xm[3];
        for (int a = 0; a < 3; ++a) xm[a] = fmaf(mid, e2[a], x[a]);
        if (sdf_slope_sign(xm[0], xm[1], xm[2], r, L, e2) < 0.f) lo = mid; else hi = mid;
    }
    float v = 0.5f * (lo + hi);
    for (int a = 0; a < 3; ++a) x[a] = fmaf(v, e2[a], x[a]);
    *v_out = v;
    return sdf_cyl(x[0], x[1], x[2], r, L, nullptr);
}

// dphi/du at u for the partial minimum phi(u) = min_v f(v0 + u e1 + v e2)
// (Danskin; valid where f is differentiable at the inner minimiser).
__device__ float outer_slope(const float *v0, const float *e1, const float *e2, float u, float r, float L, int iters)
{
    float v;
    inner_min(v0, e1, e2, u, r, L, iters, &v);
    float x[3], g[3];
    for (int a = 0; a < 3; ++a) x[a] = fmaf(v, e2[a], fmaf(u, e1[a], v0[a]));
    sdf_cyl(x[0], x[1], x[2], r, L, g);
    float s = dot3f(g, e1);
    if (v >= 1.f - u && v > 0.f) s -= dot3f(g, e2);
    return s;
}

// min of f_p over the triangle (local coordinates); returns d, writes (u, v).
// Golden-section search on phi(u) (values only: robust on the non-smooth
// medial surface), then, for a minimum outside the probe (f is C^1 there), a
// bisection on dphi/du inside a bracket that stays outside: value-based search
// locates a smooth minimum only to ~sqrt(FP32 eps), the slope to ~eps.
// First-order tests: true (with the minimum in *d and its barycentric (u, v))
// when the minimum of f over the triangle is found at a vertex or on an edge.
__device__ bool tri_min_shortcut(const float *v0, const float *v1, const float *v2, const float *fv, float r, float L,
                                 float *d, float *uo, float *vo)
{
    {
        // A vertex where f is differentiable and no edge from it descends is
        // the minimum (f convex: f(y) >= f(x) + g.(y - x) >= f(x) on the
        // triangle).  This settles most triangles, which are small against the
        // probe; fv holds f at the three vertices.
        const float *vv[3] = {v0, v1, v2};
        int ms = 0;
        if (fv[1] < fv[ms]) ms = 1;
        if (fv[2] < fv[ms]) ms = 2;
        float g[3];
        if (sdf_smooth_at(vv[ms], r, L)) {
            sdf_cyl(vv[ms][0], vv[ms][1], vv[ms][2], r, L, g);
            bool opt = true;
            for (int m = 0; m < 3; ++m) {
                if (m == ms) continue;
                float e[3] = {vv[m][0] - vv[ms][0], vv[m][1] - vv[ms][1], vv[m][2] - vv[ms][2]};
                if (dot3f(g, e) < 0.f) opt = false;
            }
            if (opt) {
                *uo = ms == 1 ? 1.f : 0.f;
                *vo = ms == 2 ? 1.f : 0.f;
                *d = fv[ms];
                return true;
            }
        }
        // An edge point that minimises f along its edge, where f is
        // differentiable and the direction to the opposite vertex does not
        // descend, is the minimum over the triangle (same argument: the
        // triangle lies in the cone of +-edge and that direction).  Typical for
        // a line contact with the probe's side.
        for (int k = 0; k < 3; ++k) {
            const float *pa = vv[k], *pb = vv[(k + 1) % 3], *po = vv[(k + 2) % 3];
            float e[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
            if (sdf_slope_sign(pa[0], pa[1], pa[2], r, L, e) >= 0.f) continue;   // f grows along the edge from pa
            if (sdf_slope_sign(pb[0], pb[1], pb[2], r, L, e) <= 0.f) continue;   // f falls all the way to pb
            float lo = 0.f, hi = 1.f;
            for (int it = 0; it < 24; ++it) {
                float mid = 0.5f * (lo + hi), xm[3];
                for (int c = 0; c < 3; ++c) xm[c] = fmaf(mid, e[c], pa[c]);
                if (sdf_slope_sign(xm[0], xm[1], xm[2], r, L, e) < 0.f) lo = mid; else hi = mid;
            }
            float s = 0.5f * (lo + hi), x[3], gx[3];
            for (int c = 0; c < 3; ++c) x[c] = fmaf(s, e[c], pa[c]);
            if (!sdf_smooth_at(x, r, L)) continue;
            float fx = sdf_cyl(x[0], x[1], x[2], r, L, gx);
            float eo[3] = {po[0] - x[0], po[1] - x[1], po[2] - x[2]};
            if (dot3f(gx, eo) < 0.f) continue;
            // barycentric (u, v) of x = (1 - u - v) v0 + u v1 + v v2
            if (k == 0) { *uo = s; *vo = 0.f; }
            else if (k == 1) { *uo = 1.f - s; *vo = s; }
            else { *uo = 0.f; *vo = 1.f - s; }
            *d = fx;
            return true;
        }
    }
    return false;
}

// Minimum of f over the triangle by golden-section search on the first
// barycentric coordinate with an inner bisection (for triangles the
// first-order tests do not settle).
__device__ __noinline__ float tri_min_search(const float *v0, const float *v1, const float *v2, float r, float L,
                                             int iters, float *uo, float *vo)
{
    float e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
    float e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
    const float ig = 0.6180339887498949f;
    float a = 0.f, b = 1.f, vc, vd;
    float c = b - ig * (b - a), d = a + ig * (b - a);
    float fc = inner_min(v0, e1, e2, c, r, L, iters, &vc);
    float fd = inner_min(v0, e1, e2, d, r, L, iters, &vd);
    int steps = iters + iters / 2;
    for (int k = 0; k < steps; ++k) {
        // one evaluation per step on every path
        const bool left = fc <= fd;
        if (left) { b = d; d = c; fd = fc; vd = vc; }
        else { a = c; c = d; fc = fd; vc = vd; }
        const float xn = left ? b - ig * (b - a) : a + ig * (b - a);
        float vn;
        const float fn = inner_min(v0, e1, e2, xn, r, L, iters, &vn);
        if (left) { c = xn; fc = fn; vc = vn; }
        else { d = xn; fd = fn; vd = vn; }
    }
    float u = fc <= fd ? c : d, v = fc <= fd ? vc : vd, best = fc <= fd ? fc : fd;
    float vu0, vu1;
    float f0 = inner_min(v0, e1, e2, 0.f, r, L, iters, &vu0);
    float f1 = inner_min(v0, e1, e2, 1.f, r, L, iters, &vu1);
    if (f0 < best) { best = f0; u = 0.f; v = vu0; }
    if (f1 < best) { best = f1; u = 1.f; v = vu1; }
    float le = sqrtf(dot3f(e1, e1));
    if (best > 1e-4f && le > 0.f) {
        float w = fminf(2e-3f, 0.5f * best / le);
        float lo = fmaxf(0.f, u - w), hi = fminf(1.f, u + w);
        if (outer_slope(v0, e1, e2, lo, r, L, iters) >= 0.f) {
            hi = lo;
        } else if (outer_slope(v0, e1, e2, hi, r, L, iters) <= 0.f) {
            lo = hi;
        } else {
            for (int k = 0; k < 16; ++k) {
                float mid = 0.5f * (lo + hi);
                if (outer_slope(v0, e1, e2, mid, r, L, iters) < 0.f) lo = mid; else hi = mid;
            }
        }
        float up = 0.5f * (lo + hi), vp;
        float fp = inner_min(v0, e1, e2, up, r, L, iters, &vp);
        if (fp <= best) { best = fp; u = up; v = vp; }
    }
    *uo = u;
    *vo = v;
    return best;
}


// Lower bound of min f over the triangle: the linearisation at the centroid
// with a subgradient there (f is convex).
__device__ __forceinline__ float lin_lower_bound(const float lv[3][3], float r, float L)
{
    float c[3], g[3];
    for (int a = 0; a < 3; ++a) c[a] = (lv[0][a] + lv[1][a] + lv[2][a]) * (1.f / 3.f);
    float fc = sdf_cyl(c[0], c[1], c[2], r, L, g);
    float m = INFINITY;
    for (int k = 0; k < 3; ++k) {
        float d[3] = {lv[k][0] - c[0], lv[k][1] - c[1], lv[k][2] - c[2]};
        m = fminf(m, dot3f(g, d));
    }
    return fc + m;
}

// Eq. (18): s(d), s'(d), s''(d) with r = tau_in / tau_out and C^1 coefficients
__device__ __forceinline__ void score3(const RefineDev &D, float d, float *s, float *s1, float *s2)
{
    float it = 1.f / D.tau_out;
    float t = d * it;
    if (t > 1.f) { *s = 0.f; *s1 = 0.f; *s2 = 0.f; }
    else if (t > 0.f) {
        float cs = cospif(0.5f * t), sn = sinpif(0.5f * t);
        *s = cs * cs;
        *s1 = -3.14159265358979f * cs * sn * it;
        *s2 = -0.5f * 9.8696044010893586f * cospif(t) * it * it;
    } else if (t > -D.rr) {
        *s = fmaf(D.A * t, t * t, D.B * t * t) + 1.f;
        *s1 = (3.f * D.A * t * t + 2.f * D.B * t) * it;
        *s2 = (6.f * D.A * t + 2.f * D.B) * it * it;
    } else {
        *s = D.k_slope * (t + D.rr);
        *s1 = D.k_slope * it;
        *s2 = 0.f;
    }
}

__device__ __forceinline__ void local_vertices(const RefineDev &D, int t, const float *A, const float *bvec,
                                               float lv[3][3])
{
    for (int m = 0; m < 3; ++m) {
        const float *v = D.Vf + 3 * D.T[3 * t + m];
        float qv[3] = {v[0] - bvec[0], v[1] - bvec[1], v[2] - bvec[2]};
        for (int a = 0; a < 3; ++a) lv[m][a] = fmaf(A[0 * 3 + a], qv[0], fmaf(A[1 * 3 + a], qv[1], A[2 * 3 + a] * qv[2]));
    }
}

// f_p at a bounding-sphere centre c (object frame) for the probe frame (A, b).
__device__ __forceinline__ float node_sdf(const RefineDev &D, const float *A, const float *bvec, const float *c)
{
    float q[3] = {c[0] - bvec[0], c[1] - bvec[1], c[2] - bvec[2]};
    float loc[3];
    for (int k = 0; k < 3; ++k) loc[k] = fmaf(A[0 * 3 + k], q[0], fmaf(A[1 * 3 + k], q[1], A[2 * 3 + k] * q[2]));
    return sdf_cyl(loc[0], loc[1], loc[2], D.r, D.L, nullptr);
}

// Distance query of the warp's 32 probe poses against the mesh (one pose per
// lane; `valid` false for lanes without a pose).  One BVH pass under the
// Eq. (21) test f_p(c) < r_node + eps: every triangle reached lowers the
// lane's upper bound UB of d* by its smallest vertex value, and f_p is
// minimised only over triangles whose linearised lower bound does not exceed
// min(UB, best so far) (a triangle attaining d* is never skipped: its lower
// bound is at most d* <= UB; ties in d keep the lower triangle index).  The warp walks one shared traversal: a node is entered
// when any lane needs it, the nearer child (by the smallest bound over the
// lanes) first, and every lane applies its own tests, so the 32 nearly equal
// poses of a trajectory run in lockstep instead of serialising their
// traversals.  Returns the lane's triangle index or -1; fills d*, the local
// witness and the local contact normal.
__device__ int dist_query(const RefineDev &D, const float *A, const float *bvec, bool valid, int hint, float *d_out,
                          float *xw, float *nl)
{
    int sn[64];
    float sl[64];
    constexpr int QN = 6;                        // deferred per-triangle searches per lane
    int qt[QN];
    float ql[QN];
    int nq = 0;
    // triangles that passed Eq. (21) and the lower-bound test during the
    // traversal, kept in increasing lower-bound order; their first-order tests
    // and searches run after the traversal, slot by slot across the warp (the
    // lanes of a slot in lockstep), and a smaller minimum found early prunes
    // the later ones
    constexpr int QC = 16;
    int ct[QC];
    float cl[QC];
    int nc = 0;
    const float eps = D.tau_out;
    float UB = valid ? INFINITY : -INFINITY;     // a lane without a pose needs nothing
    float best = INFINITY;
    int bt = -1;
    float bx[3] = {0.f, 0.f, 0.f};
    // Start from the hint (the triangle that held this query's minimum at the
    // previous evaluation, if it still passes Eq. (21)): its minimum bounds
    // d* from the first node on.  The result does not depend on the order in
    // which triangles are met, so the hint changes only the work.
    int seeded = -1;
    if (valid && hint >= 0) {
        const float *ts = D.tri_sphere + 4 * hint;
        if (node_sdf(D, A, bvec, ts) < ts[3] + eps) {
            float lv[3][3], fv[3];
            local_vertices(D, hint, A, bvec, lv);
            for (int m = 0; m < 3; ++m) {
                fv[m] = sdf_cyl(lv[m][0], lv[m][1], lv[m][2], D.r, D.L, nullptr);
                UB = fminf(UB, fv[m]);
            }
            float u, v, dk;
            if (!tri_min_shortcut(lv[0], lv[1], lv[2], fv, D.r, D.L, &dk, &u, &v))
                dk = tri_min_search(lv[0], lv[1], lv[2], D.r, D.L, D.tri_iters, &u, &v);
            best = dk;
            bt = seeded = hint;
            const float w0 = 1.f - u - v;
            for (int c = 0; c < 3; ++c) bx[c] = fmaf(w0, lv[0][c], fmaf(u, lv[1][c], v * lv[2][c]));
        }
    }
    {
        int sp = 0;
        const float lim0 = valid ? INFINITY : -INFINITY;
        {
            const BvhNode &rt = D.nodes[0];
            float fc = node_sdf(D, A, bvec, rt.c);
            float lb = fc - rt.rad;
            bool need = valid && fc < rt.rad + eps && !(lb > lim0);   // Eq. (21)
            if (__any_sync(0xFFFFFFFFu, need)) {
                sn[0] = 0;
                sl[0] = -INFINITY;
                sp = 1;
            }
        }
        while (sp > 0) {
            --sp;
            const int ni = sn[sp];
            const float lbw = sl[sp];
            const float lim = valid ? fminf(UB, best) : -INFINITY;
            // the bound stored with the node is the smallest over the lanes
            if (!__any_sync(0xFFFFFFFFu, valid && !(lbw > lim))) continue;
            const BvhNode nd = D.nodes[ni];
            if (nd.left < 0) {
                for (int k = 0; k < nd.count; ++k) {
                    const int t = D.tri_order[nd.right + k];
                    const float *ts = D.tri_sphere + 4 * t;
                    const float ft = node_sdf(D, A, bvec, ts);
                    const float limt = valid ? fminf(UB, best) : -INFINITY;
                    bool cand = valid && t != seeded && ft < ts[3] + eps && !(ft - ts[3] > limt);   // Eq. (21)
                    if (!__any_sync(0xFFFFFFFFu, cand)) continue;
                    float lv[3][3];
                    local_vertices(D, t, A, bvec, lv);
                    float fv[3] = {0.f, 0.f, 0.f};
                    if (cand) {
                        for (int m = 0; m < 3; ++m) {
                            fv[m] = sdf_cyl(lv[m][0], lv[m][1], lv[m][2], D.r, D.L, nullptr);
                            UB = fminf(UB, fv[m]);
                        }
                    }
                    float lbt = cand ? lin_lower_bound(lv, D.r, D.L) : INFINITY;
                    if (cand && lbt > fminf(UB, best)) cand = false;
                    if (cand && nc < QC) {
                        int k = nc++;
                        while (k > 0 && cl[k - 1] > lbt) {   // insertion in lower-bound order
                            ct[k] = ct[k - 1];
                            cl[k] = cl[k - 1];
                            --k;
                        }
                        ct[k] = t;
                        cl[k] = lbt;
                        cand = false;
                    }
                    if (cand) {
                        float u, v, dk;
                        bool done = tri_min_shortcut(lv[0], lv[1], lv[2], fv, D.r, D.L, &dk, &u, &v);
                        if (!done && nq < QN) {
                            // searched later, together with the other lanes' searches
                            qt[nq] = t;
                            ql[nq++] = lbt;
                        } else {
                            if (!done) dk = tri_min_search(lv[0], lv[1], lv[2], D.r, D.L, D.tri_iters, &u, &v);
                            if (dk < best || (dk == best && t < bt)) {
                                best = dk;
                                bt = t;
                                float w0 = 1.f - u - v;
                                for (int c = 0; c < 3; ++c) bx[c] = fmaf(w0, lv[0][c], fmaf(u, lv[1][c], v * lv[2][c]));
                            }
                        }
                    }
                }
            } else if (sp + 2 <= 64) {
                const BvhNode &cl = D.nodes[nd.left];
                const BvhNode &cr = D.nodes[nd.right];
                const float fl = node_sdf(D, A, bvec, cl.c), fr = node_sdf(D, A, bvec, cr.c);
                const float bl = fl - cl.rad, br = fr - cr.rad;
                const float limc = valid ? fminf(UB, best) : -INFINITY;
                const bool nl_ = valid && fl < cl.rad + eps && !(bl > limc);   // Eq. (21)
                const bool nr_ = valid && fr < cr.rad + eps && !(br > limc);
                const bool anyl = __any_sync(0xFFFFFFFFu, nl_), anyr = __any_sync(0xFFFFFFFFu, nr_);
                // smallest bound over the lanes that need the child
                float wl = nl_ ? bl : INFINITY, wr = nr_ ? br : INFINITY;
                for (int o = 16; o > 0; o >>= 1) {
                    wl = fminf(wl, __shfl_xor_sync(0xFFFFFFFFu, wl, o));
                    wr = fminf(wr, __shfl_xor_sync(0xFFFFFFFFu, wr, o));
                }
                if (anyl && anyr) {
                    const bool lfirst = wl <= wr;
                    sn[sp] = lfirst ? nd.right : nd.left;
                    sl[sp++] = lfirst ? wr : wl;
                    sn[sp] = lfirst ? nd.left : nd.right;
                    sl[sp++] = lfirst ? wl : wr;
                } else if (anyl) {
                    sn[sp] = nd.left;
                    sl[sp++] = wl;
                } else if (anyr) {
                    sn[sp] = nd.right;
                    sl[sp++] = wr;
                }
            }
        }
    }
    // queued triangles: first-order tests slot by slot (a triangle whose lower
    // bound now exceeds the upper bound or the best minimum found cannot hold
    // the minimum), the unsettled ones to the search queue
    for (int s = 0; s < QC; ++s) {
        bool has = s < nc && !(cl[s] > fminf(UB, best));
        if (!__any_sync(0xFFFFFFFFu, has)) continue;
        if (has) {
            const int t = ct[s];
            float lv[3][3], fv[3];
            local_vertices(D, t, A, bvec, lv);
            for (int m = 0; m < 3; ++m) fv[m] = sdf_cyl(lv[m][0], lv[m][1], lv[m][2], D.r, D.L, nullptr);
            float u, v, dk;
            bool done = tri_min_shortcut(lv[0], lv[1], lv[2], fv, D.r, D.L, &dk, &u, &v);
            if (!done && nq < QN) {
                qt[nq] = t;
                ql[nq++] = cl[s];
            } else {
                if (!done) dk = tri_min_search(lv[0], lv[1], lv[2], D.r, D.L, D.tri_iters, &u, &v);
                if (dk < best || (dk == best && t < bt)) {
                    best = dk;
                    bt = t;
                    float w0 = 1.f - u - v;
                    for (int c = 0; c < 3; ++c) bx[c] = fmaf(w0, lv[0][c], fmaf(u, lv[1][c], v * lv[2][c]));
                }
            }
        }
    }
    // deferred searches, slot by slot across the warp; a triangle whose lower
    // bound now exceeds the upper bound or the best minimum found cannot hold it
    for (int s = 0; s < QN; ++s) {
        bool has = s < nq && !(ql[s] > fminf(UB, best));
        if (!__any_sync(0xFFFFFFFFu, has)) continue;
        if (has) {
            const int t = qt[s];
            float lv[3][3];
            local_vertices(D, t, A, bvec, lv);
            float u, v;
            float dk = tri_min_search(lv[0], lv[1], lv[2], D.r, D.L, D.tri_iters, &u, &v);
            if (dk < best || (dk == best && t < bt)) {
                best = dk;
                bt = t;
                float w0 = 1.f - u - v;
                for (int c = 0; c < 3; ++c) bx[c] = fmaf(w0, lv[0][c], fmaf(u, lv[1][c], v * lv[2][c]));
            }
        }
    }
    if (!valid || bt < 0) {
        *d_out = INFINITY;
        return -1;
    }
    *d_out = best;
    {
        float lv[3][3];
        local_vertices(D, bt, A, bvec, lv);
        witness_subgradient(bx, lv, D.r, D.L, nl);
    }
    for (int c = 0; c < 3; ++c) xw[c] = bx[c];
    return bt;
}

// One thread per (candidate, pose), 128 threads (REF_WARPS warps) a block.
// acc_part[((c * nblk + blk) * REF_WARPS + warp) * NACC + k];
// candidate c belongs to request grp[c] (Dt[0] when grp is null); blocks past
// a request's pose count leave zero partial sums, so a candidate's sums do not
// depend on the other requests of the launch.
template <bool GRAD>
__global__ void __launch_bounds__(128, 6)
k_refine_eval(const RefineDev *Dt, const int32_t *grp, const CandF *cands, double *acc_part, float *dist_out,
              float *wit_out, float *nrm_out, int32_t *hints, const int32_t *active)
{
    const int c = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (active && !active[c]) return;   // a finished candidate (its partials are not read)
    // the candidate's request (object mesh, trajectory, probe, parameters)
    const RefineDev D = Dt[grp ? grp[c] : 0];
    double acc[NACC];
#pragma unroll
    for (int k = 0; k < NACC; ++k) acc[k] = 0.0;
    const bool valid = i < D.P;
    {
        const CandF &cf = cands[c];
        const PoseRec &pr = D.poses[valid ? i : D.P - 1];
        // probe pose in the object frame: A = R^T R_i, b = R^T (t_i - p);
        // a mesh point m maps to probe-local A^T (m - b)
        float A[9], bvec[3];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 3; ++k)
                A[a * 3 + k] = fmaf(cf.R[0 * 3 + a], pr.Rf[0 * 3 + k], fmaf(cf.R[1 * 3 + a], pr.Rf[1 * 3 + k], cf.R[2 * 3 + a] * pr.Rf[2 * 3 + k]));
        float tp[3] = {pr.tf[0] - cf.p[0], pr.tf[1] - cf.p[1], pr.tf[2] - cf.p[2]};
        for (int a = 0; a < 3; ++a) bvec[a] = fmaf(cf.R[0 * 3 + a], tp[0], fmaf(cf.R[1 * 3 + a], tp[1], cf.R[2 * 3 + a] * tp[2]));
        float d, xl[3], nl[3];
        // hints[c][i]: the query's witness triangle of the previous evaluation (-1: none)
        int32_t *hp = hints ? hints + (size_t)c * gridDim.x * blockDim.x + i : nullptr;
        const int hint = (hp && valid) ? *hp : -1;
        int bt = dist_query(D, A, bvec, valid, hint, &d, xl, nl);
        if (hp && valid) *hp = bt;
        float n[3] = {0.f, 0.f, 0.f}, w[3] = {0.f, 0.f, 0.f};
        if (bt >= 0) {
            for (int a = 0; a < 3; ++a) {
                n[a] = fmaf(pr.Rf[a * 3 + 0], nl[0], fmaf(pr.Rf[a * 3 + 1], nl[1], pr.Rf[a * 3 + 2] * nl[2]));
                w[a] = fmaf(pr.Rf[a * 3 + 0], xl[0], fmaf(pr.Rf[a * 3 + 1], xl[1], fmaf(pr.Rf[a * 3 + 2], xl[2], pr.tf[a])));
            }
        }
        if (dist_out && valid) {
            size_t o = (size_t)c * D.P + i;
            dist_out[o] = bt >= 0 ? d : INFINITY;
            for (int a = 0; a < 3; ++a) { wit_out[3 * o + a] = w[a]; nrm_out[3 * o + a] = n[a]; }
        }
        if (bt >= 0) {
            float s, s1, s2;
            score3(D, d, &s, &s1, &s2);
            acc[0] = -(double)s;
            if (GRAD && (s1 != 0.f || s2 != 0.f)) {
                float g[6];
                for (int j = 0; j < 3; ++j) g[j] = fmaf(cf.V[0 * 3 + j], n[0], fmaf(cf.V[1 * 3 + j], n[1], cf.V[2 * 3 + j] * n[2]));
                float wc[3] = {w[0] - cf.c[0], w[1] - cf.c[1], w[2] - cf.c[2]};
                float tq[3] = {wc[1] * n[2] - wc[2] * n[1], wc[2] * n[0] - wc[0] * n[2], wc[0] * n[1] - wc[1] * n[0]};
                for (int j = 0; j < 3; ++j) {
                    float a1 = fmaf(cf.V[0 * 3 + j], tq[0], fmaf(cf.V[1 * 3 + j], tq[1], cf.V[2 * 3 + j] * tq[2]));
                    float a2 = fmaf(cf.Mc[0 * 3 + j], n[0], fmaf(cf.Mc[1 * 3 + j], n[1], cf.Mc[2 * 3 + j] * n[2]));
                    g[3 + j] = a1 + a2;
                }
                for (int j = 0; j < 6; ++j) acc[1 + j] = -(double)s1 * (double)g[j];
                double wgt = s2 < 0.f ? -(double)s2 : 0.0;
                int k = 7;
                for (int a = 0; a < 6; ++a)
                    for (int b = a; b < 6; ++b) acc[k++] = wgt * (double)g[a] * (double)g[b];
            }
        }
    }
    // warp sums in a fixed order, one partial per warp (no block barrier: the
    // warps of a block finish at different times)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *dst = acc_part + (((size_t)c * gridDim.x + blockIdx.x) * REF_WARPS + warp) * NACC;
#pragma unroll
    for (int k = 0; k < NACC; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
        if (lane == 0) dst[k] = v;
    }
}

// ---------------------------------------------------------------------------
// FP64 per-candidate step
// ---------------------------------------------------------------------------
__device__ void vcoef(double th, double *a, double *b, double *da, double *db)
{
    if (th < 1e-4) {
        double t2 = th * th;
        *a = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
        *b = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
        *da = -1.0 / 12.0 + t2 / 180.0;
        *db = -1.0 / 60.0 + t2 / 1260.0;
    } else {
        double s = sin(th), c = cos(th);
        *a = (1.0 - c) / (th * th);
        *b = (th - s) / (th * th * th);
        *da = (th * s - 2.0 * (1.0 - c)) / (th * th * th * th);
        *db = ((1.0 - c) * th - 3.0 * (th - s)) / (th * th * th * th * th);
    }
}

// pose T(xi) (Eq. (14)-(17)) and the derivative data of the next evaluation
__device__ void cand_from_state(const double *st, CandF *out)
{
    const double *R0 = st, *p0 = st + 9, *an = st + 12, *xi = st + 15;
    const double *u = xi, *w = xi + 3;
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double a, b, da, db;
    vcoef(th, &a, &b, &da, &db);
    double sA = th < 1e-4 ? 1.0 - th * th / 6.0 + th * th * th * th / 120.0 : sin(th) / th;
    double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    double K2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) K2[3 * i + j] = K[3 * i] * K[j] + K[3 * i + 1] * K[3 + j] + K[3 * i + 2] * K[6 + j];
    double dR[9], V[9];
    for (int k = 0; k < 9; ++k) {
        double I = (k % 4 == 0) ? 1.0 : 0.0;
        dR[k] = I + sA * K[k] + a * K2[k];
        V[k] = I + a * K[k] + b * K2[k];
    }
    double R[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[3 * i + j] = dR[3 * i] * R0[j] + dR[3 * i + 1] * R0[3 + j] + dR[3 * i + 2] * R0[6 + j];
    double Ra[3], dRRa[3], Vu[3];
    for (int i = 0; i < 3; ++i) Ra[i] = R0[3 * i] * an[0] + R0[3 * i + 1] * an[1] + R0[3 * i + 2] * an[2];
    for (int i = 0; i < 3; ++i) dRRa[i] = dR[3 * i] * Ra[0] + dR[3 * i + 1] * Ra[1] + dR[3 * i + 2] * Ra[2];
    for (int i = 0; i < 3; ++i) Vu[i] = V[3 * i] * u[0] + V[3 * i + 1] * u[1] + V[3 * i + 2] * u[2];
    // d(V u)/dw = -a [u]x + (w x u) (a'/th) w^T + b((w.u) I + w u^T - 2 u w^T) + (w x (w x u)) (b'/th) w^T
    double wxu[3] = {w[1] * u[2] - w[2] * u[1], w[2] * u[0] - w[0] * u[2], w[0] * u[1] - w[1] * u[0]};
    double wd = w[0] * u[0] + w[1] * u[1] + w[2] * u[2], ww = th * th;
    double wxwxu[3];
    for (int k = 0; k < 3; ++k) wxwxu[k] = w[k] * wd - u[k] * ww;
    double Ku[9] = {0.0, -u[2], u[1], u[2], 0.0, -u[0], -u[1], u[0], 0.0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double I = (i == j) ? 1.0 : 0.0;
            double t1 = -a * Ku[3 * i + j] + wxu[i] * da * w[j];
            double t2 = b * ((wd * I + w[i] * u[j]) - 2.0 * u[i] * w[j]) + wxwxu[i] * db * w[j];
            out->Mc[3 * i + j] = (float)(t1 + t2);
        }
    for (int k = 0; k < 9; ++k) { out->R[k] = (float)R[k]; out->V[k] = (float)V[k]; }
    for (int i = 0; i < 3; ++i) {
        out->p[i] = (float)(((p0[i] + Vu[i]) + Ra[i]) - dRRa[i]);
        out->c[i] = (float)((p0[i] + Vu[i]) + Ra[i]);
    }
}

__device__ bool chol6(const double *H, const double *b, double *x)
{
    double L[36];
    for (int i = 0; i < 36; ++i) L[i] = 0.0;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = H[6 * i + j];
            for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[6 * i + i] = sqrt(s);
            } else {
                L[6 * i + j] = s / L[6 * j + j];
            }
        }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
        y[i] = s / L[6 * i + i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];
        x[i] = s / L[6 * i + i];
    }
    return true;
}

// prm: lambda, mu, step_t, step_r, b_t, b_r
// mode 0: only refresh the candidate data from the state
// mode 1: sum the partials, record J, take one projected Gauss-Newton step
// mode 2: sum the partials and record J (final evaluation)
__global__ void k_refine_solve(int K, int nblk, double *state, const double *acc_part, const double *prm, int mode,
                               CandF *cands)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    double *st = state + (size_t)c * ST;
    double *xi = st + 15;
    if (mode != 0) {
        double acc[NACC];
        for (int k = 0; k < NACC; ++k) acc[k] = 0.0;
        for (int q = 0; q < nblk; ++q)
            for (int k = 0; k < NACC; ++k) acc[k] += acc_part[((size_t)c * nblk + q) * NACC + k];
        const double lam = prm[0], mu = prm[1];
        double xx = 0.0;
        for (int j = 0; j < 6; ++j) xx += xi[j] * xi[j];
        st[21] = acc[0] + lam * xx;   // J (Eq. (19))
        if (mode == 1) {
            double G[6], H[36];
            for (int j = 0; j < 6; ++j) G[j] = acc[1 + j] + 2.0 * lam * xi[j];
            int k = 7;
            for (int a = 0; a < 6; ++a)
                for (int b = a; b < 6; ++b) { H[6 * a + b] = acc[k]; H[6 * b + a] = acc[k]; ++k; }
            for (int j = 0; j < 6; ++j) H[7 * j] += 2.0 * lam + mu;
            double nb[6], dl[6];
            for (int j = 0; j < 6; ++j) nb[j] = -G[j];
            if (chol6(H, nb, dl)) {
                double mt = 0.0, mr = 0.0;
                for (int j = 0; j < 3; ++j) { mt = fmax(mt, fabs(dl[j])); mr = fmax(mr, fabs(dl[3 + j])); }
                double sc = 1.0;
                if (mt > prm[2]) sc = fmin(sc, prm[2] / mt);
                if (mr > prm[3]) sc = fmin(sc, prm[3] / mr);
                for (int j = 0; j < 6; ++j) {
                    double v = xi[j] + sc * dl[j];
                    double bb = j < 3 ? prm[4] : prm[5];
                    if (v > bb) v = bb;
                    if (v < -bb) v = -bb;
                    xi[j] = v;
                }
            }
        }
    }
    cand_from_state(st, &cands[c]);
}

// ---------------------------------------------------------------------------
// L-BFGS-B (Sec. V-C as printed): one thread per candidate, FP64.  A round
// evaluates J and grad J (Eq. (19), (28)) at every active candidate's trial
// twist; this kernel then accepts or backtracks the step (Armijo), updates the
// limited-memory pairs (s, y) and builds the next trial.  The direction is the
// two-loop recursion on the variables that are not held at a bound of
// Eq. (20) (a variable is held when it sits on its bound and the gradient
// pushes it outward), steps are projected onto the box and backtracked by
// safeguarded quadratic interpolation (first step of unit length, as in
// L-BFGS-B; later ones start at alpha = 1), and a candidate stops
// when the projected gradient or the relative decrease of J is below its
// tolerance, after max_iter accepted steps, or when backtracking fails.
// ---------------------------------------------------------------------------
enum {
    LB_X = 0, LB_F = 6, LB_G = 7, LB_D = 13, LB_ALPHA = 19, LB_GTD = 20, LB_ITER = 21, LB_NBACK = 22,
    LB_NH = 23, LB_HEAD = 24, LB_STATUS = 25, LB_NEV = 26, LB_HIST = 32
};
constexpr int LB_S = LB_HIST, LB_Y = LB_HIST + 6 * LB_M, LB_RHO = LB_HIST + 12 * LB_M;
static_assert(LB_RHO + LB_M <= LB_ST, "L-BFGS state");

__device__ __forceinline__ double lb_hi(int j, const double *prm) { return j < 3 ? prm[4] : prm[5]; }

__device__ __forceinline__ double lb_clamp(double v, double hi) { return v > hi ? hi : (v < -hi ? -hi : v); }

__device__ __forceinline__ bool lb_held(const double *x, const double *g, int j, const double *prm)
{
    const double hi = lb_hi(j, prm);
    return (x[j] <= -hi && g[j] > 0.0) || (x[j] >= hi && g[j] < 0.0);
}

// d = -H g on the free variables (two-loop recursion over the stored pairs)
__device__ void lb_direction(double *L, const double *prm)
{
    const double *x = L + LB_X, *g = L + LB_G;
    double *d = L + LB_D;
    const int nh = (int)L[LB_NH], head = (int)L[LB_HEAD];
    double q[6], al[LB_M];
    for (int j = 0; j < 6; ++j) q[j] = lb_held(x, g, j, prm) ? 0.0 : g[j];
    for (int k = 0; k < nh; ++k) {
        const int i = (head - 1 - k + 2 * LB_M) % LB_M;
        const double *S = L + LB_S + 6 * i, *Y = L + LB_Y + 6 * i;
        double a = 0.0;
        for (int j = 0; j < 6; ++j) a += S[j] * q[j];
        a *= L[LB_RHO + i];
        al[k] = a;
        for (int j = 0; j < 6; ++j) q[j] -= a * Y[j];
    }
    double gam = 1.0;
    if (nh > 0) {
        const int i = (head - 1 + LB_M) % LB_M;
        const double *S = L + LB_S + 6 * i, *Y = L + LB_Y + 6 * i;
        double sy = 0.0, yy = 0.0;
        for (int j = 0; j < 6; ++j) { sy += S[j] * Y[j]; yy += Y[j] * Y[j]; }
        gam = sy / yy;
    }
    for (int j = 0; j < 6; ++j) q[j] *= gam;
    for (int k = nh - 1; k >= 0; --k) {
        const int i = (head - 1 - k + 2 * LB_M) % LB_M;
        const double *S = L + LB_S + 6 * i, *Y = L + LB_Y + 6 * i;
        double b = 0.0;
        for (int j = 0; j < 6; ++j) b += Y[j] * q[j];
        b *= L[LB_RHO + i];
        for (int j = 0; j < 6; ++j) q[j] += S[j] * (al[k] - b);
    }
    double gd = 0.0;
    for (int j = 0; j < 6; ++j) {
        d[j] = lb_held(x, g, j, prm) ? 0.0 : -q[j];
        gd += g[j] * d[j];
    }
    if (!(gd < 0.0)) {   // not a descent direction: forget the pairs, steepest descent
        L[LB_NH] = 0.0;
        for (int j = 0; j < 6; ++j) d[j] = lb_held(x, g, j, prm) ? 0.0 : -g[j];
    }
}

// trial twist x + alpha d projected onto the box; false when it does not move
__device__ bool lb_trial(double *L, double *xi, const double *prm)
{
    const double *x = L + LB_X, *g = L + LB_G, *d = L + LB_D;
    double gtd = 0.0, mv = 0.0;
    for (int j = 0; j < 6; ++j) {
        xi[j] = lb_clamp(x[j] + L[LB_ALPHA] * d[j], lb_hi(j, prm));
        gtd += g[j] * (xi[j] - x[j]);
        mv = fmax(mv, fabs(xi[j] - x[j]));
    }
    L[LB_GTD] = gtd;
    return mv > 0.0 && gtd < 0.0;
}

__device__ void lb_new_step(double *L, double *xi, const double *prm)
{
    lb_direction(L, prm);
    double dn = 0.0;
    for (int j = 0; j < 6; ++j) dn += L[LB_D + j] * L[LB_D + j];
    dn = sqrt(dn);
    L[LB_ALPHA] = (L[LB_NH] == 0.0 && dn > 1.0) ? 1.0 / dn : 1.0;
    L[LB_NBACK] = 0.0;
    if (!lb_trial(L, xi, prm)) L[LB_STATUS] = 1.0;
}

// prm: lambda, mu, step_t, step_r, b_t, b_r, pgtol, ftol, max_iter
// phase 0: start at xi = 0; phase 1: take the round's evaluation; phase 2:
// leave every candidate at its last accepted twist (J, iterations and
// evaluations in the state's slots 21, 22, 23)
__global__ void k_lbfgs(int K, int nblk, double *state, const double *acc_part, const double *prm, double *lbs,
                        int32_t *active, CandF *cands, int phase)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    double *st = state + (size_t)c * ST, *xi = st + 15, *L = lbs + (size_t)c * LB_ST;
    if (phase == 0) {
        for (int k = 0; k < LB_ST; ++k) L[k] = 0.0;
        L[LB_ITER] = -1.0;
        for (int j = 0; j < 6; ++j) xi[j] = 0.0;
        active[c] = 1;
    } else if (phase == 1) {
        if (L[LB_STATUS] != 0.0) {
            active[c] = 0;
            return;
        }
        double acc[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int q = 0; q < nblk; ++q)
            for (int k = 0; k < 7; ++k) acc[k] += acc_part[((size_t)c * nblk + q) * NACC + k];
        const double lam = prm[0];
        double xx = 0.0;
        for (int j = 0; j < 6; ++j) xx += xi[j] * xi[j];
        const double ft = acc[0] + lam * xx;
        double gt[6];
        for (int j = 0; j < 6; ++j) gt[j] = acc[1 + j] + 2.0 * lam * xi[j];
        L[LB_NEV] += 1.0;
        bool take = false;
        if (L[LB_ITER] < 0.0) {
            take = true;   // the starting point
        } else if (isfinite(ft) && ft <= L[LB_F] + 1e-4 * L[LB_GTD]) {
            take = true;
        }
        if (take) {
            const bool first = L[LB_ITER] < 0.0;
            const double fold = L[LB_F];
            if (!first) {
                double s[6], y[6], sy = 0.0, yy = 0.0;
                for (int j = 0; j < 6; ++j) {
                    s[j] = xi[j] - L[LB_X + j];
                    y[j] = gt[j] - L[LB_G + j];
                    sy += s[j] * y[j];
                    yy += y[j] * y[j];
                }
                if (sy > 1e-12 * yy) {
                    const int i = (int)L[LB_HEAD];
                    for (int j = 0; j < 6; ++j) { L[LB_S + 6 * i + j] = s[j]; L[LB_Y + 6 * i + j] = y[j]; }
                    L[LB_RHO + i] = 1.0 / sy;
                    L[LB_HEAD] = (double)((i + 1) % LB_M);
                    L[LB_NH] = fmin((double)LB_M, L[LB_NH] + 1.0);
                }
            }
            for (int j = 0; j < 6; ++j) { L[LB_X + j] = xi[j]; L[LB_G + j] = gt[j]; }
            L[LB_F] = ft;
            L[LB_ITER] = first ? 0.0 : L[LB_ITER] + 1.0;
            double pg = 0.0;
            for (int j = 0; j < 6; ++j) pg = fmax(pg, fabs(lb_clamp(xi[j] - gt[j], lb_hi(j, prm)) - xi[j]));
            const bool conv = pg <= prm[6] ||
                              (!first && fold - ft <= prm[7] * fmax(fmax(fabs(fold), fabs(ft)), 1.0)) ||
                              L[LB_ITER] >= prm[8];
            if (conv) L[LB_STATUS] = 1.0;
            else lb_new_step(L, xi, prm);
        } else {
            // backtrack to the minimiser of the quadratic through f, the
            // slope gtd and the trial value, kept within [0.1, 0.5] of the step
            const double gtd = L[LB_GTD], dphi = ft - L[LB_F];
            double t = (isfinite(ft) && dphi - gtd > 0.0) ? -gtd / (2.0 * (dphi - gtd)) : 0.1;
            t = fmin(fmax(t, 0.1), 0.5);
            L[LB_NBACK] += 1.0;
            L[LB_ALPHA] *= t;
            if (L[LB_NBACK] > 30.0 || !lb_trial(L, xi, prm)) L[LB_STATUS] = 1.0;
        }
        if (L[LB_STATUS] != 0.0) {
            for (int j = 0; j < 6; ++j) xi[j] = L[LB_X + j];
            active[c] = 0;
        }
    } else {
        if (L[LB_ITER] >= 0.0)
            for (int j = 0; j < 6; ++j) xi[j] = L[LB_X + j];
        st[21] = L[LB_F];
        st[22] = fmax(L[LB_ITER], 0.0);
        st[23] = L[LB_NEV];
        active[c] = 0;
    }
    cand_from_state(st, &cands[c]);
}

cudaError_t launch_lbfgs(int K, int nblk, double *state, const double *acc_part, const double *prm, double *lbs,
                         int32_t *active, CandF *cands, int phase, cudaStream_t st)
{
    k_lbfgs<<<(K + 63) / 64, 64, 0, st>>>(K, nblk, state, acc_part, prm, lbs, active, cands, phase);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_refine_eval(const RefineDev *Dt, const int32_t *grp, int K, int nblk, const CandF *cands,
                               double *acc_part, bool grad, float *dist_out, float *wit_out, float *nrm_out,
                               cudaStream_t st, int32_t *hints, const int32_t *active)
{
    dim3 grid(nblk, K);
    if (grad)
        k_refine_eval<true><<<grid, 128, 0, st>>>(Dt, grp, cands, acc_part, dist_out, wit_out, nrm_out, hints, active);
    else
        k_refine_eval<false><<<grid, 128, 0, st>>>(Dt, grp, cands, acc_part, dist_out, wit_out, nrm_out, hints, active);
    return cudaGetLastError();
}

cudaError_t launch_refine_solve(int K, int nblk, double *state, const double *acc_part, const double *prm, int mode,
                                CandF *cands, cudaStream_t st)
{
    k_refine_solve<<<(K + 63) / 64, 64, 0, st>>>(K, nblk, state, acc_part, prm, mode, cands);
    return cudaGetLastError();
}

size_t cand_bytes() { return sizeof(CandF); }

// Twists from a device FP32 array into the state (the differentiable form).
__global__ void k_set_xi(int B, const float *xi, double *state)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    for (int j = 0; j < 6; ++j) state[(size_t)b * ST + 15 + j] = (double)xi[6 * b + j];
}

// J[b] and grad[b] (Eq. (19), (28)) from the partials.
__global__ void k_finish_objective(int B, int nblk, const double *state, const double *acc_part, double lam, float *J,
                                   float *grad, const float *gJ)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double *xi = state + (size_t)b * ST + 15;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int q = 0; q < nblk; ++q)
        for (int k = 0; k < 7; ++k) acc[k] += acc_part[((size_t)b * nblk + q) * NACC + k];
    double xx = 0.0;
    for (int j = 0; j < 6; ++j) xx += xi[j] * xi[j];
    if (J) J[b] = (float)(acc[0] + lam * xx);
    if (grad) {
        double sc = gJ ? (double)gJ[b] : 1.0;
        for (int j = 0; j < 6; ++j) grad[6 * b + j] = (float)(sc * (acc[1 + j] + 2.0 * lam * xi[j]));
    }
}

cudaError_t launch_set_xi(int B, const float *xi, double *state, cudaStream_t st)
{
    k_set_xi<<<(B + 63) / 64, 64, 0, st>>>(B, xi, state);
    return cudaGetLastError();
}

cudaError_t launch_finish_objective(int B, int nblk, const double *state, const double *acc_part, double lam, float *J,
                                    float *grad, const float *gJ, cudaStream_t st)
{
    k_finish_objective<<<(B + 63) / 64, 64, 0, st>>>(B, nblk, state, acc_part, lam, J, grad, gJ);
    return cudaGetLastError();
}

}  // namespace dock
