/*
 * FP64 CPU oracle for probe-aware contact registration by complementary-shape
 * docking.  TEST INFRASTRUCTURE ONLY: called by tests/, by the smoke check and
 * by the bench's CPU-baseline leg, never by the product path.  It shares no
 * code with the CUDA library.
 *
 * Compile with -O2 -ffp-contract=off: every floating-point expression below is
 * evaluated exactly as written (no fused multiply-add), which is what makes
 * the bit-exact comparisons of voxel decisions meaningful.
 *
 * Contents (paper section / equation each function follows):
 *   orc_quat_to_mat      Hamilton rotation matrix of a unit quaternion
 *   orc_object_grid      Sec. IV-A.1, Eq. (1)-(4): banded template O_t of the
 *                        watertight-mesh SDF, touchable mask O_m, O = min(O_t,O_m)
 *                        sampled at h k + o_o.  SDF = exact point-triangle
 *                        distance, sign = parity of +x ray crossings.
 *   orc_sweep_grid       Sec. IV-A.2, Eq. (5)-(6): binary swept occupancy of the
 *                        probe along the trajectory, on a lattice rotated by R.
 *   orc_sweep_grid_sel   the same over a subset of the poses (contact or
 *                        non-contact labels), on the lattice of all poses.
 *   orc_rotate_object    Sec. IV-D: O rotated by R and resampled by trilinear
 *                        interpolation (the paper's own rotation mechanism).
 *   orc_probe_sdf        Sec. V-B: flat-ended cylinder SDF f_p and its gradient.
 *   orc_tri_min          Sec. V-B: minimum of f_p over a triangle (bisection
 *                        inside golden-section search; see the function).
 *   orc_objective        Sec. V-A/C, Eq. (13)-(28): J(xi), grad J(xi) and the
 *                        Gauss-Newton matrix for one candidate pose.
 *   orc_refine           Sec. V-C: fixed-iteration projected Gauss-Newton on
 *                        Eq. (20) with an FP64 6x6 Cholesky solve.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------ */
/* rotations                                                           */
/* ------------------------------------------------------------------ */

ORC_API void orc_quat_to_mat(const double *q, double *R)
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

/* ------------------------------------------------------------------ */
/* point-triangle distance: closest point by Voronoi regions of the    */
/* triangle (vertex, edge, face), the textbook construction            */
/* ------------------------------------------------------------------ */

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the parallel per-pose loops (1 = serial; results do not depend on it). */
ORC_API void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

ORC_API int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static double dot3(const double *a, const double *b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

static double pt_tri_dist2(const double *p, const double *a, const double *b, const double *c)
{
    double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double ac[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    double q[3];
    double d1 = dot3(ab, ap), d2 = dot3(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) { q[0] = a[0]; q[1] = a[1]; q[2] = a[2]; goto done; }
    double bp[3] = {p[0] - b[0], p[1] - b[1], p[2] - b[2]};
    double d3 = dot3(ab, bp), d4 = dot3(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) { q[0] = b[0]; q[1] = b[1]; q[2] = b[2]; goto done; }
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
        double v = d1 / (d1 - d3);
        q[0] = a[0] + v * ab[0]; q[1] = a[1] + v * ab[1]; q[2] = a[2] + v * ab[2];
        goto done;
    }
    double cp[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
    double d5 = dot3(ab, cp), d6 = dot3(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) { q[0] = c[0]; q[1] = c[1]; q[2] = c[2]; goto done; }
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        double w = d2 / (d2 - d6);
        q[0] = a[0] + w * ac[0]; q[1] = a[1] + w * ac[1]; q[2] = a[2] + w * ac[2];
        goto done;
    }
    double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0) {
        double w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        q[0] = b[0] + w * (c[0] - b[0]); q[1] = b[1] + w * (c[1] - b[1]); q[2] = b[2] + w * (c[2] - b[2]);
        goto done;
    }
    {
        double denom = 1.0 / ((va + vb) + vc);
        double v = vb * denom, w = vc * denom;
        q[0] = (a[0] + ab[0] * v) + ac[0] * w;
        q[1] = (a[1] + ab[1] * v) + ac[1] * w;
        q[2] = (a[2] + ab[2] * v) + ac[2] * w;
    }
done:;
    double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    return (dx * dx + dy * dy) + dz * dz;
}

ORC_API double orc_pt_tri_dist2(const double *p, const double *a, const double *b, const double *c)
{
    return pt_tri_dist2(p, a, b, c);
}

/* ------------------------------------------------------------------ */
/* +x ray / triangle crossing with simulation-of-simplicity ties       */
/* ------------------------------------------------------------------ */

/* Sign of the 2-D edge function of (a->b) at p in the (y,z) plane, with the
 * point perturbed to (y + eps, z + eps^2) so that it never lies on an edge. */
static int edge_sign(double ay, double az, double by, double bz, double py, double pz, double *val)
{
    double e = (by - ay) * (pz - az) - (bz - az) * (py - ay);
    *val = e;
    if (e > 0.0) return 1;
    if (e < 0.0) return -1;
    double dz = bz - az;
    if (dz != 0.0) return dz > 0.0 ? -1 : 1;
    double dy = by - ay;
    if (dy != 0.0) return dy > 0.0 ? 1 : -1;
    return 0;
}

/* Returns 1 and the crossing x when the line {(t, py, pz)} crosses the
 * triangle (v0, v1, v2). */
static int ray_cross(const double *v0, const double *v1, const double *v2, double py, double pz, double *xc)
{
    double e0, e1, e2;
    int s0 = edge_sign(v1[1], v1[2], v2[1], v2[2], py, pz, &e0);
    int s1 = edge_sign(v2[1], v2[2], v0[1], v0[2], py, pz, &e1);
    int s2 = edge_sign(v0[1], v0[2], v1[1], v1[2], py, pz, &e2);
    if (s0 == 0 || s0 != s1 || s1 != s2) return 0;
    double den = (e0 + e1) + e2;
    if (den == 0.0) return 0;
    *xc = ((e0 * v0[0] + e1 * v1[0]) + e2 * v2[0]) / den;
    return 1;
}

/* ------------------------------------------------------------------ */
/* object grid, Eq. (1)-(4)                                            */
/* ------------------------------------------------------------------ */

static double lattice_origin(double c, double h, int32_t N)
{
    return h * round(c / h) - (double)(N / 2) * h;
}

typedef struct { int64_t *start; int32_t *items; int64_t n; } bins_t;

/* Bin triangles into uniform cells (3-D if nd==3, (y,z) 2-D if nd==2). */
static void build_bins(bins_t *B, const double *V, const int32_t *T, int64_t nt, const uint8_t *use,
                       const double *org, double cs, const int64_t *dims, int nd, double pad)
{
    int64_t ncell = dims[0] * dims[1] * (nd == 3 ? dims[2] : 1);
    int64_t *cnt = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            int64_t acc = 0;
            for (int64_t c = 0; c < ncell; ++c) { int64_t k = cnt[c]; cnt[c] = acc; acc += k; }
            cnt[ncell] = acc;
            B->start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
            memcpy(B->start, cnt, sizeof(int64_t) * (size_t)(ncell + 1));
            B->items = (int32_t *)malloc(sizeof(int32_t) * (size_t)(acc > 0 ? acc : 1));
            B->n = ncell;
        }
        for (int64_t t = 0; t < nt; ++t) {
            if (use && !use[t]) continue;
            double lo[3], hi[3];
            for (int a = 0; a < 3; ++a) {
                double x0 = V[3 * T[3 * t] + a], x1 = V[3 * T[3 * t + 1] + a], x2 = V[3 * T[3 * t + 2] + a];
                lo[a] = fmin(x0, fmin(x1, x2)) - pad;
                hi[a] = fmax(x0, fmax(x1, x2)) + pad;
            }
            int64_t i0[3], i1[3];
            int ok = 1;
            for (int d = 0; d < nd; ++d) {
                int a = (nd == 3) ? d : d + 1;
                i0[d] = (int64_t)floor((lo[a] - org[d]) / cs);
                i1[d] = (int64_t)floor((hi[a] - org[d]) / cs);
                if (i0[d] < 0) i0[d] = 0;
                if (i1[d] > dims[d] - 1) i1[d] = dims[d] - 1;
                if (i0[d] > i1[d]) ok = 0;
            }
            if (!ok) continue;
            if (nd == 2) { i0[2] = 0; i1[2] = 0; }
            for (int64_t a = i0[0]; a <= i1[0]; ++a)
                for (int64_t b = i0[1]; b <= i1[1]; ++b)
                    for (int64_t c = i0[2]; c <= i1[2]; ++c) {
                        int64_t cell = (nd == 3) ? (c * dims[1] + b) * dims[0] + a : b * dims[0] + a;
                        if (pass == 0) cnt[cell]++;
                        else B->items[cnt[cell]++] = (int32_t)t;
                    }
        }
    }
    free(cnt);
}

static void free_bins(bins_t *B) { free(B->start); free(B->items); }

/*
 * O[(kz*N + ky)*N + kx] = O(h k + o_o), Eq. (4).
 *   f  = signed distance to the watertight mesh: exact point-triangle distance,
 *        negative inside (odd number of +x ray crossings).
 *   O_t = Eq. (1): 1 - f/tau_out on [0, tau_out); 1 + f/tau_in on (-tau_in, 0);
 *         deep_value for f <= -tau_in; 0 otherwise.
 *   O_m = Eq. (2): max(0, 1 - d/tau_out), d = unsigned distance to the
 *         touchable triangles (all triangles when touch == NULL).
 *   O   = Eq. (3): min(O_t, O_m).
 * Distances beyond max(tau_out, tau_in) never change O, so only triangles
 * within that cutoff are examined.  Returns 0, or -1 if the mesh AABB widened
 * by tau_out does not lie inside the lattice.
 */
ORC_API int orc_object_grid(const double *V, int64_t nv, const int32_t *T, int64_t nt, const uint8_t *touch,
                            double h, int32_t N, double tau_out, double tau_in, double deep_value,
                            double *origin, double *O, double *f_out)
{
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nv; ++i)
        for (int a = 0; a < 3; ++a) { mn[a] = fmin(mn[a], V[3 * i + a]); mx[a] = fmax(mx[a], V[3 * i + a]); }
    int fits = 1;
    for (int a = 0; a < 3; ++a) {
        double c = (mn[a] + mx[a]) * 0.5;
        origin[a] = lattice_origin(c, h, N);
        if (mn[a] - tau_out < origin[a] || mx[a] + tau_out > origin[a] + (double)(N - 1) * h) fits = 0;
    }
    double cut = tau_out > tau_in ? tau_out : tau_in;
    double cut2 = cut * cut;
    /* 3-D bins for the distance query */
    double cs = cut > h ? cut : h;
    int64_t dims[3];
    for (int a = 0; a < 3; ++a) dims[a] = (int64_t)ceil(((double)(N - 1) * h) / cs) + 1;
    bins_t B3, B3t, B2;
    build_bins(&B3, V, T, nt, NULL, origin, cs, dims, 3, cut);
    if (touch) build_bins(&B3t, V, T, nt, touch, origin, cs, dims, 3, cut);
    /* 2-D (y,z) bins for the ray crossings */
    double org2[2] = {origin[1], origin[2]};
    int64_t dims2[2] = {dims[1], dims[2]};
    build_bins(&B2, V, T, nt, NULL, org2, cs, dims2, 2, 0.0);
    double *xc = (double *)malloc(sizeof(double) * (size_t)(nt > 0 ? nt : 1));

    for (int32_t kz = 0; kz < N; ++kz) {
        for (int32_t ky = 0; ky < N; ++ky) {
            double py = h * (double)ky + origin[1];
            double pz = h * (double)kz + origin[2];
            /* crossings of this row's line with the mesh */
            int64_t ncross = 0;
            int64_t cy = (int64_t)floor((py - org2[0]) / cs), cz = (int64_t)floor((pz - org2[1]) / cs);
            if (cy >= 0 && cy < dims2[0] && cz >= 0 && cz < dims2[1]) {
                int64_t cell = cz * dims2[0] + cy;
                for (int64_t k = B2.start[cell]; k < B2.start[cell + 1]; ++k) {
                    int32_t t = B2.items[k];
                    double xx;
                    if (ray_cross(V + 3 * T[3 * t], V + 3 * T[3 * t + 1], V + 3 * T[3 * t + 2], py, pz, &xx))
                        xc[ncross++] = xx;
                }
            }
            for (int32_t kx = 0; kx < N; ++kx) {
                double p[3] = {h * (double)kx + origin[0], py, pz};
                int64_t cx = (int64_t)floor((p[0] - origin[0]) / cs);
                int64_t cyy = (int64_t)floor((p[1] - origin[1]) / cs);
                int64_t czz = (int64_t)floor((p[2] - origin[2]) / cs);
                int64_t cell = (czz * dims[1] + cyy) * dims[0] + cx;
                double best = INFINITY, bestt = INFINITY;
                for (int64_t k = B3.start[cell]; k < B3.start[cell + 1]; ++k) {
                    int32_t t = B3.items[k];
                    double d2 = pt_tri_dist2(p, V + 3 * T[3 * t], V + 3 * T[3 * t + 1], V + 3 * T[3 * t + 2]);
                    if (d2 < best) best = d2;
                }
                if (touch) {
                    for (int64_t k = B3t.start[cell]; k < B3t.start[cell + 1]; ++k) {
                        int32_t t = B3t.items[k];
                        double d2 = pt_tri_dist2(p, V + 3 * T[3 * t], V + 3 * T[3 * t + 1], V + 3 * T[3 * t + 2]);
                        if (d2 < bestt) bestt = d2;
                    }
                } else {
                    bestt = best;
                }
                int par = 0;
                for (int64_t c = 0; c < ncross; ++c) if (xc[c] > p[0]) par ^= 1;
                double D = best < cut2 ? sqrt(best) : INFINITY;
                double Dt = bestt < cut2 ? sqrt(bestt) : INFINITY;
                double f = par ? -D : D;
                double Ot;
                if (0.0 <= f && f < tau_out) Ot = 1.0 - f / tau_out;
                else if (-tau_in < f && f < 0.0) Ot = 1.0 + f / tau_in;
                else if (f <= -tau_in) Ot = deep_value;
                else Ot = 0.0;
                double Om = 1.0 - Dt / tau_out;
                if (!(Om > 0.0)) Om = 0.0;
                double o = Ot < Om ? Ot : Om;
                int64_t idx = ((int64_t)kz * N + ky) * N + kx;
                O[idx] = o;
                if (f_out) f_out[idx] = f;
            }
        }
    }
    free(xc);
    free_bins(&B3);
    if (touch) free_bins(&B3t);
    free_bins(&B2);
    return fits ? 0 : -1;
}

/* ------------------------------------------------------------------ */
/* swept occupancy, Eq. (5)-(6), on the lattice rotated by R           */
/* ------------------------------------------------------------------ */

/*
 * S[(jz*N + jy)*N + jx] = 1 iff some pose i has the lattice point inside its
 * probe: with p = h j + o_s, x = R p (world), l = R_i^T (x - t_i),
 * inside <=> l0^2 + l1^2 <= r^2 and 0 <= l2 <= L.
 * o_s = h round(R^T c_s / h) - (N/2) h, c_s = mean tip position.
 * Every pose counts, whatever its contact label (Eq. (5) is a max over all i).
 */
ORC_API void orc_sweep_origin(const double *poses, int64_t P, const double *q, double h, int32_t N, double *o)
{
    double R[9];
    orc_quat_to_mat(q, R);
    double c[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < P; ++i) { c[0] += poses[7 * i + 4]; c[1] += poses[7 * i + 5]; c[2] += poses[7 * i + 6]; }
    for (int a = 0; a < 3; ++a) c[a] = c[a] / (double)P;
    for (int a = 0; a < 3; ++a) {
        double u = (R[0 * 3 + a] * c[0] + R[1 * 3 + a] * c[1]) + R[2 * 3 + a] * c[2];
        o[a] = lattice_origin(u, h, N);
    }
}

/*
 * Eq. (5)-(6) over the poses i with use[i] != 0 (all poses when use is NULL);
 * the lattice origin always follows the mean tip of ALL P poses, so the grids
 * of two pose subsets share one lattice (the label-aware score splits the
 * sweep by contact label this way).
 */
ORC_API void orc_sweep_grid_sel(const double *poses, int64_t P, const uint8_t *use, const double *q, double h,
                                int32_t N, double r, double L, double *origin, uint8_t *S)
{
    double R[9];
    orc_quat_to_mat(q, R);
    orc_sweep_origin(poses, P, q, h, N, origin);
    memset(S, 0, (size_t)N * N * N);
    double r2 = r * r;
    for (int64_t i = 0; i < P; ++i) {
        if (use && !use[i]) continue;
        double Ri[9];
        orc_quat_to_mat(poses + 7 * i, Ri);
        const double *t = poses + 7 * i + 4;
        /* conservative voxel box: the capsule around the probe axis segment */
        int64_t lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            double e0 = (R[0 * 3 + a] * t[0] + R[1 * 3 + a] * t[1]) + R[2 * 3 + a] * t[2];
            double ax = (R[0 * 3 + a] * Ri[2] + R[1 * 3 + a] * Ri[5]) + R[2 * 3 + a] * Ri[8];
            double e1 = e0 + L * ax;
            double a0 = (fmin(e0, e1) - r - origin[a]) / h, a1 = (fmax(e0, e1) + r - origin[a]) / h;
            lo[a] = (int64_t)floor(a0) - 2;
            hi[a] = (int64_t)ceil(a1) + 2;
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > N - 1) hi[a] = N - 1;
        }
        for (int64_t jz = lo[2]; jz <= hi[2]; ++jz)
            for (int64_t jy = lo[1]; jy <= hi[1]; ++jy)
                for (int64_t jx = lo[0]; jx <= hi[0]; ++jx) {
                    int64_t idx = (jz * N + jy) * N + jx;
                    if (S[idx]) continue;
                    double p[3] = {h * (double)jx + origin[0], h * (double)jy + origin[1], h * (double)jz + origin[2]};
                    double d[3];
                    for (int b = 0; b < 3; ++b)
                        d[b] = ((R[b * 3 + 0] * p[0] + R[b * 3 + 1] * p[1]) + R[b * 3 + 2] * p[2]) - t[b];
                    double l0 = (Ri[0] * d[0] + Ri[3] * d[1]) + Ri[6] * d[2];
                    double l1 = (Ri[1] * d[0] + Ri[4] * d[1]) + Ri[7] * d[2];
                    double l2 = (Ri[2] * d[0] + Ri[5] * d[1]) + Ri[8] * d[2];
                    if (l0 * l0 + l1 * l1 <= r2 && 0.0 <= l2 && l2 <= L) S[idx] = 1;
                }
    }
}

ORC_API void orc_sweep_grid(const double *poses, int64_t P, const double *q, double h, int32_t N,
                            double r, double L, double *origin, uint8_t *S)
{
    orc_sweep_grid_sel(poses, P, NULL, q, h, N, r, L, origin, S);
}

/*
 * Sec. IV-D, the paper's rotation mechanism: the object grid rotated by R and
 * resampled by trilinear interpolation onto a lattice of spacing h.
 *   o_R = h round(R c_o / h) - (N/2) h with c_o = o_o + (N/2) h, so the
 *         rotated lattice follows the rotated lattice centre (the rule of
 *         o_s,R with R in place of R^T);
 *   O_R[k] = O~(R^T (h k + o_R)), O~ the trilinear interpolant of O on its
 *         lattice (h k + o_o), zero at lattice points outside [0, N)^3.
 */
ORC_API void orc_rotate_object(const double *O, int32_t N, const double *o_o, const double *q, double h,
                               double *O_R, double *o_R)
{
    double R[9];
    orc_quat_to_mat(q, R);
    double c[3];
    for (int a = 0; a < 3; ++a) c[a] = o_o[a] + (double)(N / 2) * h;
    for (int a = 0; a < 3; ++a) {
        double u = (R[a * 3 + 0] * c[0] + R[a * 3 + 1] * c[1]) + R[a * 3 + 2] * c[2];
        o_R[a] = lattice_origin(u, h, N);
    }
    for (int64_t kz = 0; kz < N; ++kz)
        for (int64_t ky = 0; ky < N; ++ky)
            for (int64_t kx = 0; kx < N; ++kx) {
                double x[3] = {h * (double)kx + o_R[0], h * (double)ky + o_R[1], h * (double)kz + o_R[2]};
                double v[3];
                int64_t i0[3];
                double f[3];
                for (int a = 0; a < 3; ++a) {
                    double y = (R[0 * 3 + a] * x[0] + R[1 * 3 + a] * x[1]) + R[2 * 3 + a] * x[2];
                    v[a] = (y - o_o[a]) / h;
                    i0[a] = (int64_t)floor(v[a]);
                    f[a] = v[a] - (double)i0[a];
                }
                double acc = 0.0;
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) {
                            int64_t jx = i0[0] + dx, jy = i0[1] + dy, jz = i0[2] + dz;
                            if (jx < 0 || jy < 0 || jz < 0 || jx >= N || jy >= N || jz >= N) continue;
                            double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                            acc += w * O[(jz * N + jy) * N + jx];
                        }
                O_R[(kz * N + ky) * N + kx] = acc;
            }
}

/* ------------------------------------------------------------------ */
/* probe SDF (flat-ended cylinder) and Frank-Wolfe over a triangle      */
/* ------------------------------------------------------------------ */

/*
 * f_p of a flat-ended cylinder: radius r, tip face at z = 0, body z in [0, L].
 * dr = rho - r, dz = max(-z, z - L).  Inside (dr <= 0, dz <= 0): max(dr, dz);
 * outside: dr (side), dz (cap) or sqrt(dr^2 + dz^2) (rim).  g receives a
 * subgradient: the gradient of the active branch (the cap branch when
 * dr == dz inside), +x as the radial direction on the axis.
 */
ORC_API double orc_probe_sdf(const double *x, double r, double L, double *g)
{
    double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
    double ux = 1.0, uy = 0.0;
    if (rho > 0.0) { ux = x[0] / rho; uy = x[1] / rho; }
    double dr = rho - r;
    double zlo = -x[2], zhi = x[2] - L;
    double dz = zlo >= zhi ? zlo : zhi;
    double cz = zlo >= zhi ? -1.0 : 1.0;
    double f;
    if (dr <= 0.0 && dz <= 0.0) {
        if (dr > dz) { f = dr; if (g) { g[0] = ux; g[1] = uy; g[2] = 0.0; } }
        else { f = dz; if (g) { g[0] = 0.0; g[1] = 0.0; g[2] = cz; } }
    } else if (dr > 0.0 && dz > 0.0) {
        f = sqrt(dr * dr + dz * dz);
        if (g) { g[0] = dr * ux / f; g[1] = dr * uy / f; g[2] = dz * cz / f; }
    } else if (dr > 0.0) {
        f = dr;
        if (g) { g[0] = ux; g[1] = uy; g[2] = 0.0; }
    } else {
        f = dz;
        if (g) { g[0] = 0.0; g[1] = 0.0; g[2] = cz; }
    }
    return f;
}

/*
 * Contact normal n* of Eq. (23) at x: the unit SDF gradient, where f_p is
 * not differentiable (the medial surface dr == dz inside the cylinder, the
 * axis) the gradient of the branch orc_probe_sdf reports (the cap on ties,
 * +x as the radial direction on the axis).
 */
ORC_API void orc_probe_normal(const double *x, double r, double L, double *n)
{
    double g[3];
    orc_probe_sdf(x, r, L, g);
    double gn = sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);
    n[0] = g[0] / gn; n[1] = g[1] / gn; n[2] = g[2] / gn;
}

/* Distance (mm) from the medial surface within which a witness is treated
 * as lying on it: the Danskin rule below then picks the subgradient; off the
 * surface that rule returns the branch gradient itself for an optimal face
 * or edge witness, so the width only decides where the rule is evaluated. */
#define KINK_BAND 1e-3

static void comb(const double *v0, const double *v1, const double *v2, const double *lam, double *x)
{
    for (int a = 0; a < 3; ++a) x[a] = (lam[0] * v0[a] + lam[1] * v1[a]) + lam[2] * v2[a];
}

/*
 * The subgradient of f_p at the witness x that gives the derivative of
 * d = min over the triangle of f_p (Sec. V-B, Eq. (22)-(24)).  Where f_p is
 * differentiable it is the gradient.  On the medial surface inside the
 * probe (|dr - dz| <= KINK_BAND) the subdifferential is the segment between
 * the radial gradient a and the cap gradient b, and the minimum over the
 * triangle selects the element whose component along the face holding x
 * (the triangle's plane, or the edge when a barycentric weight is zero)
 * vanishes (the optimality condition of the convex minimum; the value then
 * moves with the pose as that subgradient says, by Danskin's theorem):
 * n = lam a + (1 - lam) b with lam minimising |P (lam a + (1 - lam) b)|,
 * P the projection onto the face.  A vertex of the triangle lies on the
 * medial surface only by coincidence (a set of poses of measure zero), so at
 * a vertex witness f_p is differentiable and n is the gradient of its active
 * branch (orc_probe_normal).  n is not normalised.
 */
static void witness_subgradient(const double *x, const double loc[3][3], const double *lam, double r, double L,
                                double *n)
{
    double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
    double dr = rho - r, zlo = -x[2], zhi = x[2] - L;
    double dz = zlo >= zhi ? zlo : zhi;
    int nz = 0, zi = -1;
    for (int k = 0; k < 3; ++k)
        if (lam[k] <= 1e-9) { ++nz; zi = k; }
    if (!(dr <= 0.0 && dz <= 0.0 && fabs(dr - dz) <= KINK_BAND && rho > 0.0) || nz >= 2) {
        orc_probe_normal(x, r, L, n);
        return;
    }
    double a[3] = {x[0] / rho, x[1] / rho, 0.0}, b[3] = {0.0, 0.0, zlo >= zhi ? -1.0 : 1.0};
    double Pa[3], Pb[3];
    if (nz == 0) {
        double e1[3], e2[3], nu[3];
        for (int i = 0; i < 3; ++i) { e1[i] = loc[1][i] - loc[0][i]; e2[i] = loc[2][i] - loc[0][i]; }
        nu[0] = e1[1] * e2[2] - e1[2] * e2[1];
        nu[1] = e1[2] * e2[0] - e1[0] * e2[2];
        nu[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double nn = (nu[0] * nu[0] + nu[1] * nu[1]) + nu[2] * nu[2];
        double an = ((a[0] * nu[0] + a[1] * nu[1]) + a[2] * nu[2]) / nn;
        double bn = ((b[0] * nu[0] + b[1] * nu[1]) + b[2] * nu[2]) / nn;
        for (int i = 0; i < 3; ++i) { Pa[i] = a[i] - an * nu[i]; Pb[i] = b[i] - bn * nu[i]; }
    } else {
        const double *p = loc[(zi + 1) % 3], *q = loc[(zi + 2) % 3];
        double e[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
        double ee = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2];
        double ae = ((a[0] * e[0] + a[1] * e[1]) + a[2] * e[2]) / ee;
        double be = ((b[0] * e[0] + b[1] * e[1]) + b[2] * e[2]) / ee;
        for (int i = 0; i < 3; ++i) { Pa[i] = ae * e[i]; Pb[i] = be * e[i]; }
    }
    double df[3] = {Pa[0] - Pb[0], Pa[1] - Pb[1], Pa[2] - Pb[2]};
    double dd = (df[0] * df[0] + df[1] * df[1]) + df[2] * df[2];
    double lm = 0.5;
    if (dd > 0.0) {
        lm = -((Pb[0] * df[0] + Pb[1] * df[1]) + Pb[2] * df[2]) / dd;
        if (lm < 0.0) lm = 0.0;
        if (lm > 1.0) lm = 1.0;
    }
    for (int i = 0; i < 3; ++i) n[i] = lm * a[i] + (1.0 - lm) * b[i];
}

/*
 * min over the triangle conv{v0,v1,v2} (probe-local coordinates) of f_p, the
 * per-triangle minimisation of Sec. V-B.  f_p is convex (the signed distance
 * of a convex body), so with x(u,v) = v0 + u (v1 - v0) + v (v2 - v0) the
 * partial minimum phi(u) = min_{0 <= v <= 1-u} f(x(u,v)) is convex too.  The
 * inner minimum is found by bisection on the sign of a subgradient along v
 * (any subgradient of f projects to a subgradient of the 1-D restriction);
 * the outer one by golden-section search on phi, which needs only values.
 * Both converge on the non-smooth medial surface inside the cylinder, where
 * Frank-Wolfe can stall.  `iters` steps per level (the outer level runs
 * iters + iters/2 golden steps, giving the same interval width).
 * lam_out receives the barycentric weights of the returned point.
 */
static double inner_min(const double *v0, const double *e1, const double *e2, double u, double r, double L,
                        int iters, double *v_out)
{
    double vmax = 1.0 - u;
    double x[3], g[3];
    for (int a = 0; a < 3; ++a) x[a] = v0[a] + u * e1[a];
    double f0 = orc_probe_sdf(x, r, L, g);
    if (vmax <= 0.0 || dot3(g, e2) >= 0.0) { *v_out = 0.0; return f0; }
    for (int a = 0; a < 3; ++a) x[a] = (v0[a] + u * e1[a]) + vmax * e2[a];
    double f1 = orc_probe_sdf(x, r, L, g);
    if (dot3(g, e2) <= 0.0) { *v_out = vmax; return f1; }
    double lo = 0.0, hi = vmax;
    for (int k = 0; k < iters; ++k) {
        double mid = 0.5 * (lo + hi);
        for (int a = 0; a < 3; ++a) x[a] = (v0[a] + u * e1[a]) + mid * e2[a];
        orc_probe_sdf(x, r, L, g);
        if (dot3(g, e2) < 0.0) lo = mid; else hi = mid;
    }
    double v = 0.5 * (lo + hi);
    for (int a = 0; a < 3; ++a) x[a] = (v0[a] + u * e1[a]) + v * e2[a];
    *v_out = v;
    return orc_probe_sdf(x, r, L, NULL);
}

ORC_API double orc_tri_min(const double *v0, const double *v1, const double *v2, double r, double L,
                           int iters, double *lam_out)
{
    double e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
    double e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
    const double ig = 0.6180339887498949;   /* 1 / golden ratio */
    double a = 0.0, b = 1.0, vc, vd;
    double c = b - ig * (b - a), d = a + ig * (b - a);
    double fc = inner_min(v0, e1, e2, c, r, L, iters, &vc);
    double fd = inner_min(v0, e1, e2, d, r, L, iters, &vd);
    int steps = iters + iters / 2;
    for (int k = 0; k < steps; ++k) {
        if (fc <= fd) {
            b = d; d = c; fd = fc; vd = vc;
            c = b - ig * (b - a);
            fc = inner_min(v0, e1, e2, c, r, L, iters, &vc);
        } else {
            a = c; c = d; fc = fd; vc = vd;
            d = a + ig * (b - a);
            fd = inner_min(v0, e1, e2, d, r, L, iters, &vd);
        }
    }
    double u = fc <= fd ? c : d, v = fc <= fd ? vc : vd, best = fc <= fd ? fc : fd;
    /* the golden interval never reaches its closed ends exactly */
    double vu0, vu1;
    double f0 = inner_min(v0, e1, e2, 0.0, r, L, iters, &vu0);
    double f1 = inner_min(v0, e1, e2, 1.0, r, L, iters, &vu1);
    if (f0 < best) { best = f0; u = 0.0; v = vu0; }
    if (f1 < best) { best = f1; u = 1.0; v = vu1; }
    if (lam_out) { lam_out[0] = (1.0 - u) - v; lam_out[1] = u; lam_out[2] = v; }
    return best;
}

/* ------------------------------------------------------------------ */
/* Lie-algebra pose update, Eq. (13)-(17)                               */
/* ------------------------------------------------------------------ */

/* a(th) = (1-cos th)/th^2, b(th) = (th - sin th)/th^3 and their derivatives
 * divided by th; series below 1e-4 as the paper prescribes for th -> 0. */
static void vcoef(double th, double *a, double *b, double *da_th, double *db_th)
{
    if (th < 1e-4) {
        double t2 = th * th;
        *a = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
        *b = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
        *da_th = -1.0 / 12.0 + t2 / 180.0;
        *db_th = -1.0 / 60.0 + t2 / 1260.0;
    } else {
        double s = sin(th), c = cos(th);
        *a = (1.0 - c) / (th * th);
        *b = (th - s) / (th * th * th);
        *da_th = (th * s - 2.0 * (1.0 - c)) / (th * th * th * th);
        *db_th = ((1.0 - c) * th - 3.0 * (th - s)) / (th * th * th * th * th);
    }
}

static void skew(const double *w, double *K)
{
    K[0] = 0.0;   K[1] = -w[2]; K[2] = w[1];
    K[3] = w[2];  K[4] = 0.0;   K[5] = -w[0];
    K[6] = -w[1]; K[7] = w[0];  K[8] = 0.0;
}

static void matmul3(const double *A, const double *B, double *C)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = (A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j]) + A[3 * i + 2] * B[6 + j];
}

/* exp(w^) by Rodrigues, V(w) = I + a w^ + b (w^)^2 (Eq. (14)-(15)). */
ORC_API void orc_so3_exp_V(const double *w, double *Rexp, double *V)
{
    double th = sqrt(dot3(w, w));
    double a, b, da, db;
    vcoef(th, &a, &b, &da, &db);
    double sA;   /* sin th / th */
    if (th < 1e-4) { double t2 = th * th; sA = 1.0 - t2 / 6.0 + t2 * t2 / 120.0; }
    else sA = sin(th) / th;
    double K[9], K2[9];
    skew(w, K);
    matmul3(K, K, K2);
    for (int i = 0; i < 9; ++i) {
        double I = (i % 4 == 0) ? 1.0 : 0.0;
        Rexp[i] = I + sA * K[i] + a * K2[i];
        V[i] = I + a * K[i] + b * K2[i];
    }
}

/* d(V(w) u)/dw (3x3, row = component of V u, column = component of w). */
static void dVu_dw(const double *w, const double *u, double *M)
{
    double th = sqrt(dot3(w, w));
    double a, b, da, db;
    vcoef(th, &a, &b, &da, &db);
    double wxu[3] = {w[1] * u[2] - w[2] * u[1], w[2] * u[0] - w[0] * u[2], w[0] * u[1] - w[1] * u[0]};
    double wd = dot3(w, u), ww = dot3(w, w);
    double wxwxu[3];
    for (int k = 0; k < 3; ++k) wxwxu[k] = w[k] * wd - u[k] * ww;
    double Ku[9];
    skew(u, Ku);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double I = (i == j) ? 1.0 : 0.0;
            /* d(a w x u)/dw = -a [u]x + (w x u) (da/dth / th) w^T */
            double t1 = -a * Ku[3 * i + j] + wxu[i] * da * w[j];
            /* d(b w x (w x u))/dw = b ((w.u) I + w u^T - 2 u w^T) + (w x (w x u)) (db/dth / th) w^T */
            double t2 = b * ((wd * I + w[i] * u[j]) - 2.0 * u[i] * w[j]) + wxwxu[i] * db * w[j];
            M[3 * i + j] = t1 + t2;
        }
}

/* T(xi): R = dR R0, p = p0 + V u + (I - dR) R0 a  (Eq. (16)-(17)). */
ORC_API void orc_pose_of_xi(const double *R0, const double *p0, const double *anchor, const double *xi,
                            double *R, double *p)
{
    double dR[9], V[9];
    orc_so3_exp_V(xi + 3, dR, V);
    matmul3(dR, R0, R);
    double Ra[3], dRRa[3], Vu[3];
    for (int i = 0; i < 3; ++i) Ra[i] = (R0[3 * i] * anchor[0] + R0[3 * i + 1] * anchor[1]) + R0[3 * i + 2] * anchor[2];
    for (int i = 0; i < 3; ++i) dRRa[i] = (dR[3 * i] * Ra[0] + dR[3 * i + 1] * Ra[1]) + dR[3 * i + 2] * Ra[2];
    for (int i = 0; i < 3; ++i) Vu[i] = (V[3 * i] * xi[0] + V[3 * i + 1] * xi[1]) + V[3 * i + 2] * xi[2];
    for (int i = 0; i < 3; ++i) p[i] = ((p0[i] + Vu[i]) + Ra[i]) - dRRa[i];
}

/* ------------------------------------------------------------------ */
/* proximity score, Eq. (18)                                           */
/* ------------------------------------------------------------------ */

typedef struct { double tau_out, tau_in, k, A, B, r; } score_t;

/* Eq. (18) with r = tau_in / tau_out and the C^1 coefficients
 * A = k/r^2 - 2/r^3, B = k/r - 3/r^2 (the printed ones are not C^1). */
static void score_init(score_t *S, double tau_out, double tau_in, double k)
{
    S->tau_out = tau_out; S->tau_in = tau_in; S->k = k;
    S->r = tau_in / tau_out;
    S->A = k / (S->r * S->r) - 2.0 / (S->r * S->r * S->r);
    S->B = k / S->r - 3.0 / (S->r * S->r);
}

/* s(d), ds/dd and d2s/dd2. */
ORC_API void orc_score(double d, double tau_out, double tau_in, double k, double *s, double *s1, double *s2)
{
    score_t S;
    score_init(&S, tau_out, tau_in, k);
    double t = d / S.tau_out, it = 1.0 / S.tau_out;
    if (t > 1.0) { *s = 0.0; *s1 = 0.0; *s2 = 0.0; }
    else if (t > 0.0) {
        double c = cos(0.5 * M_PI * t), sn = sin(0.5 * M_PI * t);
        *s = c * c;
        *s1 = -M_PI * c * sn * it;                          /* = -(pi/2) sin(pi t) / tau */
        *s2 = -0.5 * M_PI * M_PI * cos(M_PI * t) * it * it;
    } else if (t > -S.r) {
        *s = (S.A * t * t * t + S.B * t * t) + 1.0;
        *s1 = (3.0 * S.A * t * t + 2.0 * S.B * t) * it;
        *s2 = (6.0 * S.A * t + 2.0 * S.B) * it * it;
    } else {
        *s = S.k * (t + S.r);
        *s1 = S.k * it;
        *s2 = 0.0;
    }
}

/* ------------------------------------------------------------------ */
/* distance query, Eq. (21)-(23)                                       */
/* ------------------------------------------------------------------ */

typedef struct {
    double r, L;      /* probe */
    double eps;       /* pruning margin of Eq. (21) */
    int iters;        /* bisection steps per level of the triangle minimisation */
} query_t;

/* d* = min over triangles of min f_p; returns the triangle index (-1 when no
 * triangle passes the Eq. (21) circumsphere test), the witness in world
 * coordinates and the world-frame outward probe normal n* (Eq. (23)).
 * Object pose (R, p); probe pose (Ri, ti). */
static int64_t dist_query(const query_t *Q, const double *V, const int32_t *T, int64_t nt,
                          const double *R, const double *p, const double *Ri, const double *ti,
                          double *d_out, double *w_out, double *n_out)
{
    double best = INFINITY;
    int64_t bt = -1;
    double bx[3] = {0, 0, 0}, blam[3] = {0, 0, 0}, bloc[3][3];
    for (int64_t t = 0; t < nt; ++t) {
        double loc[3][3];
        for (int k = 0; k < 3; ++k) {
            const double *v = V + 3 * T[3 * t + k];
            double xw[3], dd[3];
            for (int i = 0; i < 3; ++i) xw[i] = ((R[3 * i] * v[0] + R[3 * i + 1] * v[1]) + R[3 * i + 2] * v[2]) + p[i];
            for (int i = 0; i < 3; ++i) dd[i] = xw[i] - ti[i];
            for (int i = 0; i < 3; ++i) loc[k][i] = (Ri[i] * dd[0] + Ri[3 + i] * dd[1]) + Ri[6 + i] * dd[2];
        }
        /* Eq. (21) for the triangle's circumsphere (centre = AABB centre,
         * radius = farthest vertex) */
        double c[3], rad = 0.0;
        for (int i = 0; i < 3; ++i) {
            double lo = fmin(loc[0][i], fmin(loc[1][i], loc[2][i])), hi = fmax(loc[0][i], fmax(loc[1][i], loc[2][i]));
            c[i] = 0.5 * (lo + hi);
        }
        for (int k = 0; k < 3; ++k) {
            double dx = loc[k][0] - c[0], dy = loc[k][1] - c[1], dz = loc[k][2] - c[2];
            double rr = sqrt((dx * dx + dy * dy) + dz * dz);
            if (rr > rad) rad = rr;
        }
        if (!(orc_probe_sdf(c, Q->r, Q->L, NULL) < rad + Q->eps)) continue;
        double lam[3];
        double dk = orc_tri_min(loc[0], loc[1], loc[2], Q->r, Q->L, Q->iters, lam);
        if (dk < best) {
            best = dk; bt = t;
            comb(loc[0], loc[1], loc[2], lam, bx);
            memcpy(blam, lam, sizeof(blam));
            memcpy(bloc, loc, sizeof(bloc));
        }
    }
    *d_out = best;
    if (bt >= 0) {
        double g[3];
        witness_subgradient(bx, (const double(*)[3])bloc, blam, Q->r, Q->L, g);
        for (int i = 0; i < 3; ++i) {
            n_out[i] = (Ri[3 * i] * g[0] + Ri[3 * i + 1] * g[1]) + Ri[3 * i + 2] * g[2];
            w_out[i] = ((Ri[3 * i] * bx[0] + Ri[3 * i + 1] * bx[1]) + Ri[3 * i + 2] * bx[2]) + ti[i];
        }
    }
    return bt;
}

/* Per-pose distance d_i for object pose (R, p).  Poses with no surviving
 * triangle get +inf. */
ORC_API void orc_distances(const double *V, int64_t nv, const int32_t *T, int64_t nt, const double *poses, int64_t P,
                           const double *R, const double *p, double r, double L, double eps, int iters,
                           double *d, double *w, double *n, int64_t *tri)
{
    (void)nv;
    query_t Q = {r, L, eps, iters};
    /* poses are independent: each writes only its own outputs */
#pragma omp parallel for schedule(dynamic, 2)
    for (int64_t i = 0; i < P; ++i) {
        double Ri[9];
        orc_quat_to_mat(poses + 7 * i, Ri);
        double ww[3] = {0, 0, 0}, nn[3] = {0, 0, 0};
        int64_t bt = dist_query(&Q, V, T, nt, R, p, Ri, poses + 7 * i + 4, d + i, ww, nn);
        if (w) for (int a = 0; a < 3; ++a) w[3 * i + a] = ww[a];
        if (n) for (int a = 0; a < 3; ++a) n[3 * i + a] = nn[a];
        if (tri) tri[i] = bt;
    }
}

/* ------------------------------------------------------------------ */
/* objective, gradient and Gauss-Newton matrix, Eq. (19), (24)-(28)     */
/* ------------------------------------------------------------------ */

typedef struct {
    double r, L;                  /* probe */
    double tau_out, tau_in, k;    /* Eq. (18) */
    double lambda;                /* Eq. (19) */
    double mu;                    /* Gauss-Newton damping */
    int iters;                    /* bisection steps of the triangle minimisation */
} refine_params_t;

/*
 * J(xi) = -sum_i s(d_i(xi)) + lambda |xi|^2, grad J (Eq. (28)) and
 * H = sum_i max(-s''(d_i), 0) g_i g_i^T + (2 lambda + mu) I, where
 * g_i = [V^T n_i ; V^T ((w_i - c) x n_i) + (d(V u)/dw)^T n_i] is the exact
 * derivative of d_i w.r.t. xi: Eq. (24)-(27) with the rotational term taken
 * through the left Jacobian V(w) of the increment (identical at xi = 0).
 * Poses with d_i >= tau_out contribute nothing (s = s' = s'' = 0).
 * Returns J; grad (6) and H (36, row-major) are filled when non-NULL.
 */
ORC_API double orc_objective(const double *V, int64_t nv, const int32_t *T, int64_t nt,
                             const double *poses, int64_t P, const double *R0, const double *p0,
                             const double *anchor, const double *xi, const double *prm,
                             double *grad, double *H, double *d_out)
{
    (void)nv;
    refine_params_t Pp = {prm[0], prm[1], prm[2], prm[3], prm[4], prm[5], prm[6], (int)prm[7]};
    double R[9], p[3], dR[9], Vm[9];
    orc_pose_of_xi(R0, p0, anchor, xi, R, p);
    orc_so3_exp_V(xi + 3, dR, Vm);
    double M[9];
    dVu_dw(xi + 3, xi, M);
    double Ra[3], Vu[3], c[3];
    for (int i = 0; i < 3; ++i) Ra[i] = (R0[3 * i] * anchor[0] + R0[3 * i + 1] * anchor[1]) + R0[3 * i + 2] * anchor[2];
    for (int i = 0; i < 3; ++i) Vu[i] = (Vm[3 * i] * xi[0] + Vm[3 * i + 1] * xi[1]) + Vm[3 * i + 2] * xi[2];
    for (int i = 0; i < 3; ++i) c[i] = (p0[i] + Vu[i]) + Ra[i];
    query_t Q = {Pp.r, Pp.L, Pp.tau_out, Pp.iters};
    double J = 0.0;
    double G[6] = {0, 0, 0, 0, 0, 0};
    double HH[36];
    memset(HH, 0, sizeof(HH));
    /* the per-pose queries are independent (computed in parallel); the sums
     * below run in pose order, so the result does not depend on the threads */
    double *qd = (double *)malloc(sizeof(double) * 7 * (size_t)(P > 0 ? P : 1));
    int64_t *qt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P > 0 ? P : 1));
    if (!qd || !qt) {
        free(qd);
        free(qt);
        return NAN;
    }
#pragma omp parallel for schedule(dynamic, 2)
    for (int64_t i = 0; i < P; ++i) {
        double Ri[9];
        orc_quat_to_mat(poses + 7 * i, Ri);
        qt[i] = dist_query(&Q, V, T, nt, R, p, Ri, poses + 7 * i + 4, qd + 7 * i, qd + 7 * i + 1, qd + 7 * i + 4);
    }
    for (int64_t i = 0; i < P; ++i) {
        const double d = qd[7 * i], *w = qd + 7 * i + 1, *n = qd + 7 * i + 4;
        const int64_t bt = qt[i];
        if (d_out) d_out[i] = d;
        if (bt < 0) continue;
        double s, s1, s2;
        orc_score(d, Pp.tau_out, Pp.tau_in, Pp.k, &s, &s1, &s2);
        J -= s;
        if (s1 == 0.0 && s2 == 0.0) continue;
        double g[6];
        for (int j = 0; j < 3; ++j) g[j] = (Vm[j] * n[0] + Vm[3 + j] * n[1]) + Vm[6 + j] * n[2];
        double wc[3] = {w[0] - c[0], w[1] - c[1], w[2] - c[2]};
        double tq[3] = {wc[1] * n[2] - wc[2] * n[1], wc[2] * n[0] - wc[0] * n[2], wc[0] * n[1] - wc[1] * n[0]};
        for (int j = 0; j < 3; ++j) {
            double a1 = (Vm[j] * tq[0] + Vm[3 + j] * tq[1]) + Vm[6 + j] * tq[2];
            double a2 = (M[j] * n[0] + M[3 + j] * n[1]) + M[6 + j] * n[2];
            g[3 + j] = a1 + a2;
        }
        for (int j = 0; j < 6; ++j) G[j] -= s1 * g[j];
        double wgt = -s2 > 0.0 ? -s2 : 0.0;
        if (wgt > 0.0)
            for (int a = 0; a < 6; ++a)
                for (int b = 0; b < 6; ++b) HH[6 * a + b] += wgt * g[a] * g[b];
    }
    free(qd);
    free(qt);
    double xx = 0.0;
    for (int j = 0; j < 6; ++j) xx += xi[j] * xi[j];
    J += Pp.lambda * xx;
    for (int j = 0; j < 6; ++j) G[j] += 2.0 * Pp.lambda * xi[j];
    for (int j = 0; j < 6; ++j) HH[7 * j] += 2.0 * Pp.lambda + Pp.mu;
    if (grad) memcpy(grad, G, sizeof(G));
    if (H) memcpy(H, HH, sizeof(HH));
    return J;
}

/* In-place Cholesky solve of the SPD 6x6 system H x = b. Returns -1 if H is
 * not positive definite. */
ORC_API int orc_chol6(const double *H, const double *b, double *x)
{
    double Lm[36];
    memset(Lm, 0, sizeof(Lm));
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = H[6 * i + j];
            for (int k = 0; k < j; ++k) s -= Lm[6 * i + k] * Lm[6 * j + k];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                Lm[6 * i + i] = sqrt(s);
            } else {
                Lm[6 * i + j] = s / Lm[6 * j + j];
            }
        }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= Lm[6 * i + k] * y[k];
        y[i] = s / Lm[6 * i + i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= Lm[6 * k + i] * x[k];
        x[i] = s / Lm[6 * i + i];
    }
    return 0;
}

/*
 * Fixed-iteration projected Gauss-Newton on Eq. (20) from xi = 0 (Sec. V-C
 * starts L-BFGS-B at xi_0 = 0 under the same box; the solver itself is the
 * normal-equation step): delta = -H^{-1} grad J, uniformly scaled so that
 * |delta_u|_inf <= step_t and |delta_w|_inf <= step_r, then xi is clipped to
 * |u|_inf <= b_t, |w|_inf <= b_r.  The trust-region radii shrink by `decay`
 * after every iteration, so the last steps are small whatever the local
 * conditioning (there is no accept/reject branch: an FP32 and an FP64 run
 * take the same control path).  Writes xi (6) and returns the final J.
 * prm: r, L, tau_out, tau_in, k, lambda, mu, bisection steps, (unused),
 *      (unused), iters, step_t, step_r, b_t, b_r, decay.
 */
ORC_API double orc_refine(const double *V, int64_t nv, const int32_t *T, int64_t nt, const double *poses, int64_t P,
                          const double *R0, const double *p0, const double *anchor, const double *prm, double *xi,
                          double *J_hist)
{
    int iters = (int)prm[10];
    double step_t = prm[11], step_r = prm[12], bt = prm[13], br = prm[14], decay = prm[15];
    for (int j = 0; j < 6; ++j) xi[j] = 0.0;
    for (int it = 0; it < iters; ++it) {
        double G[6], H[36], dlt[6], nb[6];
        double J = orc_objective(V, nv, T, nt, poses, P, R0, p0, anchor, xi, prm, G, H, NULL);
        if (J_hist) J_hist[it] = J;
        for (int j = 0; j < 6; ++j) nb[j] = -G[j];
        if (orc_chol6(H, nb, dlt) != 0) break;
        double mt = 0.0, mr = 0.0;
        for (int j = 0; j < 3; ++j) { mt = fmax(mt, fabs(dlt[j])); mr = fmax(mr, fabs(dlt[3 + j])); }
        double sc = 1.0;
        if (mt > step_t) sc = fmin(sc, step_t / mt);
        if (mr > step_r) sc = fmin(sc, step_r / mr);
        step_t *= decay;
        step_r *= decay;
        for (int j = 0; j < 6; ++j) {
            double v = xi[j] + sc * dlt[j];
            double b = j < 3 ? bt : br;
            if (v > b) v = b;
            if (v < -b) v = -b;
            xi[j] = v;
        }
    }
    return orc_objective(V, nv, T, nt, poses, P, R0, p0, anchor, xi, prm, NULL, NULL, NULL);
}
