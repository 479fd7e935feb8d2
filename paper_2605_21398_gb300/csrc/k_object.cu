// Object grid (Sec. IV-A.1, Eq. (1)-(4)) and its canvas spectrum (Eq. (9)).
//
// This translation unit is compiled with -fmad=false: every FP64 expression
// is rounded exactly as written, so the signed distance, its sign and the band
// value O are the same numbers a plain FP64 evaluation of the definition gives.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dock_internal.h"

namespace dock {

// Squared distance from p to triangle (a, b, c): closest point by the Voronoi
// regions of the triangle (three vertices, three edges, interior).
__device__ double tri_dist2(const double *p, const double *a, const double *b, const double *c)
{
    double e0[3], e1[3], w[3];
    for (int i = 0; i < 3; ++i) { e0[i] = b[i] - a[i]; e1[i] = c[i] - a[i]; w[i] = p[i] - a[i]; }
    double s1 = (e0[0] * w[0] + e0[1] * w[1]) + e0[2] * w[2];
    double s2 = (e1[0] * w[0] + e1[1] * w[1]) + e1[2] * w[2];
    double q[3];
    if (s1 <= 0.0 && s2 <= 0.0) {                      // vertex a
        q[0] = a[0]; q[1] = a[1]; q[2] = a[2];
    } else {
        double wb[3] = {p[0] - b[0], p[1] - b[1], p[2] - b[2]};
        double s3 = (e0[0] * wb[0] + e0[1] * wb[1]) + e0[2] * wb[2];
        double s4 = (e1[0] * wb[0] + e1[1] * wb[1]) + e1[2] * wb[2];
        double vc = s1 * s4 - s3 * s2;
        if (s3 >= 0.0 && s4 <= s3) {                   // vertex b
            q[0] = b[0]; q[1] = b[1]; q[2] = b[2];
        } else if (vc <= 0.0 && s1 >= 0.0 && s3 <= 0.0) {   // edge ab
            double t = s1 / (s1 - s3);
            for (int i = 0; i < 3; ++i) q[i] = a[i] + t * e0[i];
        } else {
            double wc[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
            double s5 = (e0[0] * wc[0] + e0[1] * wc[1]) + e0[2] * wc[2];
            double s6 = (e1[0] * wc[0] + e1[1] * wc[1]) + e1[2] * wc[2];
            double vb = s5 * s2 - s1 * s6;
            double va = s3 * s6 - s5 * s4;
            if (s6 >= 0.0 && s5 <= s6) {               // vertex c
                q[0] = c[0]; q[1] = c[1]; q[2] = c[2];
            } else if (vb <= 0.0 && s2 >= 0.0 && s6 <= 0.0) {   // edge ac
                double t = s2 / (s2 - s6);
                for (int i = 0; i < 3; ++i) q[i] = a[i] + t * e1[i];
            } else if (va <= 0.0 && (s4 - s3) >= 0.0 && (s5 - s6) >= 0.0) {   // edge bc
                double t = (s4 - s3) / ((s4 - s3) + (s5 - s6));
                for (int i = 0; i < 3; ++i) q[i] = b[i] + t * (c[i] - b[i]);
            } else {                                   // interior
                double inv = 1.0 / ((va + vb) + vc);
                double v = vb * inv, u = vc * inv;
                for (int i = 0; i < 3; ++i) q[i] = (a[i] + e0[i] * v) + e1[i] * u;
            }
        }
    }
    double dx = p[0] - q[0], dy = p[1] - q[1], dz = p[2] - q[2];
    return (dx * dx + dy * dy) + dz * dz;
}

// 2-D edge function of (a -> b) at (py, pz) with the point perturbed to
// (py + eps, pz + eps^2) (simulation of simplicity): never zero for a
// non-degenerate edge, so a row through a shared edge or vertex is counted
// by exactly one triangle.
__device__ int edge_side(double ay, double az, double by, double bz, double py, double pz, double *e)
{
    double v = (by - ay) * (pz - az) - (bz - az) * (py - ay);
    *e = v;
    if (v > 0.0) return 1;
    if (v < 0.0) return -1;
    if (bz != az) return bz > az ? -1 : 1;
    if (by != ay) return by > ay ? 1 : -1;
    return 0;
}

// One block per lattice row (ky, kz); thread kx.  The row's crossings with
// the mesh along +x decide the sign (odd count beyond x = inside).
__global__ void k_object_grid(const double *V, const int32_t *T, const uint8_t *touch, ObjBins bins, int N, double h,
                              double o0, double o1, double o2, double tau_out, double tau_in, double deep, float *O,
                              float *f_out, int *err)
{
    __shared__ double xs[1024];
    __shared__ int nx;
    const int ky = blockIdx.x % N, kz = blockIdx.x / N;
    const double py = h * (double)ky + o1;
    const double pz = h * (double)kz + o2;
    if (threadIdx.x == 0) nx = 0;
    __syncthreads();
    {
        int cy = (int)floor((py - o1) / bins.cs), cz = (int)floor((pz - o2) / bins.cs);
        if (cy >= 0 && cy < bins.d2[0] && cz >= 0 && cz < bins.d2[1]) {
            int cell = cz * bins.d2[0] + cy;
            for (int k = bins.cell2_start[cell] + threadIdx.x; k < bins.cell2_start[cell + 1]; k += blockDim.x) {
                int t = bins.cell2_items[k];
                const double *v0 = V + 3 * T[3 * t], *v1 = V + 3 * T[3 * t + 1], *v2 = V + 3 * T[3 * t + 2];
                double e0, e1, e2;
                int s0 = edge_side(v1[1], v1[2], v2[1], v2[2], py, pz, &e0);
                int s1 = edge_side(v2[1], v2[2], v0[1], v0[2], py, pz, &e1);
                int s2 = edge_side(v0[1], v0[2], v1[1], v1[2], py, pz, &e2);
                if (s0 == 0 || s0 != s1 || s1 != s2) continue;
                double den = (e0 + e1) + e2;
                if (den == 0.0) continue;
                double x = ((e0 * v0[0] + e1 * v1[0]) + e2 * v2[0]) / den;
                int slot = atomicAdd(&nx, 1);
                if (slot < 1024) xs[slot] = x;
                else atomicExch(err, DOCK_E_OVERFLOW);
            }
        }
    }
    __syncthreads();
    const int n_cross = min(nx, 1024);
    const double cut = tau_out > tau_in ? tau_out : tau_in;
    const double cut2 = cut * cut;
    for (int kx = threadIdx.x; kx < N; kx += blockDim.x) {
        double p[3] = {h * (double)kx + o0, py, pz};
        int par = 0;
        for (int c = 0; c < n_cross; ++c) par ^= (xs[c] > p[0]) ? 1 : 0;
        int cx = (int)floor((p[0] - o0) / bins.cs);
        int cyy = (int)floor((p[1] - o1) / bins.cs);
        int czz = (int)floor((p[2] - o2) / bins.cs);
        double best = INFINITY, bestt = INFINITY;
        if (cx >= 0 && cx < bins.d3[0] && cyy >= 0 && cyy < bins.d3[1] && czz >= 0 && czz < bins.d3[2]) {
            int cell = (czz * bins.d3[1] + cyy) * bins.d3[0] + cx;
            for (int k = bins.cell3_start[cell]; k < bins.cell3_start[cell + 1]; ++k) {
                int t = bins.cell3_items[k];
                double d2 = tri_dist2(p, V + 3 * T[3 * t], V + 3 * T[3 * t + 1], V + 3 * T[3 * t + 2]);
                if (d2 < best) best = d2;
                if ((touch == nullptr || touch[t]) && d2 < bestt) bestt = d2;
            }
        }
        double D = best < cut2 ? sqrt(best) : INFINITY;
        double Dt = bestt < cut2 ? sqrt(bestt) : INFINITY;
        double f = par ? -D : D;
        double Ot;
        if (0.0 <= f && f < tau_out) Ot = 1.0 - f / tau_out;          // Eq. (1), first branch
        else if (-tau_in < f && f < 0.0) Ot = 1.0 + f / tau_in;      // shallow penetration
        else if (f <= -tau_in) Ot = deep;                            // deep penetration
        else Ot = 0.0;
        double Om = 1.0 - Dt / tau_out;                              // Eq. (2)
        if (!(Om > 0.0)) Om = 0.0;
        double val = Ot < Om ? Ot : Om;                              // Eq. (3)
        size_t idx = ((size_t)kz * N + ky) * N + kx;
        O[idx] = (float)val;
        if (f_out) f_out[idx] = (float)f;
    }
}

cudaError_t launch_object_grid(const double *V, const int32_t *T, const uint8_t *touch, const ObjBins &bins, int N,
                               double h, const double *o, double tau_out, double tau_in, double deep, float *O,
                               float *f_out, int *err, cudaStream_t st)
{
    k_object_grid<<<N * N, 128, 0, st>>>(V, T, touch, bins, N, h, o[0], o[1], o[2], tau_out, tau_in, deep, O, f_out,
                                         err);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// conj(F(O)) / M^3 on the zero-padded M^3 canvas, FP64 direct DFT per axis
// (O occupies the corner [0, N)^3), stored as FP32 in the z-pass tile order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cmuld(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// A[z][y][kx] = sum_x O[z][y][x] w^(kx x), kx in [0, H]  (min(O, 0) when pen)
__global__ void k_spec_x(const float *O, int N, int M, const double2 *tw, double2 *A, bool pen)
{
    const int H = M / 2;
    const int row = blockIdx.x;   // z * N + y
    const float *o = O + (size_t)row * N;
    for (int kx = threadIdx.x; kx <= H; kx += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int x = 0; x < N; ++x) {
            double v = (double)o[x];
            if (pen) v = fmin(v, 0.0);
            if (v != 0.0) {
                double2 w = tw[(kx * x) % M];
                acc.x += v * w.x;
                acc.y += v * w.y;
            }
        }
        A[(size_t)row * (H + 1) + kx] = acc;
    }
}

// B[z][ky][kx] = sum_y A[z][y][kx] w^(ky y)
__global__ void k_spec_y(const double2 *A, int N, int M, const double2 *tw, double2 *Bo)
{
    const int H = M / 2;
    const int z = blockIdx.y, ky = blockIdx.x;
    for (int kx = threadIdx.x; kx <= H; kx += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int y = 0; y < N; ++y) {
            double2 a = A[((size_t)z * N + y) * (H + 1) + kx];
            double2 r = cmuld(a, tw[(ky * y) % M]);
            acc.x += r.x;
            acc.y += r.y;
        }
        Bo[((size_t)z * M + ky) * (H + 1) + kx] = acc;
    }
}

// spec tile: conj(sum_z B[z][ky][kx] w^(kz z)) / M^3 at f = ky P + kx (no conj when !cj)
__global__ void k_spec_z(const double2 *Bi, int N, int M, int P, const double2 *tw, float2 *spec, bool cj)
{
    const int H = M / 2;
    const int ky = blockIdx.y, kz = blockIdx.x;
    const double sc = 1.0 / ((double)M * (double)M * (double)M);
    for (int kx = threadIdx.x; kx < P; kx += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        if (kx <= H) {
            for (int z = 0; z < N; ++z) {
                double2 r = cmuld(Bi[((size_t)z * M + ky) * (H + 1) + kx], tw[(kz * z) % M]);
                acc.x += r.x;
                acc.y += r.y;
            }
        }
        size_t f = (size_t)ky * P + kx;
        size_t chunk = f / 32, lane = f % 32;
        spec[(chunk * M + kz) * 32 + lane] = make_float2((float)(acc.x * sc), (float)((cj ? -acc.y : acc.y) * sc));
    }
}

cudaError_t launch_spectrum(const float *O, int N, int M, int P, double2 *work1, double2 *work2, const double2 *twd,
                            float2 *spec, cudaStream_t st, bool pen, bool conj)
{
    k_spec_x<<<N * N, 160, 0, st>>>(O, N, M, twd, work1, pen);
    k_spec_y<<<dim3(M, N), 160, 0, st>>>(work1, N, M, twd, work2);
    k_spec_z<<<dim3(M, M), 160, 0, st>>>(work2, N, M, P, twd, spec, conj);
    return cudaGetLastError();
}

}  // namespace dock
