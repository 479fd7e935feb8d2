// Docking search kernels (Sec. IV): rotated swept-volume voxeliser fused with
// the forward 2-D FFT of each lattice slab, the z-pass with the conjugate
// object-spectrum multiply, and the inverse plane pass with the C2R along x
// and the per-rotation argmax.  Correlation per Eq. (7), computed as
// C = F^-1(conj(F(O)) . F(S)) (Eq. (9) with the conjugate on the object, the
// reading that agrees with Eq. (7)-(8)).
//
// Data layout (complex64, kx fastest):
//   Y[b][z < N][ky < M][kx < P]   forward x,y transform of slab z of S_b
//   Z[b][z < M][ky < M][kx < P]   after forward z, multiply, inverse z
//   spec[chunk][kz < M][32]       conj(F(O)) / M^3, f = ky P + kx in chunks of 32
// P = M/2 + 2 (16-byte aligned rows); entries kx in (M/2, P) are zero.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dock_internal.h"
#include "fft.cuh"
#include "peak_key.cuh"

namespace cg = cooperative_groups;

namespace dock {

// ---------------------------------------------------------------------------
// exact FP64 helpers (no contraction: every product and sum rounded as written)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }

// asynchronous 8-byte global -> shared copies (completion: cp_async_wait_all)
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
// wait until at most n (0..3) of this thread's committed groups are pending
__device__ __forceinline__ void cp_async_wait_pending(int n)
{
    switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    }
}

__device__ void quat_to_mat_exact(const double *q, double *R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = ds(1.0, dm(2.0, da(dm(y, y), dm(z, z))));
    R[1] = dm(2.0, ds(dm(x, y), dm(w, z)));
    R[2] = dm(2.0, da(dm(x, z), dm(w, y)));
    R[3] = dm(2.0, da(dm(x, y), dm(w, z)));
    R[4] = ds(1.0, dm(2.0, da(dm(x, x), dm(z, z))));
    R[5] = dm(2.0, ds(dm(y, z), dm(w, x)));
    R[6] = dm(2.0, ds(dm(x, z), dm(w, y)));
    R[7] = dm(2.0, da(dm(y, z), dm(w, x)));
    R[8] = ds(1.0, dm(2.0, da(dm(x, x), dm(y, y))));
}

// R = R(q), o = h round(R^T c_s / h) - (N/2) h   (Sec. IV-A: lattice origin).
// With o_o (the object rotated, Sec. IV-D): c = o_o + (N/2) h,
// o = o_R = h round(R c / h) - (N/2) h and ub = (R^T o_R - o_o) / h.
__global__ void k_rot_setup(const double *quats, int n, int rot0, int req, const double *c_s, double h, int N,
                            RotRec *out, const double *o_o)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    RotRec rr;
    double q[4] = {quats[4 * i], quats[4 * i + 1], quats[4 * i + 2], quats[4 * i + 3]};
    quat_to_mat_exact(q, rr.R);
    const double half = dm((double)(N / 2), h);
    if (o_o) {
        double c[3];
        for (int a = 0; a < 3; ++a) c[a] = da(o_o[a], half);
        for (int a = 0; a < 3; ++a) {
            double u = da(da(dm(rr.R[a * 3 + 0], c[0]), dm(rr.R[a * 3 + 1], c[1])), dm(rr.R[a * 3 + 2], c[2]));
            rr.o[a] = ds(dm(h, round(__ddiv_rn(u, h))), half);
        }
        for (int a = 0; a < 3; ++a) {
            double y = da(da(dm(rr.R[0 * 3 + a], rr.o[0]), dm(rr.R[1 * 3 + a], rr.o[1])), dm(rr.R[2 * 3 + a], rr.o[2]));
            rr.ub[a] = (float)__ddiv_rn(ds(y, o_o[a]), h);
        }
    } else {
        double c0 = c_s[0], c1 = c_s[1], c2 = c_s[2];
        for (int a = 0; a < 3; ++a) {
            double u = da(da(dm(rr.R[0 * 3 + a], c0), dm(rr.R[1 * 3 + a], c1)), dm(rr.R[2 * 3 + a], c2));
            rr.o[a] = ds(dm(h, round(__ddiv_rn(u, h))), half);
            rr.ub[a] = 0.f;
        }
    }
    for (int k = 0; k < 9; ++k) rr.Rf[k] = (float)rr.R[k];
    for (int a = 0; a < 3; ++a) rr.of[a] = (float)rr.o[a];
    rr.rot = rot0 + i;
    rr.req = req;
    out[i] = rr;
}

cudaError_t launch_rot_setup(const double *quats, int n, int rot0, int req, const double *c_s, double h, int N,
                             RotRec *out, cudaStream_t st, const double *o_o)
{
    if (n <= 0) return cudaSuccess;
    k_rot_setup<<<(n + 127) / 128, 128, 0, st>>>(quats, n, rot0, req, c_s, h, N, out, o_o);
    return cudaGetLastError();
}

// Corner cells of the object grid for trilinear interpolation: cell
// (cx, cy, cz), c in [-1, N) per axis, holds O at (cx, cy), (cx+1, cy),
// (cx, cy+1), (cx+1, cy+1) of plane cz (zero off the lattice), stored at
// ((cz+1) (N+1) + cy+1) (N+1) + cx+1.  An interpolation then reads two
// 16-byte cells (planes cz and cz+1) instead of eight scattered floats.
__global__ void k_corner_cells(const float *__restrict__ O, int N, float4 *cells)
{
    const int N1 = N + 1;
    const size_t n = (size_t)N1 * N1 * N1;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int cx = (int)(i % N1) - 1, cy = (int)((i / N1) % N1) - 1, cz = (int)(i / ((size_t)N1 * N1)) - 1;
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = cx + (k & 1), y = cy + (k >> 1);
            const bool in = (unsigned)x < (unsigned)N && (unsigned)y < (unsigned)N && (unsigned)cz < (unsigned)N;
            v[k] = in ? O[((size_t)cz * N + y) * N + x] : 0.f;
        }
        cells[i] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

cudaError_t launch_corner_cells(const float *O, int N, float4 *cells, cudaStream_t st)
{
    k_corner_cells<<<152 * 4, 256, 0, st>>>(O, N, cells);
    return cudaGetLastError();
}

// Trilinear interpolant of the N^3 grid O (as corner cells) at continuous
// index (ux, uy, uz); lattice points outside [0, N)^3 count as zero (Sec.
// IV-D resampling).  Interpolates along x, then y, then z.
__device__ __forceinline__ float trilerp(const float4 *__restrict__ cells, int N, float ux, float uy, float uz)
{
    const float fx = floorf(ux), fy = floorf(uy), fz = floorf(uz);
    const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    if (ix < -1 || iy < -1 || iz < -1 || ix >= N || iy >= N || iz >= N) return 0.f;
    const float ax = ux - fx, ay = uy - fy, az = uz - fz;
    const int N1 = N + 1;
    const size_t c = ((size_t)(iz + 1) * N1 + (iy + 1)) * N1 + (ix + 1);
    const float4 p = __ldg(&cells[c]);
    const float4 q = iz + 1 < N ? __ldg(&cells[c + (size_t)N1 * N1]) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float e00 = fmaf(ax, p.y - p.x, p.x), e01 = fmaf(ax, p.w - p.z, p.z);
    const float e10 = fmaf(ax, q.y - q.x, q.x), e11 = fmaf(ax, q.w - q.z, q.z);
    const float f0 = fmaf(ay, e01 - e00, e00);
    const float f1 = fmaf(ay, e11 - e10, e10);
    return fmaf(az, f1 - f0, f0);
}

// Voxel (x, y, z) of the rotated object grid of rotation rr.
__device__ __forceinline__ float rotated_object_voxel(const RotRec &rr, const float4 *cells, int N, int x, int y, int z)
{
    const float fx = (float)x, fy = (float)y, fz = (float)z;
    const float ux = fmaf(rr.Rf[0], fx, fmaf(rr.Rf[3], fy, fmaf(rr.Rf[6], fz, rr.ub[0])));
    const float uy = fmaf(rr.Rf[1], fx, fmaf(rr.Rf[4], fy, fmaf(rr.Rf[7], fz, rr.ub[1])));
    const float uz = fmaf(rr.Rf[2], fx, fmaf(rr.Rf[5], fy, fmaf(rr.Rf[8], fz, rr.ub[2])));
    return trilerp(cells, N, ux, uy, uz);
}

// ---------------------------------------------------------------------------
// swept-volume voxeliser (Eq. (5)-(6)) for one slab z of the rotated lattice
// ---------------------------------------------------------------------------

// Exact inside test of Eq. (5) at lattice voxel (jx, jy, jz): the same FP64
// expression, in the same order, as the definition:
//   p = h j + o ; x = R p ; d = x - t_i ; l = R_i^T d ;
//   l0^2 + l1^2 <= r^2  and  0 <= l2 <= L.
__device__ __noinline__ bool inside_exact(const RotRec &rr, const PoseRec &pr, double h, double r2, double L, int jx,
                                          int jy, int jz)
{
    double p0 = da(dm(h, (double)jx), rr.o[0]);
    double p1 = da(dm(h, (double)jy), rr.o[1]);
    double p2 = da(dm(h, (double)jz), rr.o[2]);
    double d[3];
    for (int b = 0; b < 3; ++b)
        d[b] = ds(da(da(dm(rr.R[b * 3 + 0], p0), dm(rr.R[b * 3 + 1], p1)), dm(rr.R[b * 3 + 2], p2)), pr.t[b]);
    const double *Ri = pr.R;
    double l0 = da(da(dm(Ri[0], d[0]), dm(Ri[3], d[1])), dm(Ri[6], d[2]));
    double l1 = da(da(dm(Ri[1], d[0]), dm(Ri[4], d[1])), dm(Ri[7], d[2]));
    double l2 = da(da(dm(Ri[2], d[0]), dm(Ri[5], d[1])), dm(Ri[8], d[2]));
    return da(dm(l0, l0), dm(l1, l1)) <= r2 && 0.0 <= l2 && l2 <= L;
}

struct VoxCtx {
    // FP32 pose frame in lattice voxel units: l(j) = B^T (j - c)
    float B[9];   // B[a*3+k] = (R^T R_i)[a][k]
    float c[3];
};

// Classify voxel jx on the row whose FP32 local coordinates at jx = 0 are l0
// (step bx per voxel).  Margins cover the FP32 error of l (bounded well below
// 2e-4 voxels for lattices of <= 256 voxels); inside the margin band the exact
// FP64 predicate decides.
__device__ __forceinline__ int classify(const float *l0, const float *bx, int jx, float rv2, float lv, float mr,
                                        float mz, const RotRec &rr, const PoseRec &pr, double h, double r2d,
                                        double Ld, int jy, int jz)
{
    float fx = (float)jx;
    float a = fmaf(fx, bx[0], l0[0]);
    float b = fmaf(fx, bx[1], l0[1]);
    float z = fmaf(fx, bx[2], l0[2]);
    float rad2 = fmaf(a, a, b * b);
    if (rad2 <= rv2 - mr && z >= mz && z <= lv - mz) return 1;
    if (rad2 > rv2 + mr || z < -mz || z > lv + mz) return 0;
    return inside_exact(rr, pr, h, r2d, Ld, jx, jy, jz) ? 1 : 0;
}

__device__ __forceinline__ void set_bits(uint32_t *row, int lo, int hi)
{
    int w0 = lo >> 5, w1 = hi >> 5;
    for (int w = w0; w <= w1; ++w) {
        int a = (w == w0) ? (lo & 31) : 0;
        int b = (w == w1) ? (hi & 31) : 31;
        uint32_t m = (b == 31 ? 0xFFFFFFFFu : ((1u << (b + 1)) - 1u)) & ~((1u << a) - 1u);
        atomicOr(&row[w], m);
    }
}

// Pose frame of pose i in lattice voxel units for rotation rr (FP32):
// l(j) = B^T (j - c), B = R^T R_i, c = (R^T t_i - o) / h.
__device__ __forceinline__ void pose_frame(const RotRec &rr, const PoseRec &pr, float ih, float *B, float *c)
{
    const float *Rf = rr.Rf;
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a)
            B[a * 3 + k] = fmaf(Rf[0 * 3 + a], pr.Rf[0 * 3 + k], fmaf(Rf[1 * 3 + a], pr.Rf[1 * 3 + k], Rf[2 * 3 + a] * pr.Rf[2 * 3 + k]));
    for (int a = 0; a < 3; ++a)
        c[a] = (fmaf(Rf[0 * 3 + a], pr.tf[0], fmaf(Rf[1 * 3 + a], pr.tf[1], Rf[2 * 3 + a] * pr.tf[2])) - rr.of[a]) * ih;
}

// One lattice row (jy, jz) of one pose: set the bits of the voxels inside the
// probe.  The FP32 interval from the radial quadratic and the axial slab is
// only a starting point: the exact end voxels are found by classifying
// neighbours (an interval, since the cylinder is convex), with the exact
// FP64 predicate deciding inside the FP32 error band.
template <int N>
__device__ __forceinline__ void vox_row(const float *B, const float *c, int jy, int jz, float rv2, float lv, float mr,
                                        float mz, const RotRec &rr, const PoseRec &pr, double h, double r2d, double Ld,
                                        uint32_t *row)
{
    const float bx[3] = {B[0], B[1], B[2]};   // B^T e_x
    const float Aq = fmaf(bx[0], bx[0], bx[1] * bx[1]);
    float dyv = (float)jy - c[1], dzv = (float)jz - c[2], dxv = -c[0];
    float l0[3];
    for (int k = 0; k < 3; ++k) l0[k] = fmaf(B[0 * 3 + k], dxv, fmaf(B[1 * 3 + k], dyv, B[2 * 3 + k] * dzv));
    float lo = -1e30f, hi = 1e30f;
    int wide = 2;
    if (Aq > 1e-6f) {
        float Bq = fmaf(l0[0], bx[0], l0[1] * bx[1]);
        float Cq = fmaf(l0[0], l0[0], l0[1] * l0[1]) - rv2;
        float disc = fmaf(Bq, Bq, -Aq * Cq);
        if (disc < -1e-3f * (Bq * Bq + fabsf(Aq * Cq)) - 1e-2f) return;
        float sq = sqrtf(fmaxf(disc, 0.f));
        lo = (-Bq - sq) / Aq;
        hi = (-Bq + sq) / Aq;
        if (Aq < 0.05f) wide = N;
    } else {
        float Cq = fmaf(l0[0], l0[0], l0[1] * l0[1]) - rv2;
        if (Cq > mr + 1e-2f) return;
        wide = N;
    }
    if (fabsf(bx[2]) >= 1e-3f) {
        float za = -l0[2] / bx[2], zb = (lv - l0[2]) / bx[2];
        lo = fmaxf(lo, fminf(za, zb));
        hi = fminf(hi, fmaxf(za, zb));
    } else {
        // row nearly parallel to the cap planes: only a row clearly outside them
        // is dropped; otherwise the walk below finds the ends exactly
        const float zA = l0[2], zB = fmaf((float)(N - 1), bx[2], l0[2]);
        if (fmaxf(zA, zB) < -0.3f || fminf(zA, zB) > lv + 0.3f) return;
    }
    if (lo > hi + 2.f) return;
    lo = fmaxf(lo, -4.f);
    hi = fminf(hi, (float)N + 4.f);
    const int jmax = min(N - 1, (int)ceilf(hi) + wide);
    int jl = min(N - 1, max(0, (int)ceilf(lo)));
    if (wide > 2) jl = max(0, (int)floorf(lo) - wide);
    if (jl > jmax) return;
    if (classify(l0, bx, jl, rv2, lv, mr, mz, rr, pr, h, r2d, Ld, jy, jz)) {
        while (jl > 0 && classify(l0, bx, jl - 1, rv2, lv, mr, mz, rr, pr, h, r2d, Ld, jy, jz)) --jl;
    } else {
        do { ++jl; } while (jl <= jmax && !classify(l0, bx, jl, rv2, lv, mr, mz, rr, pr, h, r2d, Ld, jy, jz));
        if (jl > jmax) return;
    }
    int jr = max(jl, min(N - 1, (int)floorf(hi)));
    if (classify(l0, bx, jr, rv2, lv, mr, mz, rr, pr, h, r2d, Ld, jy, jz)) {
        while (jr < N - 1 && classify(l0, bx, jr + 1, rv2, lv, mr, mz, rr, pr, h, r2d, Ld, jy, jz)) ++jr;
    } else {
        do { --jr; } while (jr > jl && !classify(l0, bx, jr, rv2, lv, mr, mz, rr, pr, h, r2d, Ld, jy, jz));
    }
    set_bits(row, jl, jr);
}

// Fill bits[jy * NW + w] for slab jz with the union of all probe cylinders.
//
// A warp takes 32 consecutive poses (one per lane; consecutive poses of a
// trajectory are nearly identical) and walks the rows their cylinders reach
// in lockstep.  On a row each lane estimates its pose's interval in FP32
// (measured from the point of the row nearest the probe axis, so the estimate
// carries no cancellation) and proposes the voxels at least CORE_M inside it
// as its core; the core's two end voxels are classified exactly, and since the
// cylinder is convex both inside means the whole core is inside.  If the cores
// of all such lanes share a voxel, every lane's exact interval contains it, so
// the union of the lanes' intervals is one interval: the warp sets its known
// part [min core start, max core end] and extends it outward one voxel at a
// time, asking every lane to classify the voxel, until no lane holds it.
// Voxels already set in the slab are stepped over unclassified (they are in
// the result whatever this warp decides, and the union being an interval
// keeps the stop rule valid).  Lanes whose estimate is unusable (axis nearly
// along the row, short intervals, failed core ends, or cores that do not
// overlap) classify their row voxel by voxel with vox_row.
template <int N>
__device__ void voxelise_slab(const Geo &g, const RotRec &rr, const PoseRec *poses, int P, int jz, uint32_t *bits,
                              int *next_chunk)
{
    constexpr int NW = N / 32;
    // twice the bound on the FP32 error of the probe-frame coordinates l
    // (2e-4 voxels on lattices of <= 256 voxels), times a safety factor 2
    constexpr float ELB = 8e-4f;
    const float rv = g.rv, lv = g.lv, rv2 = rv * rv;
    const float mz = 8e-4f, mr = 1.6e-3f * rv + 1e-3f;
    const double h = g.h, r2d = g.r * g.r, Ld = g.L;
    const float ih = g.inv_h;
    const float *Rf = rr.Rf;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const float fz = (float)jz;
    const volatile uint32_t *vb = bits;
    (void)warp;
    (void)nwarp;
    for (;;) {
        // warps take chunks of 32 poses from a block-wide counter, so a warp
        // that drew chunks far from this slab goes on to the next chunk
        int base = 0;
        if (lane == 0) base = atomicAdd(next_chunk, 32);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= P) break;
        const int i = base + lane;
        bool hit = false;
        float B[9], c[3];
        int y0 = N, y1 = -1;
        if (i < P) {
            const PoseRec &pr = poses[i];
            float cz = (fmaf(Rf[2], pr.tf[0], fmaf(Rf[5], pr.tf[1], Rf[8] * pr.tf[2])) - rr.of[2]) * ih;
            float Az = fmaf(Rf[2], pr.Rf[2], fmaf(Rf[5], pr.Rf[5], Rf[8] * pr.Rf[8]));
            float sz = rv * sqrtf(fmaxf(0.f, 1.f - Az * Az)) + 1.5f;
            float z0 = fminf(cz, cz + lv * Az) - sz, z1 = fmaxf(cz, cz + lv * Az) + sz;
            if (!(fz < z0 || fz > z1)) {
                pose_frame(rr, pr, ih, B, c);
                float Ay = B[1 * 3 + 2];
                float u0, u1;
                if (fabsf(Az) > 1e-6f) {
                    float ua = (fz - c[2] - sz) / Az, ub = (fz - c[2] + sz) / Az;
                    u0 = fmaxf(0.f, fminf(ua, ub));
                    u1 = fminf(lv, fmaxf(ua, ub));
                } else {
                    u0 = 0.f;
                    u1 = lv;
                }
                if (u0 <= u1) {
                    float sy = rv * sqrtf(fmaxf(0.f, 1.f - Ay * Ay)) + 1.5f;
                    float ylo = c[1] + fminf(u0 * Ay, u1 * Ay) - sy, yhi = c[1] + fmaxf(u0 * Ay, u1 * Ay) + sy;
                    y0 = max(0, (int)ceilf(ylo));
                    y1 = min(N - 1, (int)floorf(yhi));
                    hit = y0 <= y1;
                }
            }
        }
        if (!__any_sync(0xFFFFFFFFu, hit)) continue;
        const int Y0 = __reduce_min_sync(0xFFFFFFFFu, hit ? y0 : N);
        const int Y1 = __reduce_max_sync(0xFFFFFFFFu, hit ? y1 : -1);
        const PoseRec &pr = poses[min(i, P - 1)];
        const float bx[3] = {B[0], B[1], B[2]};
        // per-pose constants of the row walk: the row direction in the probe frame
        const float Aq = fmaf(bx[0], bx[0], bx[1] * bx[1]);
        const bool radial_ok = Aq >= 0.05f;          // axis not within ~13 deg of the row direction
        const float iAq = radial_ok ? 1.f / Aq : 0.f;
        const bool cap_ok = fabsf(bx[2]) >= 1e-3f;     // cap crossings located to < 0.25 voxel
        const float ibz = cap_ok ? 1.f / bx[2] : 0.f;
        const float rsAq = radial_ok ? rsqrtf(Aq) : 0.f;
        const float ez = cap_ok ? ELB * fabsf(ibz) : 0.f;   // cap crossings: error of l2 / |bz|
        const float erq = ELB * rv * iAq;
        // l0(jy) = B^T ((0, jy, jz) - c) = B_y^T jy + base: one FMA per coordinate per row
        float lbase[3];
        for (int k = 0; k < 3; ++k) lbase[k] = fmaf(B[0 * 3 + k], -c[0], fmaf(B[1 * 3 + k], -c[1], B[2 * 3 + k] * (fz - c[2])));
        for (int jy = Y0; jy <= Y1; ++jy) {
            const bool act = hit && jy >= y0 && jy <= y1;
            int st = 0;            // 0: nothing, 1: exact interval [ia, ib], 2: walk voxel by voxel, 3: few candidates
            int ia = N, ib = -1;
            int qa = 0, qb = -1;   // st 3: the candidate voxels
            float l0[3];
            if (act) {
                for (int k = 0; k < 3; ++k) l0[k] = fmaf(B[1 * 3 + k], (float)jy, lbase[k]);
                if (!radial_ok) {
                    st = 2;
                } else {
                    // nearest point of the row to the axis, then the radial chord around it
                    const float js = -fmaf(l0[0], bx[0], l0[1] * bx[1]) * iAq;
                    const float sa = fmaf(js, bx[0], l0[0]), sb = fmaf(js, bx[1], l0[1]);
                    const float Cs = fmaf(sa, sa, sb * sb) - rv2;
                    const float disc = -Aq * Cs;
                    if (disc > 0.f) {
                        // (the rounding of an approximate square root and
                        // reciprocal, a few ulp, is far inside the 1e-5
                        // relative term added to E below)
                        const float hw = disc * rsqrtf(disc) * iAq;
                        float lo = js - hw, hi = js + hw;
                        // error of the chord ends: a radius error dl moves a crossing
                        // by about dl rv / (Aq hw), the nearest point by dl / sqrt(Aq)
                        float E = fmaf(erq, __frcp_rn(hw), ELB * rsAq);
                        bool empty = false, unsure = false;
                        if (cap_ok) {
                            const float za = -l0[2] * ibz, zb = (lv - l0[2]) * ibz;
                            lo = fmaxf(lo, fminf(za, zb));
                            hi = fminf(hi, fmaxf(za, zb));
                            E = fmaxf(E, ez);
                        } else {
                            // row nearly parallel to the cap planes: z moves < N/1000 voxels along it
                            const float zA = l0[2], zB = fmaf((float)(N - 1), bx[2], l0[2]);
                            const float zmin = fminf(zA, zB), zmax = fmaxf(zA, zB);
                            if (zmax < -0.3f || zmin > lv + 0.3f) empty = true;
                            else if (!(zmin >= 0.3f && zmax <= lv - 0.3f)) unsure = true;
                        }
                        E += 1e-5f * fmaxf(fabsf(lo), fabsf(hi));   // rounding of lo, hi themselves
                        if (empty || lo > (float)N + 1.f || hi < -2.f || lo > hi + 2.f) {
                            st = 0;
                        } else if (unsure || E > 0.25f) {
                            st = 2;
                        } else if (hi - lo < 2.f * E + 1.f) {
                            // short chord: its voxels lie in [lo - E, hi + E]
                            st = 3;
                            qa = max(0, (int)floorf(fmaxf(lo - E, -1.f)));
                            qb = min(N - 1, (int)ceilf(fminf(hi + E, (float)N)));
                        } else {
                            // voxels below lo - E are outside, those in (lo + E, hi - E)
                            // inside (the cylinder is convex); an integer in either
                            // band is classified exactly
                            st = 1;
                            int ka = (int)ceilf(lo - E), kb = (int)floorf(hi + E);
                            ia = ka;
                            if ((float)ka <= lo + E && ka >= 0 && ka < N &&
                                !classify(l0, bx, ka, rv2, lv, mr, mz, rr, pr, h, r2d, Ld, jy, jz))
                                ia = ka + 1;
                            ib = kb;
                            if ((float)kb >= hi - E && kb >= 0 && kb < N &&
                                !classify(l0, bx, kb, rv2, lv, mr, mz, rr, pr, h, r2d, Ld, jy, jz))
                                ib = kb - 1;
                            ia = max(ia, 0);
                            ib = min(ib, N - 1);
                            if (ia > ib) st = 0;
                        }
                    } else if (disc > -1e-2f * (1.f + fabsf(Aq * rv2))) {
                        // tangent row: the exact chord (if any) is within a quarter
                        // voxel of js
                        st = 3;
                        qa = max(0, (int)floorf(fmaxf(js, -2.f)) - 1);
                        qb = min(N - 1, (int)ceilf(fminf(js, (float)N + 1.f)) + 1);
                    }
                }
            }
            // exact intervals: one union when they overlap (the usual case for
            // consecutive poses), else each lane sets its own
            if (__any_sync(0xFFFFFFFFu, st == 1)) {
                const int A = __reduce_min_sync(0xFFFFFFFFu, st == 1 ? ia : N);
                const int Bm = __reduce_max_sync(0xFFFFFFFFu, st == 1 ? ib : -1);
                const int mxa = __reduce_max_sync(0xFFFFFFFFu, st == 1 ? ia : -1);
                const int mnb = __reduce_min_sync(0xFFFFFFFFu, st == 1 ? ib : N);
                if (mxa <= mnb + 1) {
                    if (lane < NW) {
                        const int lo = max(A, 32 * lane) - 32 * lane, hi = min(Bm, 32 * lane + 31) - 32 * lane;
                        if (lo <= hi) {
                            const uint32_t m = (hi == 31 ? 0xFFFFFFFFu : ((1u << (hi + 1)) - 1u)) & ~((1u << lo) - 1u);
                            if (m & ~vb[jy * NW + lane]) atomicOr(&bits[jy * NW + lane], m);
                        }
                    }
                } else if (st == 1) {
                    set_bits(bits + jy * NW, ia, ib);
                }
            }
            // short chords: the lanes classify their few candidate voxels together
            if (__any_sync(0xFFFFFFFFu, st == 3)) {
                const int len = (st == 3) ? qb - qa + 1 : 0;
                const int maxlen = __reduce_max_sync(0xFFFFFFFFu, len);
                for (int k = 0; k < maxlen; ++k) {
                    const int j = qa + k;
                    bool in = false;
                    if (k < len && !((vb[jy * NW + (j >> 5)] >> (j & 31)) & 1u))
                        in = classify(l0, bx, j, rv2, lv, mr, mz, rr, pr, h, r2d, Ld, jy, jz);
                    if (in) atomicOr(&bits[jy * NW + (j >> 5)], 1u << (j & 31));
                }
            }
            if (st == 2) vox_row<N>(B, c, jy, jz, rv2, lv, mr, mz, rr, pr, h, r2d, Ld, bits + jy * NW);
        }
    }
}

// Geometry of the request that rotation rr belongs to.
__device__ __forceinline__ Geo req_geo(const Geo &g, const ReqDev &q)
{
    Geo r = g;
    r.h = q.h;
    r.inv_h = q.inv_h;
    r.rv = q.rv;
    r.lv = q.lv;
    r.r = q.r;
    r.L = q.L;
    return r;
}

// S_b slab bits to global memory: bits[((b * N + jz) * N + jy) * NW + w].
// MINB: resident 256-thread blocks per SM the register allocation is built for
// (3: up to 80 registers; 4: 64 registers, a few spills); the autotuner picks
// one.  The launches use blocks of 128 threads, twice as many per SM.
template <int N, int MINB>
__global__ void __launch_bounds__(256, MINB)
k_voxelise(Geo g, const ReqDev *reqs, const RotRec *rots, uint32_t *bits_out, int pose_set)
{
    constexpr int NW = N / 32;
    __shared__ uint32_t bits[N * NW];
    __shared__ int next_chunk;
    // slabs from the lattice centre outward (the swept volume is centred, so
    // the heaviest slabs of every rotation are scheduled first)
    const int k = blockIdx.y, b = blockIdx.x;
    const int jz = N / 2 + ((k & 1) ? -((k + 1) >> 1) : (k >> 1));
    for (int i = threadIdx.x; i < N * NW; i += blockDim.x) bits[i] = 0u;
    if (threadIdx.x == 0) next_chunk = 0;
    __syncthreads();
    const RotRec &rr = rots[b];
    const ReqDev &q = reqs[rr.req];
    if (q.rotate_object) return;   // its grid is the resampled object, made in k_fwd2d
    voxelise_slab<N>(req_geo(g, q), rr, pose_set ? q.poses_nc : q.poses, pose_set ? q.P_nc : q.P, jz, bits,
                     &next_chunk);
    __syncthreads();
    uint32_t *o = bits_out + ((size_t)b * N + jz) * N * NW;
    for (int i = threadIdx.x; i < N * NW; i += blockDim.x) o[i] = bits[i];
}

template <int MINB>
static cudaError_t launch_voxelise_t(const Geo &g, const ReqDev *reqs, const RotRec *rots, int B, uint32_t *bits,
                                     cudaStream_t st, int ps)
{
    dim3 grid(B, g.N);
    // 4 warps per slab block: a block waits at its barriers for the warps
    // that found poses, and smaller blocks wait less (38 -> 34 us per rotation
    // at 128^3 for the label-aware pass's 1000 non-contact poses, 48.6 -> 48.0
    // us for the 5000 contact poses); the register target is that of
    // 256-thread blocks, so twice as many blocks are resident
    const int nt = 128;
    switch (g.N) {
    case 32: k_voxelise<32, MINB><<<grid, nt, 0, st>>>(g, reqs, rots, bits, ps); break;
    case 64: k_voxelise<64, MINB><<<grid, nt, 0, st>>>(g, reqs, rots, bits, ps); break;
    case 96: k_voxelise<96, MINB><<<grid, nt, 0, st>>>(g, reqs, rots, bits, ps); break;
    case 128: k_voxelise<128, MINB><<<grid, nt, 0, st>>>(g, reqs, rots, bits, ps); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_voxelise(const Geo &g, const ReqDev *reqs, const RotRec *rots, int B, uint32_t *bits,
                            cudaStream_t st, int minb, int pose_set)
{
    if (B < 1 || B > 65535 || (pose_set != 0 && pose_set != 1)) return cudaErrorInvalidValue;
    switch (minb) {
    case 3: return launch_voxelise_t<3>(g, reqs, rots, B, bits, st, pose_set);
    case 4: return launch_voxelise_t<4>(g, reqs, rots, B, bits, st, pose_set);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// K_A: forward transform of slab z of S_b along x (R2C in closed form per run
// of set bits) and y (radix FFT, N non-zero inputs of M); writes Y[b][z].
// ---------------------------------------------------------------------------
// Shared-memory layout of k_fwd2d (complex elements unless noted): X [N][H]
// plus 4N bytes of slack (the resampled slab's row pairs overhang X by that
// much), the exchange buffer (the FFT's [M][32], or [32][M + 1] for the
// resampled rows), twiddles [M], column 0 after the y FFT [M], bits [N][N/32].
template <int M> struct Fwd2dSmem {
    static constexpr int N = M / 2, H = M / 2;
    static constexpr size_t X_BYTES = (size_t)N * H * 8 + ((4 * N + 15) / 16) * 16;
    static constexpr size_t XB_ELEMS = (size_t)32 * (M + 1);
    static constexpr size_t BYTES = X_BYTES + 8 * (XB_ELEMS + 2 * M) + 4 * (size_t)N * (N / 32);
    static_assert(BYTES <= 227 * 1024, "fwd2d shared memory");
};

// Sec. IV-D as printed, x stage: slab z of the rotated object grid (trilinear
// resampling of O, lanes along x so that neighbouring lanes read neighbouring
// corners) is transformed along x two rows at a time, rows 2p and 2p+1 as the
// real and imaginary parts of one complex FFT, and unpacked into X[y][kx]
// (kx in [0, H); column 0 holds the real kx = 0 and kx = H values as one
// complex number, as the closed-form path stores them).  The row pairs sit in
// the upper half of X's bytes as float2 [N/2][N + 1]: the pairs a round reads
// are loaded into registers before its outputs overwrite that memory, and
// later rounds' pairs lie above what a round writes.
template <int M, int V = 0>
__device__ __forceinline__ void resampled_x_stage(const RotRec &rr, const ReqDev &q, int jz, cf *X, cf *xbt, cf *xb,
                                                  const cf *tw, const float *slab)
{
    constexpr int N = M / 2, H = M / 2, COLS = 32, E = Plan<M, V>::E, NP = N / 2, PP = N + 1;
    float2 *pairs = reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(X) + (size_t)N * H * 4);
    if (slab) {
        // the slab resampled beforehand by k_resample (N x N floats)
        for (int i = threadIdx.x; i < NP * N; i += blockDim.x) {
            const int x = i % N, p = i / N;
            pairs[p * PP + x] = make_float2(slab[(2 * p) * N + x], slab[(2 * p + 1) * N + x]);
        }
    } else {
        const float4 *O = q.Og4;
#pragma unroll 4
        for (int i = threadIdx.x; i < NP * N; i += blockDim.x) {
            const int x = i % N, p = i / N;
            pairs[p * PP + x] = make_float2(rotated_object_voxel(rr, O, N, x, 2 * p, jz),
                                            rotated_object_voxel(rr, O, N, x, 2 * p + 1, jz));
        }
    }
    __syncthreads();
    const int c = threadIdx.x % COLS, j = threadIdx.x / COLS;
    for (int p0 = 0; p0 < NP; p0 += COLS) {
        const int p = p0 + c;
        cf v[E];
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const int x = in_index<M, V>(j, s);
            float2 t = make_float2(0.f, 0.f);
            if (slot_in_lower_half<M, V>(s) && p < NP) t = pairs[p * PP + x];   // x < N
            v[s] = cmake(t.x, t.y);
        }
        fft_column<M, false, 1, V>(v, j, xb, c, COLS, tw);
        __syncthreads();   // every pair of this round is in registers before X is written
#pragma unroll
        for (int s = 0; s < E; ++s) xbt[c * (M + 1) + out_index<M, V>(j, s)] = v[s];
        __syncthreads();
        for (int e = threadIdx.x; e < COLS * H; e += blockDim.x) {
            const int kx = e % H, cc = e / H, pp = p0 + cc;
            if (pp >= NP) continue;
            const cf *col = xbt + cc * (M + 1);
            const cf a = col[kx];
            cf A, B;
            if (kx == 0) {
                const cf hq = col[H];
                A = cmake(a.x, hq.x);
                B = cmake(a.y, hq.y);
            } else {
                const cf r = col[M - kx];
                A = cmake(0.5f * (a.x + r.x), 0.5f * (a.y - r.y));
                B = cmake(0.5f * (a.y + r.y), -0.5f * (a.x - r.x));
            }
            X[(2 * pp) * H + kx] = A;
            X[(2 * pp + 1) * H + kx] = B;
        }
        __syncthreads();
    }
}

// Closed-form x stage on binary data: X[y][kx] = sum over runs [a, a+len) of
// set bits of sum_x w^(kx x) = (w^(kx a) - w^(kx (a+len))) / (1 - w^kx)
// (kx != 0), the Nyquist column packed into column 0 (bits & ~mask when a
// mask is given).
template <int M>
__device__ __forceinline__ void bits_x_stage(const uint32_t *bits_g, const uint32_t *mask_g, int b, int jz, cf *X,
                                             uint32_t *bits, const cf *tw, const float2 *q_g)
{
    constexpr int N = M / 2, H = M / 2, NW = N / 32;
    const uint32_t *bg = bits_g + ((size_t)b * N + jz) * N * NW;
    if (mask_g) {
        const uint32_t *mg = mask_g + ((size_t)b * N + jz) * N * NW;
        for (int i = threadIdx.x; i < N * NW; i += blockDim.x) bits[i] = bg[i] & ~mg[i];
    } else {
        for (int i = threadIdx.x; i < N * NW; i += blockDim.x) bits[i] = bg[i];
    }
    __syncthreads();

    // x: X[y][kx] = sum over runs [a, a+len) of sum_x exp(-2 pi i kx x / M)
    //             = (w^(kx a) - w^(kx (a+len))) / (1 - w^kx)   (kx != 0)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    constexpr int KPL = H / 32;   // kx values per lane
    cf qv[KPL];
#pragma unroll
    for (int m = 0; m < KPL; ++m) { float2 t = q_g[lane + 32 * m]; qv[m] = cmake(t.x, t.y); }
    for (int y = warp; y < N; y += nwarp) {
        cf acc[KPL];
#pragma unroll
        for (int m = 0; m < KPL; ++m) acc[m] = cmake(0.f, 0.f);
        float nyq = 0.f;
        uint32_t prevw = 0;
        int open = -1;
        for (int w = 0; w <= NW; ++w) {
            uint32_t cur = (w < NW) ? bits[y * NW + w] : 0u;
            uint32_t prev = (cur << 1) | (prevw >> 31);
            uint32_t rise = cur & ~prev, fall = ~cur & prev;
            uint32_t ev = rise | fall;
            while (ev) {
                int bpos = __ffs(ev) - 1;
                ev &= ev - 1;
                int xpos = w * 32 + bpos;
                if ((rise >> bpos) & 1u) {
                    open = xpos;
                } else {
                    int a = open, len = xpos - open;
#pragma unroll
                    for (int m = 0; m < KPL; ++m) {
                        int kx = lane + 32 * m;
                        if (kx == 0) {
                            acc[m].x += (float)len;
                        } else {
                            int i0 = (kx * a) % M, i1 = (kx * (a + len)) % M;
                            acc[m] = cadd(acc[m], cmul(csub(tw[i0], tw[i1]), qv[m]));
                        }
                    }
                    if (len & 1) nyq += (a & 1) ? -1.f : 1.f;
                    open = -1;
                }
            }
            prevw = cur;
        }
#pragma unroll
        for (int m = 0; m < KPL; ++m) {
            int kx = lane + 32 * m;
            cf val = acc[m];
            if (kx == 0) val.y = nyq;          // pack the Nyquist column into column 0
            X[y * H + kx] = val;
        }
    }
}

template <int M, int V = 0>
__global__ void __launch_bounds__(Plan<M, V>::T * 32)
k_fwd2d(int P, const uint32_t *bits_g, float2 *Y, const float2 *tw_g, const float2 *q_g, const uint32_t *mask_g,
        const RotRec *rots, const ReqDev *reqs, const float *ogrids)
{
    constexpr int N = M / 2, H = M / 2, COLS = 32, E = Plan<M, V>::E;
    using L = Fwd2dSmem<M>;
    extern __shared__ __align__(16) unsigned char smem[];
    cf *X = reinterpret_cast<cf *>(smem);                       // [N][H] packed columns
    cf *xb = reinterpret_cast<cf *>(smem + L::X_BYTES);         // [M][COLS] exchange (or [COLS][M + 1])
    cf *tw = xb + L::XB_ELEMS;                                   // [M]
    cf *c0 = tw + M;                                             // [M] packed column 0 after the y FFT
    uint32_t *bits = reinterpret_cast<uint32_t *>(c0 + M);       // [N][NW]

    const int jz = blockIdx.x, b = blockIdx.y;
    const bool resample = rots && reqs[rots[b].req].rotate_object;
    if (resample && mask_g) return;   // no second (non-contact) grid for a rotated object
    for (int i = threadIdx.x; i < M; i += blockDim.x) { float2 w = tw_g[i]; tw[i] = cmake(w.x, w.y); }
    if (resample) {
        __syncthreads();
        resampled_x_stage<M, V>(rots[b], reqs[rots[b].req], jz, X, xb, xb, tw,
                             ogrids ? ogrids + ((size_t)b * (M / 2) + jz) * (M / 2) * (M / 2) : nullptr);
    } else {
        bits_x_stage<M>(bits_g, mask_g, b, jz, X, bits, tw, q_g);
    }
    __syncthreads();

    // y: FFT of each packed column; thread (c, j) of a round of 32 columns
    // stores ky = out_index(j, s) for column p0 + c: a warp writes 32
    // consecutive kx (256 contiguous bytes).  Column 0 carries kx = 0 + i kx = M/2
    // and is unpacked from its ky and M - ky outputs.
    float2 *Yb = Y + ((size_t)b * N + jz) * (size_t)M * P;
    const int c = threadIdx.x % COLS, j = threadIdx.x / COLS;
    for (int p0 = 0; p0 < H; p0 += COLS) {
        cf v[E];
#pragma unroll
        for (int s = 0; s < E; ++s) {
            int yy = in_index<M, V>(j, s);
            v[s] = slot_in_lower_half<M, V>(s) ? X[yy * H + p0 + c] : cmake(0.f, 0.f);   // yy < N
        }
        fft_column<M, false, 1, V>(v, j, xb, c, COLS, tw);
        const int kx = p0 + c;
#pragma unroll
        for (int s = 0; s < E; ++s) {
            int ky = out_index<M, V>(j, s);
            if (kx == 0) c0[ky] = v[s];
            else Yb[ky * P + kx] = make_float2(v[s].x, v[s].y);
        }
        __syncthreads();
    }
    for (int ky = threadIdx.x; ky < M; ky += blockDim.x) {
        cf val = c0[ky], oc = cconj(c0[(M - ky) % M]);
        cf y0 = cscale(cadd(val, oc), 0.5f);
        cf w = csub(val, oc);
        float2 *row = Yb + ky * P;
        row[0] = make_float2(y0.x, y0.y);
        row[H] = make_float2(0.5f * w.y, -0.5f * w.x);
        for (int k2 = H + 1; k2 < P; ++k2) row[k2] = make_float2(0.f, 0.f);
    }
}

template <int M, int V = 0>
static cudaError_t launch_fwd2d_t(const Geo &g, int B, const uint32_t *bits, float2 *Y, const float2 *tw,
                                  const float2 *q, cudaStream_t st, const uint32_t *mask, const RotRec *rots,
                                  const ReqDev *reqs, const float *ogrids)
{
    size_t sm = Fwd2dSmem<M>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(k_fwd2d<M, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_fwd2d<M, V><<<dim3(M / 2, B), Plan<M, V>::T * 32, sm, st>>>(g.P, bits, Y, tw, q, mask, rots, reqs, ogrids);
    return cudaGetLastError();
}

cudaError_t launch_fwd2d(const Geo &g, int B, const uint32_t *bits, float2 *Y, const float2 *tw, const float2 *q,
                         cudaStream_t st, const uint32_t *mask, const RotRec *rots, const ReqDev *reqs,
                         const float *ogrids, int fft_plan)
{
    if ((rots == nullptr) != (reqs == nullptr)) return cudaErrorInvalidValue;
    switch (g.M) {
    case 64:
        return fft_plan == 1 ? launch_fwd2d_t<64, 1>(g, B, bits, Y, tw, q, st, mask, rots, reqs, ogrids)
                             : launch_fwd2d_t<64>(g, B, bits, Y, tw, q, st, mask, rots, reqs, ogrids);
    case 128:
        return fft_plan == 1 ? launch_fwd2d_t<128, 1>(g, B, bits, Y, tw, q, st, mask, rots, reqs, ogrids)
                             : launch_fwd2d_t<128>(g, B, bits, Y, tw, q, st, mask, rots, reqs, ogrids);
    case 192: return launch_fwd2d_t<192>(g, B, bits, Y, tw, q, st, mask, rots, reqs, ogrids);
    case 256: return launch_fwd2d_t<256>(g, B, bits, Y, tw, q, st, mask, rots, reqs, ogrids);
    default: return cudaErrorInvalidValue;
    }
}

// Bits of S_b to a byte array (test hook): the production voxeliser, then
// one byte per voxel.
template <int N>
__global__ void __launch_bounds__(256) k_vox_export(Geo g, const ReqDev *reqs, const RotRec *rots, uint8_t *out,
                                                    int pose_set)
{
    constexpr int NW = N / 32;
    __shared__ uint32_t bits[N * NW];
    __shared__ int next_chunk;
    const int jz = blockIdx.x, b = blockIdx.y;
    for (int i = threadIdx.x; i < N * NW; i += blockDim.x) bits[i] = 0u;
    if (threadIdx.x == 0) next_chunk = 0;
    __syncthreads();
    const RotRec &rr = rots[b];
    const ReqDev &q = reqs[rr.req];
    voxelise_slab<N>(req_geo(g, q), rr, pose_set ? q.poses_nc : q.poses, pose_set ? q.P_nc : q.P, jz, bits,
                     &next_chunk);
    __syncthreads();
    uint8_t *o = out + ((size_t)b * N + jz) * N * N;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        int y = i / N, x = i % N;
        o[i] = (bits[y * NW + (x >> 5)] >> (x & 31)) & 1u;
    }
}

cudaError_t launch_vox_export(const Geo &g, const ReqDev *reqs, const RotRec *rots, int B, uint8_t *bits,
                              cudaStream_t st, int ps)
{
    dim3 grid(g.N, B);
    if (ps != 0 && ps != 1) return cudaErrorInvalidValue;
    switch (g.N) {
    case 32: k_vox_export<32><<<grid, 256, 0, st>>>(g, reqs, rots, bits, ps); break;
    case 64: k_vox_export<64><<<grid, 256, 0, st>>>(g, reqs, rots, bits, ps); break;
    case 96: k_vox_export<96><<<grid, 256, 0, st>>>(g, reqs, rots, bits, ps); break;
    case 128: k_vox_export<128><<<grid, 256, 0, st>>>(g, reqs, rots, bits, ps); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// S of rotation 0 as floats (the fixed swept grid whose spectrum a rotated
// object is correlated with).
template <int N>
__global__ void __launch_bounds__(256) k_vox_float(Geo g, const ReqDev *reqs, const RotRec *rots, float *out)
{
    constexpr int NW = N / 32;
    __shared__ uint32_t bits[N * NW];
    __shared__ int next_chunk;
    const int jz = blockIdx.x;
    for (int i = threadIdx.x; i < N * NW; i += blockDim.x) bits[i] = 0u;
    if (threadIdx.x == 0) next_chunk = 0;
    __syncthreads();
    const RotRec &rr = rots[0];
    const ReqDev &q = reqs[rr.req];
    voxelise_slab<N>(req_geo(g, q), rr, q.poses, q.P, jz, bits, &next_chunk);
    __syncthreads();
    float *o = out + (size_t)jz * N * N;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        int y = i / N, x = i % N;
        o[i] = (float)((bits[y * NW + (x >> 5)] >> (x & 31)) & 1u);
    }
}

cudaError_t launch_vox_float(const Geo &g, const ReqDev *reqs, const RotRec *rots, float *out, cudaStream_t st)
{
    switch (g.N) {
    case 32: k_vox_float<32><<<g.N, 256, 0, st>>>(g, reqs, rots, out); break;
    case 64: k_vox_float<64><<<g.N, 256, 0, st>>>(g, reqs, rots, out); break;
    case 96: k_vox_float<96><<<g.N, 256, 0, st>>>(g, reqs, rots, out); break;
    case 128: k_vox_float<128><<<g.N, 256, 0, st>>>(g, reqs, rots, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The resampled object grid of rotation b, slab z (test hook; the same voxel
// function as the fused x stage).
__global__ void __launch_bounds__(256) k_rot_export(int N, const ReqDev *reqs, const RotRec *rots, float *out)
{
    const int jz = blockIdx.x, b = blockIdx.y;
    const RotRec &rr = rots[b];
    const ReqDev &q = reqs[rr.req];
    float *o = out + ((size_t)b * N + jz) * N * N;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) o[i] = rotated_object_voxel(rr, q.Og4, N, i % N, i / N, jz);
}

// The rotated object grids of a launch's rotate_object rotations, slab by
// slab at full occupancy (the fused x stage of k_fwd2d runs one CTA per SM,
// too few warps to hide the corner-cell loads); other rotations are skipped.
template <int N>
__global__ void __launch_bounds__(256) k_resample(const ReqDev *reqs, const RotRec *rots, float *out)
{
    const int jz = blockIdx.x, b = blockIdx.y;
    const RotRec &rr = rots[b];
    const ReqDev &q = reqs[rr.req];
    if (!q.rotate_object) return;
    float *o = out + ((size_t)b * N + jz) * N * N;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) o[i] = rotated_object_voxel(rr, q.Og4, N, i % N, i / N, jz);
}

cudaError_t launch_resample(const Geo &g, const ReqDev *reqs, const RotRec *rots, int B, float *out, cudaStream_t st)
{
    if (B < 1 || B > 65535) return cudaErrorInvalidValue;
    dim3 grid(g.N, B);
    switch (g.N) {
    case 32: k_resample<32><<<grid, 256, 0, st>>>(reqs, rots, out); break;
    case 64: k_resample<64><<<grid, 256, 0, st>>>(reqs, rots, out); break;
    case 96: k_resample<96><<<grid, 256, 0, st>>>(reqs, rots, out); break;
    case 128: k_resample<128><<<grid, 256, 0, st>>>(reqs, rots, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rot_export(const Geo &g, const ReqDev *reqs, const RotRec *rots, int B, float *out, cudaStream_t st)
{
    if (B < 1 || B > 65535) return cudaErrorInvalidValue;
    k_rot_export<<<dim3(g.N, B), 256, 0, st>>>(g.N, reqs, rots, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K_B: per chunk of 32 columns f = ky P + kx: forward FFT along z (N non-zero
// inputs), multiply by conj(F(O)) / M^3 (for a rotated object: conjugate the
// tile, multiply by F(S) / M^3), inverse FFT along z.  The spectrum
// of the chunk stays in registers across the `group` rotations of the block.
// DUAL (label-aware score): each rotation has a second tile, Y2, the
// transform of the voxels reached only by non-contact poses; its product
// with conj(F(min(O, 0))) / M^3 is added before the inverse FFT, so one
// inverse transform yields the sum of both correlations.  Requests without
// non-contact poses skip the addition and keep the plain result bit for bit.
// ---------------------------------------------------------------------------
template <int M, bool DUAL, int V = 0>
__global__ void __launch_bounds__(Plan<M, V>::T * 32)
k_zpass(int P, int B, int group, const float2 *Y, const float2 *Y2, const RotRec *rots, const ReqDev *reqs, float2 *Z,
        const float2 *tw_g)
{
    constexpr int N = M / 2, E = Plan<M, V>::E, COLS = 32;
    constexpr int R_LAST = Plan<M, V>::R(Plan<M, V>::S - 1);
    constexpr int TPR = DUAL ? 2 : 1;        // tiles per rotation
    extern __shared__ __align__(16) unsigned char smem[];
    cf *xb = reinterpret_cast<cf *>(smem);   // [M][COLS]
    cf *tw = xb + M * COLS;                  // [M]
    cf *yt = tw + M;                         // two [N][COLS] tiles of Y (double buffer)
    for (int i = threadIdx.x; i < M; i += blockDim.x) { float2 w = tw_g[i]; tw[i] = cmake(w.x, w.y); }
    const int chunk = blockIdx.x;
    const int c = threadIdx.x % COLS, j = threadIdx.x / COLS;
    const size_t plane = (size_t)M * P;
    const size_t f0 = (size_t)chunk * COLS;
    const int b0 = blockIdx.y * group;
    const int nb = min(group, B - b0);
    const int nt = nb * TPR;
    // spectrum values in input-slot order of the inverse transform: slot
    // s <-> kz = j + (M/E) s; held in registers across the block's rotations
    // and reloaded when the request (object) changes
    cf sp[E];
    int sp_req = -1;
    // asynchronous copy of tile t's non-zero z rows of this chunk (coalesced 256-byte rows)
    auto prefetch = [&](int t) {
        const float2 *src = (DUAL && (t & 1)) ? Y2 : Y;
        const float2 *Yb = src + (size_t)(b0 + t / TPR) * N * plane + f0;
        cf *dst = yt + (t & 1) * N * COLS;
        for (int e = threadIdx.x; e < N * COLS; e += blockDim.x) cp_async8(&dst[e], &Yb[(size_t)(e / COLS) * plane + e % COLS]);
        cp_async_commit();
    };
    if (nt > 0) prefetch(0);
    cf w[E];
    for (int t = 0; t < nt; ++t) {
        if (t + 1 < nt) {
            prefetch(t + 1);
            cp_async_wait_one();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        const int bi = t / TPR;
        const bool second = DUAL && (t & 1);
        const int req = rots[b0 + bi].req;
        if (!second && req != sp_req) {
            const float2 *spec = reqs[req].spec;
#pragma unroll
            for (int s = 0; s < E; ++s) {
                float2 v = spec[((size_t)chunk * M + (j + (M / E) * s)) * COLS + c];
                sp[s] = cmake(v.x, v.y);
            }
            sp_req = req;
        }
        const cf *src = yt + (t & 1) * N * COLS;
        cf v[E];
#pragma unroll
        for (int s = 0; s < E; ++s) {
            int z = in_index<M, V>(j, s);
            v[s] = slot_in_lower_half<M, V>(s) ? src[z * COLS + c] : cmake(0.f, 0.f);   // z < N
        }
        fft_column<M, false, 1, V>(v, j, xb, c, COLS, tw);
        // forward output slot (bb, r) holds kz = j + (M/E)(bb + (E/R_LAST) r)
        if (!second) {
            // a rotated object: this tile is F(O_R) and spec is F(S) / M^3,
            // so the product is conj(F(O_R)) F(S) / M^3 (Eq. (9) read as Eq. (7))
            const float cj = reqs[req].rotate_object ? -1.f : 1.f;
#pragma unroll
            for (int bb = 0; bb < E / R_LAST; ++bb)
#pragma unroll
                for (int r = 0; r < R_LAST; ++r) {
                    int k = bb + (E / R_LAST) * r;
                    cf a = v[bb * R_LAST + r];
                    a.y *= cj;
                    w[k] = cmul(a, sp[k]);
                }
        } else if (reqs[req].P_nc > 0) {
            const float2 *pen = reqs[req].spec_pen;
#pragma unroll
            for (int bb = 0; bb < E / R_LAST; ++bb)
#pragma unroll
                for (int r = 0; r < R_LAST; ++r) {
                    int k = bb + (E / R_LAST) * r;
                    float2 q = pen[((size_t)chunk * M + (j + (M / E) * k)) * COLS + c];
                    w[k] = cadd(w[k], cmul(v[bb * R_LAST + r], cmake(q.x, q.y)));
                }
        }
        if (!DUAL || second) {
            __syncthreads();
            fft_column<M, true, 1, V>(w, j, xb, c, COLS, tw);
            float2 *Zb = Z + (size_t)(b0 + bi) * M * plane + f0 + c;
#pragma unroll
            for (int s = 0; s < E; ++s) {
                int z = out_index<M, V>(j, s);
                Zb[(size_t)z * plane] = make_float2(w[s].x, w[s].y);
            }
        }
        __syncthreads();
    }
}

template <int MM, bool DUAL, int V = 0>
static cudaError_t launch_zpass_t(const Geo &g, dim3 grid, int B, int group, const float2 *Y, const float2 *Y2,
                                  const RotRec *rots, const ReqDev *reqs, float2 *Z, const float2 *tw, cudaStream_t st)
{
    size_t sm = sizeof(cf) * ((size_t)MM * 32 + MM + (size_t)MM * 32);
    cudaError_t e = cudaFuncSetAttribute(k_zpass<MM, DUAL, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_zpass<MM, DUAL, V><<<grid, Plan<MM, V>::T * 32, sm, st>>>(g.P, B, group, Y, Y2, rots, reqs, Z, tw);
    return cudaGetLastError();
}

cudaError_t launch_zpass(const Geo &g, int B, int group, const float2 *Y, const RotRec *rots, const ReqDev *reqs,
                         float2 *Z, const float2 *tw, cudaStream_t st, const float2 *Y2, int fft_plan)
{
    int chunks = g.M * g.P / 32;
    dim3 grid(chunks, (B + group - 1) / group);
    switch (g.M) {
#define ZCASE(MM, V)                                                                                 \
        return Y2 ? launch_zpass_t<MM, true, V>(g, grid, B, group, Y, Y2, rots, reqs, Z, tw, st)     \
                  : launch_zpass_t<MM, false, V>(g, grid, B, group, Y, nullptr, rots, reqs, Z, tw, st);
    case 64:
        if (fft_plan == 1) ZCASE(64, 1)
        ZCASE(64, 0)
    case 128:
        if (fft_plan == 1) ZCASE(128, 1)
        ZCASE(128, 0)
    case 192: ZCASE(192, 0)
    case 256: ZCASE(256, 0)
#undef ZCASE
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// K_C: plane z of rotation b: inverse FFT along y of every packed column
// (column 0 carries kx = 0 + i kx = M/2), then C2R along x of every row by a
// half-length complex inverse FFT, and the argmax with the lowest linear
// index on ties.  For M = 256 the plane (256 KB) is split over a 2-CTA
// cluster; each CTA reads the other half of its rows through distributed
// shared memory.
// ---------------------------------------------------------------------------
template <int M, int V = 0> struct PlaneCfg {
    static constexpr int CL = (M >= 256) ? 2 : 1;          // CTAs per plane
    static constexpr int H = M / 2;
    static constexpr int VH = HasPlan<H, V>::value ? V : 0;   // the C2R's plan (length H)
    static constexpr int PC = H / CL;                      // packed columns per CTA
    static constexpr int PP = PC + 1;                      // odd pitch: a warp's rows hit distinct banks
    static constexpr int NT = Plan<M, V>::T * 32;             // threads
    static constexpr int COLS = 32;                        // columns per round of the y transform
    static constexpr int RPR = NT / Plan<H, VH>::T;            // rows per round of the C2R
    static constexpr int S1 = M * COLS;                    // phase-1 exchange
    static constexpr int S2 = CL > 1 ? (M / CL) * PP : 0;  // peer rows (cluster only)
    static constexpr int S3 = H * RPR;                     // phase-2 exchange (single CTA)
    static constexpr int STG = S1 > S2 ? (S1 > S3 ? S1 : S3) : (S2 > S3 ? S2 : S3);
    static constexpr size_t SMEM = sizeof(cf) * ((size_t)M * PP + STG + 2 * M);   // + twiddles + Nyquist column
    static_assert(SMEM <= 227 * 1024, "plane pass exceeds the shared memory of one CTA");
};

template <int M, bool EXPORT, int V = 0>
__device__ __forceinline__ void plane_body(const float2 *Zp, const float2 *tw_g, unsigned long long *key, float *Cout,
                                           int zc, cf *pb, cf *stg, cf *tw, int rank)
{
    using C = PlaneCfg<M, V>;
    constexpr int VH = C::VH;
    constexpr int H = M / 2, CL = C::CL, PC = C::PC, PP = C::PP, E = Plan<M, V>::E, COLS = C::COLS;
    const int P = H + 2;
    for (int i = threadIdx.x; i < M; i += blockDim.x) { float2 w = tw_g[i]; tw[i] = cmake(w.x, w.y); }
    __syncthreads();
    // phase 1: this CTA's packed columns, all ky, are copied asynchronously
    // into pb, one copy group per round of COLS columns (all in flight at
    // once; a round starts as soon as its own group has landed), column 0 is
    // packed with the Nyquist column (W0 + i W_{M/2}), and each column is
    // inverse transformed along y in place: pb[ky][col] -> pb[y][col].
    {
        constexpr int NR = (PC + COLS - 1) / COLS;
        static_assert(NR <= 4, "copy groups");
        cf *nyq = tw + M;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int p0 = r * COLS, nc = (PC - p0) < COLS ? (PC - p0) : COLS;
            for (int e = threadIdx.x; e < M * nc; e += blockDim.x) {
                int ky = e / nc, pl = p0 + e % nc;
                cp_async8(&pb[ky * PP + pl], &Zp[ky * P + rank * PC + pl]);
            }
            if (r == 0 && rank == 0)
                for (int ky = threadIdx.x; ky < M; ky += blockDim.x) cp_async8(&nyq[ky], &Zp[ky * P + H]);
            cp_async_commit();
        }
        const int c = threadIdx.x % COLS, j = threadIdx.x / COLS;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            cp_async_wait_pending(NR - 1 - r);
            __syncthreads();
            if (r == 0 && rank == 0) {
                for (int ky = threadIdx.x; ky < M; ky += blockDim.x) {
                    cf a = pb[ky * PP], u = nyq[ky];
                    pb[ky * PP] = cmake(a.x - u.y, a.y + u.x);   // + i * Z[ky][M/2]
                }
                __syncthreads();
            }
            const int pl = r * COLS + c;       // local packed column
            const bool act = pl < PC;
            cf v[E];
#pragma unroll
            for (int s = 0; s < E; ++s) v[s] = act ? pb[in_index<M, V>(j, s) * PP + pl] : cmake(0.f, 0.f);
            fft_column<M, true, 1, V>(v, j, stg, c, COLS, tw);
            if (act) {
#pragma unroll
                for (int s = 0; s < E; ++s) pb[out_index<M, V>(j, s) * PP + pl] = v[s];
            }
            __syncthreads();
        }
    }
    // my rows [rank M/CL, (rank+1) M/CL); with a cluster, the peer's columns of
    // those rows are copied once (coalesced) into stg, and after a second
    // barrier the half of pb the peer read is free for the C2R exchange
    const int rows = M / CL, row0 = rank * rows;
    cf *xb2 = stg;
    if constexpr (CL > 1) {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        const cf *peer = cl.map_shared_rank(pb, rank ^ 1);
        // the peer's rows [row0, row0 + rows) are one contiguous, 16-byte
        // aligned block of its pb (padding included): copy it verbatim into
        // stg with 16-byte loads, every thread's loads in flight at once
        constexpr int NV = (M / CL) * PP * (int)sizeof(cf) / 16;
        constexpr int PER = (NV + C::NT - 1) / C::NT;
        static_assert((M / CL) * PP * sizeof(cf) % 16 == 0 && (M * PP * sizeof(cf)) % 16 == 0, "16-byte copy");
        const float4 *src4 = reinterpret_cast<const float4 *>(peer + row0 * PP);
        float4 *dst4 = reinterpret_cast<float4 *>(stg);
        float4 tmp[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int v = threadIdx.x + k * C::NT;
            if (v < NV) tmp[k] = src4[v];
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int v = threadIdx.x + k * C::NT;
            if (v < NV) dst4[v] = tmp[k];
        }
        cl.sync();
        xb2 = pb + (rank ^ 1) * rows * PP;
    } else {
        __syncthreads();
    }
    // phase 2: C2R along x of my rows by a half-length complex inverse FFT
    {
        constexpr int EH = Plan<H, VH>::E, RPR = C::RPR;
        const int rowl = threadIdx.x % RPR, j = threadIdx.x / RPR;
        float best = -INFINITY;
        uint32_t bidx = 0xFFFFFFFFu;
        for (int r0 = 0; r0 < rows; r0 += RPR) {
            int yl = r0 + rowl;
            int y = row0 + yl;
            bool act = yl < rows;
            cf v[EH];
#pragma unroll
            for (int s = 0; s < EH; ++s) {
                int k = in_index<H, VH>(j, s);
                cf Ek = cmake(0.f, 0.f), Ok = cmake(0.f, 0.f);
                if (act) {
                    // W[k] and W[H - k]; column 0 holds W[0] + i W[H]
                    cf Wk, Wm;
                    auto fetch = [&](int col) -> cf {
                        int own = col / PC, l = col % PC;
                        if (CL == 1 || own == rank) return pb[y * PP + l];
                        return stg[yl * PP + l];
                    };
                    if (k == 0) {
                        cf p = fetch(0);
                        Wk = cmake(p.x, 0.f);
                        Wm = cmake(p.y, 0.f);
                    } else {
                        Wk = fetch(k);
                        Wm = fetch(H - k);
                    }
                    cf wc = cconj(Wm);
                    Ek = cadd(Wk, wc);
                    Ok = cmul(csub(Wk, wc), cconj(tw[k]));   // exp(+2 pi i k / M)
                }
                v[s] = cmake(Ek.x - Ok.y, Ek.y + Ok.x);   // E + i O
            }
            fft_column<H, true, 2, VH>(v, j, xb2, rowl, RPR, tw);
            if (act) {
                const uint32_t rowbase = ((uint32_t)zc * M + (uint32_t)y) * M;
                if (EXPORT) {
#pragma unroll
                    for (int s = 0; s < EH; ++s) {
                        const uint32_t base = rowbase + 2u * out_index<H, VH>(j, s);
                        Cout[base] = v[s].x;
                        Cout[base + 1] = v[s].y;
                    }
                }
                // the thread's maximum first; the canvas index (lowest among
                // equal values) only for the values that reach it
                float m = v[0].x;
#pragma unroll
                for (int s = 0; s < EH; ++s) m = fmaxf(m, fmaxf(v[s].x, v[s].y));
                if (m >= best) {
                    uint32_t bi = 0xFFFFFFFFu;
#pragma unroll
                    for (int s = 0; s < EH; ++s) {
                        if (v[s].x == m || v[s].y == m) {
                            const uint32_t base = rowbase + 2u * out_index<H, VH>(j, s);
                            if (v[s].x == m) bi = min(bi, base);
                            if (v[s].y == m) bi = min(bi, base + 1u);
                        }
                    }
                    if (m > best || bi < bidx) { best = m; bidx = bi; }
                }
            }
            __syncthreads();
        }
        if (!EXPORT) {
            unsigned long long kk = (bidx == 0xFFFFFFFFu) ? 0ull : pack_key(best, bidx);
            for (int o = 16; o > 0; o >>= 1) {
                unsigned long long k2 = __shfl_down_sync(0xFFFFFFFFu, kk, o);
                kk = k2 > kk ? k2 : kk;
            }
            __shared__ unsigned long long wk[32];
            int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            if (lane == 0) wk[warp] = kk;
            __syncthreads();
            if (warp == 0) {
                kk = (lane < (int)(blockDim.x >> 5)) ? wk[lane] : 0ull;
                for (int o = 16; o > 0; o >>= 1) {
                    unsigned long long k2 = __shfl_down_sync(0xFFFFFFFFu, kk, o);
                    kk = k2 > kk ? k2 : kk;
                }
                if (lane == 0 && kk) atomicMax(key, kk);
            }
        }
    }
}

template <int M, int V = 0>
__global__ void __launch_bounds__(PlaneCfg<M, V>::NT)
k_plane(int B, const float2 *Z, const float2 *tw_g, const RotRec *rots, const ReqDev *reqs, int ahead)
{
    using C = PlaneCfg<M, V>;
    extern __shared__ __align__(16) unsigned char smem[];
    cf *pb = reinterpret_cast<cf *>(smem);    // [M][PP]
    cf *stg = pb + M * C::PP;                 // [STG]
    cf *tw = stg + C::STG;                    // [M]
    const int zc = blockIdx.x / C::CL, b = blockIdx.y;
    int rank = 0;
    if constexpr (C::CL > 1) rank = (int)cg::this_cluster().block_rank();
    const size_t plane = (size_t)M * (M / 2 + 2);
    const float2 *Zp = Z + ((size_t)b * M + zc) * plane;
    // One CTA fits an SM, so its column loads cannot overlap another CTA's
    // compute.  Ask L2 for the same half of the plane `ahead` planes on (the
    // one the CTA that next runs on this SM is likely to take): every line
    // of each row's half (kx in [rank PC, rank PC + PC), plus the Nyquist
    // column for rank 0), all addresses inside that row.
    const size_t nxt = (size_t)b * M + zc + (size_t)ahead;
    if (ahead > 0 && nxt < (size_t)B * M) {
        constexpr int HB = C::PC * (int)sizeof(float2);   // bytes of a half row
        constexpr int NL = (HB + 127) / 128 + 1;           // prefetches per half row (the last at its end)
        const char *rows = reinterpret_cast<const char *>(Z + nxt * plane);
        for (int i = threadIdx.x; i < M * (NL + 1); i += blockDim.x) {
            const int ky = i / (NL + 1), k = i % (NL + 1);
            const char *row = rows + (size_t)ky * (M / 2 + 2) * sizeof(float2);
            int off;
            if (k < NL - 1) off = rank * HB + 128 * k;
            else if (k == NL - 1) off = rank * HB + HB - 1;
            else off = (M / 2) * (int)sizeof(float2);   // the Nyquist column
            if (k == NL && rank != 0) continue;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(row + off));
        }
    }
    plane_body<M, false, V>(Zp, tw_g, &reqs[rots[b].req].keys[rots[b].rot], nullptr, zc, pb, stg, tw, rank);
}

template <int M, int V = 0>
__global__ void __launch_bounds__(PlaneCfg<M, V>::NT)
k_plane_export(const float2 *Z, const float2 *tw_g, float *C)
{
    using Cf = PlaneCfg<M, V>;
    extern __shared__ __align__(16) unsigned char smem[];
    cf *pb = reinterpret_cast<cf *>(smem);
    cf *stg = pb + M * Cf::PP;
    cf *tw = stg + Cf::STG;
    const int zc = blockIdx.x / Cf::CL;
    int rank = 0;
    if constexpr (Cf::CL > 1) rank = (int)cg::this_cluster().block_rank();
    const size_t plane = (size_t)M * (M / 2 + 2);
    plane_body<M, true, V>(Z + (size_t)zc * plane, tw_g, nullptr, C, zc, pb, stg, tw, rank);
}

template <int M, int V = 0>
static size_t plane_smem() { return PlaneCfg<M, V>::SMEM; }

template <int M, bool EXPORT, int V = 0>
static cudaError_t launch_plane_t(int B, const float2 *Z, const float2 *tw, const RotRec *rots,
                                  const ReqDev *reqs, float *C, cudaStream_t st)
{
    constexpr int CL = PlaneCfg<M, V>::CL;
    size_t sm = plane_smem<M, V>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(M * CL, EXPORT ? 1 : B);
    cfg.blockDim = dim3(PlaneCfg<M, V>::NT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (EXPORT) {
        e = cudaFuncSetAttribute(k_plane_export<M, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        e = cudaLaunchKernelEx(&cfg, k_plane_export<M, V>, Z, tw, C);
    } else {
        e = cudaFuncSetAttribute(k_plane<M, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        // planes in flight at one CTA per SM: the next CTA on an SM takes
        // roughly the plane this many further on
        int dev = 0, sms = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        e = cudaLaunchKernelEx(&cfg, k_plane<M, V>, B, Z, tw, rots, reqs, sms / CL);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_plane(const Geo &g, int B, const float2 *Z, const float2 *tw, const RotRec *rots,
                         const ReqDev *reqs, cudaStream_t st, int plane_cl, int *err, int plane_tma, int fft_plan)
{
    if (plane_tma && plane_ps_supported(g.M, plane_cl)) {
        const cudaError_t e = launch_plane_ps(g, plane_cl, B, Z, rots, reqs, err, st);
        if (!plane_ps_unavailable(e)) return e;
    }
    if (plane_cl_supported(g.M, plane_cl)) return launch_plane_cl(g, plane_cl, B, Z, tw, rots, reqs, err, st);
    switch (g.M) {
    case 64:
        return fft_plan == 1 ? launch_plane_t<64, false, 1>(B, Z, tw, rots, reqs, nullptr, st)
                             : launch_plane_t<64, false>(B, Z, tw, rots, reqs, nullptr, st);
    case 128:
        return fft_plan == 1 ? launch_plane_t<128, false, 1>(B, Z, tw, rots, reqs, nullptr, st)
                             : launch_plane_t<128, false>(B, Z, tw, rots, reqs, nullptr, st);
    case 192: return launch_plane_t<192, false>(B, Z, tw, rots, reqs, nullptr, st);
    case 256: return launch_plane_t<256, false>(B, Z, tw, rots, reqs, nullptr, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_plane_export(const Geo &g, const float2 *Z, const float2 *tw, float *C, cudaStream_t st,
                                int plane_cl, int *err, int plane_tma, int fft_plan)
{
    if (plane_tma && plane_ps_supported(g.M, plane_cl)) {
        const cudaError_t e = launch_plane_ps_export(g, plane_cl, Z, C, err, st);
        if (!plane_ps_unavailable(e)) return e;
    }
    if (plane_cl_supported(g.M, plane_cl)) return launch_plane_cl_export(g, plane_cl, Z, tw, C, err, st);
    switch (g.M) {
    case 64:
        return fft_plan == 1 ? launch_plane_t<64, true, 1>(1, Z, tw, nullptr, nullptr, C, st)
                             : launch_plane_t<64, true>(1, Z, tw, nullptr, nullptr, C, st);
    case 128:
        return fft_plan == 1 ? launch_plane_t<128, true, 1>(1, Z, tw, nullptr, nullptr, C, st)
                             : launch_plane_t<128, true>(1, Z, tw, nullptr, nullptr, C, st);
    case 192: return launch_plane_t<192, true>(1, Z, tw, nullptr, nullptr, C, st);
    case 256: return launch_plane_t<256, true>(1, Z, tw, nullptr, nullptr, C, st);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// K9: top-K over rotations, score descending then rotation ascending, and the
// candidate poses T = (R, R (h dk + o_s - o_o)) (Eq. (8)).
// ---------------------------------------------------------------------------
__global__ void k_topk(const unsigned long long *keys, int n, int K, int N, int M, double h, const double *o_o,
                       const double *quats, const RotRec *rots_all, dock_candidate *out, const double *o_s)
{
    __shared__ unsigned long long red[32];
    __shared__ unsigned long long prev;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) prev = ~0ull;
    __syncthreads();
    for (int k = 0; k < K; ++k) {
        // composite key: high 32 bits = ordered score, low 32 = ~rotation;
        // unique per rotation, so the k-th best is the largest below the (k-1)-th
        const unsigned long long lim = prev;
        unsigned long long best = 0ull;
        for (int i = tid; i < n; i += blockDim.x) {
            unsigned long long key = keys[i];
            if (!key) continue;
            unsigned long long c = (key & 0xFFFFFFFF00000000ull) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)i);
            if (c < lim && c > best) best = c;
        }
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long b2 = __shfl_down_sync(0xFFFFFFFFu, best, o);
            best = b2 > best ? b2 : best;
        }
        if (lane == 0) red[warp] = best;
        __syncthreads();
        if (warp == 0) {
            best = lane < nw ? red[lane] : 0ull;
            for (int o = 16; o > 0; o >>= 1) {
                unsigned long long b2 = __shfl_down_sync(0xFFFFFFFFu, best, o);
                best = b2 > best ? b2 : best;
            }
            if (lane == 0) {
                prev = best ? best : 0ull;
                int rot = best ? (int)(0xFFFFFFFFu - (uint32_t)(best & 0xFFFFFFFFull)) : -1;
                dock_candidate cd;
                if (rot >= 0) {
                    unsigned long long key = keys[rot];
                    uint32_t sk = (uint32_t)(key >> 32);
                    uint32_t u = (sk & 0x80000000u) ? (sk & 0x7FFFFFFFu) : ~sk;
                    cd.score = __uint_as_float(u);
                    uint32_t idx = 0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull);
                    cd.canvas_idx = (int32_t)idx;
                    int cz = idx / (M * M), cy = (idx / M) % M, cx = idx % M;
                    cd.dk[0] = cx <= N - 1 ? cx : cx - M;
                    cd.dk[1] = cy <= N - 1 ? cy : cy - M;
                    cd.dk[2] = cz <= N - 1 ? cz : cz - M;
                    cd.rot = rot;
                    for (int a = 0; a < 4; ++a) cd.q[a] = quats[4 * rot + a];
                    const RotRec &rr = rots_all[rot];
                    if (o_s) {
                        // rotated object: T = (R, h dk + o_s - o_R)
                        for (int a = 0; a < 3; ++a) cd.t[a] = ds(da(dm(h, (double)cd.dk[a]), o_s[a]), rr.o[a]);
                    } else {
                        double v[3];
                        for (int a = 0; a < 3; ++a) v[a] = ds(da(dm(h, (double)cd.dk[a]), rr.o[a]), o_o[a]);
                        for (int a = 0; a < 3; ++a)
                            cd.t[a] = da(da(dm(rr.R[3 * a], v[0]), dm(rr.R[3 * a + 1], v[1])), dm(rr.R[3 * a + 2], v[2]));
                    }
                } else {
                    cd.score = -INFINITY;
                    cd.canvas_idx = -1;
                    cd.rot = -1;
                    for (int a = 0; a < 3; ++a) { cd.dk[a] = 0; cd.t[a] = 0.0; }
                    for (int a = 0; a < 4; ++a) cd.q[a] = 0.0;
                }
                out[k] = cd;
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_topk(const unsigned long long *keys, int n, int K, int N, int M, double h, const double *o_o,
                        const double *quats, const RotRec *rots_all, dock_candidate *out, cudaStream_t st,
                        const double *o_s)
{
    if (K > 1024) return cudaErrorInvalidValue;
    k_topk<<<1, 1024, 0, st>>>(keys, n, K, N, M, h, o_o, quats, rots_all, out, o_s);
    return cudaGetLastError();
}

}  // namespace dock
