// Search passes at canvas side M = 256 (Eq. (7), (9)), the lattice side of
// the 128^3 workload:
//   k_fwd2d_runs     forward x and y transforms of binary slabs from their run
//                    lists (the default forward pass)
//   k_zpass16        z pass with the spectrum multiply, 16 columns per block
//   k_zpass16_dual   the same for the label-aware score (two sweeps, two spectra)
//   k_zpass_tc       the z pass with its DFT stages on the tensor cores
//   k_plane_cl       inverse plane pass with the argmax, one cluster per plane
//   k_plane_ps       the same as persistent clusters with TMA-loaded columns
//                    (the default plane pass)
//
// Plane pass, over a cluster of CL = 4 or 8 CTAs per plane (the last two
// inverse transforms of C = F^-1(conj(F(O)) . F(S)) and the per-rotation
// argmax).
//
// Plane z of rotation b holds Z[ky][kx], ky < 256, kx <= 128 (row pitch 130).
// CTA `rank` of the cluster owns the packed columns kx in [rank CPC,
// (rank + 1) CPC) (CPC = 128 / CL; packed column 0 carries kx = 0 plus i
// times the Nyquist column kx = 128):
//   phase 1  loads its columns straight from global memory into registers
//            (half-warp lanes on 16 consecutive kx: 128-byte rows) and
//            inverse transforms them along y (radix 16 x 16, the exchange
//            between the two stages in place in shared memory);
//   push     the rows of its columns that another CTA needs are one
//            contiguous block per destination, copied into that CTA's
//            shared memory by the bulk-copy engine (cp.async.bulk, completion
//            counted in bytes on the receiver's mbarrier);
//   phase 2  C2R along x of its RPC = 256 / CL rows (half-length complex
//            inverse FFT, radix 16 x 8, exchange in place) and the argmax
//            with the lowest canvas index on ties.
// Shared memory (complex elements): A [CL][CPC][RPC] holds phase 2's rows of
// every source CTA at kx RPC (A[rank] is also phase 1's block of its own
// rows), X [CL - 1][CPC][RPC] phase 1's blocks for the other CTAs.  Element
// (local column c, row y) sits at offset (y mod RPC) ^ (c mod 16) of its
// column in the block: half-warps that touch 16 columns at one row and warps
// that touch 32 rows of one column both hit distinct banks, and most
// addresses are a per-thread base plus a constant.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "dock_internal.h"
#include "fft.cuh"
#include "peak_key.cuh"

namespace cg = cooperative_groups;

namespace dock {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *m, uint32_t bytes)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(m)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// shared::cluster address of the same shared-memory offset in CTA `rank`
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void bulk_push(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst),
                 "r"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// exp(-2 pi i m / 256), FP64 values rounded to FP32, in the constant bank
// (per-thread twiddles are read once, through the constant cache, and kept in
// registers; set per device before the first launch)
__constant__ float2 c_tw256[256];

// exp(+2 pi i m / 256)
__device__ __forceinline__ cf twc_inv(int m)
{
    const float2 w = c_tw256[m & 255];
    return cmake(w.x, -w.y);
}

}  // namespace

template <int CL> struct PlaneClCfg {
    static constexpr int M = 256, H = 128, P = H + 2;
    static constexpr int NT = 256;                 // threads per CTA
    static constexpr int CPC = H / CL;             // packed columns per CTA
    static constexpr int RPC = M / CL;             // rows per CTA in phase 2
    static constexpr int LR = RPC == 64 ? 6 : 5;   // log2 RPC
    static constexpr int BLK = CPC * RPC;          // elements of one (row block, column block)
    static constexpr int MINB = CL == 4 ? 2 : 3;   // resident CTAs per SM
    static constexpr size_t A_OFF = 0;
    static constexpr size_t X_OFF = (size_t)CL * BLK * 8;
    static constexpr uint32_t PUSH_BYTES = (uint32_t)BLK * 8;
    static constexpr uint32_t RECV_BYTES = (uint32_t)(CL - 1) * BLK * 8;
    static constexpr size_t MB_OFF = X_OFF + (size_t)(CL - 1) * BLK * 8;
    static constexpr size_t SMEM = MB_OFF + 16 + 8 * (NT / 32);
    static_assert(CPC % 16 == 0 && RPC % 32 == 0 && (1 << LR) == RPC, "tile shape");
    static_assert((SMEM + 1024) * MINB <= 228 * 1024, "resident CTAs per SM");
    static_assert(PUSH_BYTES % 16 == 0 && X_OFF % 16 == 0, "bulk copies move 16-byte multiples");
};

// Upper bound on the wait for the peers' blocks (clock cycles, about a second).
constexpr long long PLANE_WAIT_CYCLES = 1ll << 31;

template <int CL, bool EXPORT>
__global__ void __launch_bounds__(PlaneClCfg<CL>::NT, PlaneClCfg<CL>::MINB)
k_plane_cl(const float2 *__restrict__ Z, const float2 *__restrict__ tw, const RotRec *rots, const ReqDev *reqs,
           float *Cout, int *err, int withhold)
{
    using C = PlaneClCfg<CL>;
    constexpr int M = C::M, H = C::H, P = C::P, CPC = C::CPC, RPC = C::RPC, LR = C::LR, BLK = C::BLK;
    extern __shared__ __align__(128) unsigned char smem[];
    cf *A = reinterpret_cast<cf *>(smem + C::A_OFF);
    cf *X = reinterpret_cast<cf *>(smem + C::X_OFF);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + C::MB_OFF);
    unsigned long long *wk = reinterpret_cast<unsigned long long *>(smem + C::MB_OFF + 16);
    const int tid = threadIdx.x;
    const int rank = (int)cg::this_cluster().block_rank();
    const int zc = blockIdx.x / CL, b = blockIdx.y;
    const float2 *Zp = Z + ((size_t)b * M + zc) * ((size_t)M * P);
    if (tid == 0) {
        mbar_init(mbar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(mbar, C::RECV_BYTES);
    }
    // element offset of phase-1 row block q (rows [q RPC, (q + 1) RPC)) of my columns
    auto blk = [&](int q) -> int { return q == rank ? rank * BLK : (CL + (q < rank ? q : q - 1)) * BLK; };

    // ---- phase 1: inverse FFT along y of my packed columns ----------------
    // both rounds of 16 columns at once (NR = CPC / 16): every load of the
    // CTA in flight together, one barrier for the stage exchange
    {
        constexpr int NR = CPC / 16;
        const int c = tid & 15, j = tid >> 4;
        int boff[CL];   // indexed by compile-time row blocks only
#pragma unroll
        for (int q = 0; q < CL; ++q) boff[q] = blk(q);
        cf v[NR][16];
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
            // ky = j + 16 s of packed column rank CPC + 16 rr + c
            const int kx = rank * CPC + rr * 16 + c;
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const float2 a = __ldcs(&Zp[(j + 16 * s) * P + kx]);
                v[rr][s] = cmake(a.x, a.y);
            }
            if (kx == 0) {   // + i * Z[ky][M/2]
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const float2 u = __ldcs(&Zp[(j + 16 * s) * P + H]);
                    v[rr][s] = cmake(v[rr][s].x - u.y, v[rr][s].y + u.x);
                }
            }
        }
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
            // stage 0: DFT over ky = j + 16 s; output r is index 16 j + r
            const int col = rr * 16 + c;
            DFT<16, true>::run(v[rr]);
            cf *bq = A + blk((16 * j) >> LR) + col * RPC + ((16 * j) & (RPC - 1));
#pragma unroll
            for (int r = 0; r < 16; ++r) bq[r ^ c] = v[rr][r];
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
            // stage 1: inputs j + 16 r, twiddles exp(+2 pi i j r / 256), DFT;
            // output r is row y = j + 16 r, stored where it was read
            const int col = rr * 16 + c;
            cf *b1 = A + col * RPC + (j ^ c);
            auto at1 = [&](int r) -> cf * { return b1 + boff[(16 * r) >> LR] + ((16 * r) & (RPC - 1)); };
            cf w[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) w[r] = *at1(r);
#pragma unroll
            for (int r = 1; r < 16; ++r) w[r] = cmul(w[r], twc_inv(j * r));
            DFT<16, true>::run(w);
#pragma unroll
            for (int r = 0; r < 16; ++r) *at1(r) = w[r];
        }
    }
    // ---- push: X[q] -> CTA q's A[rank] -------------------------------------
    fence_proxy_async();
    cg::this_cluster().sync();
    // withhold (test hook of the failure path): no block is pushed, so every
    // CTA's bounded wait below runs out, reports DOCK_E_TIMEOUT and returns
    if (tid == 0 && !withhold) {
        const uint32_t mb = smem_u32(mbar);
        const uint32_t dst = smem_u32(A + (size_t)rank * BLK);
#pragma unroll 1
        for (int q = 0; q < CL; ++q) {
            if (q == rank) continue;
            bulk_push(cluster_addr(dst, (uint32_t)q), smem_u32(X + (size_t)(q < rank ? q : q - 1) * BLK),
                      C::PUSH_BYTES, cluster_addr(mb, (uint32_t)q));
        }
        bulk_commit();
    }
    bool ok = true;
    {
        const long long t0 = clock64();
        while (!mbar_try_wait(mbar, 0)) {
            if (clock64() - t0 > PLANE_WAIT_CYCLES) {
                ok = false;
                break;
            }
        }
    }
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            if (err) atomicExch(err, DOCK_E_TIMEOUT);
            bulk_wait_read();
        }
        return;
    }

    // ---- phase 2: C2R along x of my rows, argmax ---------------------------
    // element (kx, row y) of A: kx RPC + (y mod RPC) ^ (kx mod 16); both rounds
    // of 32 rows at once (NRR = RPC / 32), one barrier per exchange
    {
        constexpr int NRR = RPC / 32;
        const int rowl = tid & 31, j = tid >> 5;   // j is warp-uniform: the twiddle reads broadcast
        float best = -INFINITY;
        uint32_t bidx = 0xFFFFFFFFu;
        cf v[NRR][16];
#pragma unroll
        for (int rr = 0; rr < NRR; ++rr) {
            const int ylo = (rank * RPC + rr * 32 + rowl) & (RPC - 1);
            // k = j + 8 s has k mod 16 = j + 8 (s mod 2); H - k has
            // (16 - j - 8 (s mod 2)) mod 16
            const cf *pk[2] = {A + j * RPC + (ylo ^ j), A + j * RPC + (ylo ^ (j + 8))};
            const cf *pm[2] = {A + (H - j) * RPC + (ylo ^ ((16 - j) & 15)), A + (H - j) * RPC + (ylo ^ ((8 - j) & 15))};
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                cf Wk, Wm;
                if (s == 0 && j == 0) {   // column 0 holds W[0] + i W[H]
                    const cf p = A[ylo];
                    Wk = cmake(p.x, 0.f);
                    Wm = cmake(p.y, 0.f);
                } else {
                    Wk = pk[s & 1][8 * s * RPC];
                    Wm = pm[s & 1][-8 * s * RPC];
                }
                const cf wc = cconj(Wm);
                const cf Ek = cadd(Wk, wc);
                const cf Ok = cmul(csub(Wk, wc), twc_inv(j + 8 * s));   // exp(+2 pi i k / M)
                v[rr][s] = cmake(Ek.x - Ok.y, Ek.y + Ok.x);             // E + i O
            }
        }
        __syncthreads();   // every W of these rows is in registers
#pragma unroll
        for (int rr = 0; rr < NRR; ++rr) {
            // stage 0 (radix 16 over k = j + 8 s): output r to index 16 j + r
            const int ylo = (rank * RPC + rr * 32 + rowl) & (RPC - 1);
            DFT<16, true>::run(v[rr]);
            cf *b0 = A + 16 * j * RPC;
#pragma unroll
            for (int r = 0; r < 16; ++r) b0[r * RPC + (ylo ^ r)] = v[rr][r];
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < NRR; ++rr) {
            const int y = rank * RPC + rr * 32 + rowl;
            const int ylo = y & (RPC - 1);
            // stage 1 (radix 8): butterfly jj = j + 8 bb reads jj + 16 r,
            // twiddles exp(+2 pi i 2 jj r / 256); output r is pair n = jj + 16 r
            cf w[16];
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
                const int jj = j + 8 * bb;
                const cf *b1 = A + jj * RPC + (ylo ^ jj);
#pragma unroll
                for (int r = 0; r < 8; ++r) w[bb * 8 + r] = b1[16 * r * RPC];
#pragma unroll
                for (int r = 1; r < 8; ++r) w[bb * 8 + r] = cmul(w[bb * 8 + r], twc_inv(2 * jj * r));
                DFT<8, true>::run(w + bb * 8);
            }
            const uint32_t rowbase = ((uint32_t)zc * M + (uint32_t)y) * M;
            if (EXPORT) {
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const uint32_t base = rowbase + 2u * (uint32_t)(j + 8 * (s >> 3) + 16 * (s & 7));
                    Cout[base] = w[s].x;
                    Cout[base + 1] = w[s].y;
                }
            } else {
                float m = w[0].x;
#pragma unroll
                for (int s = 0; s < 16; ++s) m = fmaxf(m, fmaxf(w[s].x, w[s].y));
                if (m >= best) {
                    uint32_t bi = 0xFFFFFFFFu;
#pragma unroll
                    for (int s = 0; s < 16; ++s) {
                        const uint32_t base = rowbase + 2u * (uint32_t)(j + 8 * (s >> 3) + 16 * (s & 7));
                        if (w[s].x == m) bi = min(bi, base);
                        if (w[s].y == m) bi = min(bi, base + 1u);
                    }
                    if (m > best || bi < bidx) {
                        best = m;
                        bidx = bi;
                    }
                }
            }
        }
        if (!EXPORT) {
            unsigned long long kk = (bidx == 0xFFFFFFFFu) ? 0ull : pack_key(best, bidx);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long k2 = __shfl_down_sync(0xFFFFFFFFu, kk, o);
                kk = k2 > kk ? k2 : kk;
            }
            const int lane = tid & 31, warp = tid >> 5;
            if (lane == 0) wk[warp] = kk;
            __syncthreads();
            if (warp == 0) {
                kk = lane < C::NT / 32 ? wk[lane] : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long k2 = __shfl_down_sync(0xFFFFFFFFu, kk, o);
                    kk = k2 > kk ? k2 : kk;
                }
                if (lane == 0 && kk) atomicMax(&reqs[rots[b].req].keys[rots[b].rot], kk);
            }
        }
    }
    // the bulk copies out of X have read their source before the CTA exits
    if (tid == 0) bulk_wait_read();
}

// ---------------------------------------------------------------------------
// Persistent plane pass with TMA staging (canvas 256, clusters of CL = 4 or 8
// CTAs; one CTA of 512 threads per SM for CL = 4, three of 256 for CL = 8).
// The same transforms as k_plane_cl (CTA `rank` owns packed columns
// [CPC rank, CPC (rank + 1)) in phase 1 and rows [RPC rank, RPC (rank + 1))
// in phase 2, CPC = 128 / CL, RPC = 256 / CL), but each cluster walks the
// planes p = cluster + G i of the launch (G clusters), and the
// tensor-memory-access unit loads the next plane's columns from HBM into the
// staging buffer U (one 2-D box of 256 rows x CPC complex, plus the Nyquist
// column for rank 0) while phase 2 of the current plane runs:
//   phase 1  radix 16 x 16 inverse FFT along y, from U through V (idle until
//            the pushes) back into U; thread (c, j) (tid = CPC j + c) holds
//            column c at rows j + 16 s; the last stage writes row y's column
//            c at c ^ (y mod CPC), so that phase 2's warps (32 rows of one
//            column) hit distinct banks
//   push     U's row block q (RPC rows, contiguous) to CTA q's V[rank]
//            by the bulk-copy engine, completion counted in bytes on CTA q's
//            mbarrier (the own block included)
//   phase 2  C2R along x of rows [RPC rank, RPC (rank + 1)) from V, the
//            exchange in place in V, argmax with the lowest canvas index on
//            ties (a row whose maximum scores below the rotation's best key
//            so far, written by planes done before, skips the index search)
// Per plane one cluster barrier (after it every CTA has finished phase 1 of
// this plane and phase 2 of the previous one, so V may be overwritten) and
// four block barriers; the waits' failure checks ride on two of them, and the
// plane's peak key collects in shared memory and leaves after the next one.
// Every wait is bounded; a CTA that gave up tells its peers through their
// shared memory before the next cluster barrier and the whole cluster stops
// there.
// ---------------------------------------------------------------------------
template <int CL_> struct PlanePsCfg {
    static constexpr int M = 256, H = 128, P = 130, CL = CL_, CPC = H / CL, RPC = M / CL;
    static constexpr int NT = 8 * RPC;                             // phase 2: 8 threads per row
    static constexpr int MINB = CL == 4 ? 1 : 3;                   // resident CTAs per SM
    static constexpr int BLK = RPC * CPC;                          // complex elements of one row block
    static constexpr uint32_t BOX_BYTES = M * CPC * 8;             // all rows of my packed columns
    static constexpr uint32_t NYQ_BYTES = M * 16;                  // all rows of kx = 128, 129
    static constexpr uint32_t BLK_BYTES = BLK * 8;
    static constexpr size_t U_OFF = 0, V_OFF = BOX_BYTES, N_OFF = V_OFF + (size_t)CL * BLK_BYTES;
    static constexpr size_t MB_OFF = N_OFF + NYQ_BYTES;            // two mbarriers, the stop flag, two plane keys
    static constexpr size_t SMEM = MB_OFF + 48;
    static constexpr long long WAIT_CYCLES = 1ll << 31;
    static_assert(MINB * (SMEM + 1024) <= 228 * 1024, "resident CTAs per SM");
    static_assert(NT == 16 * CPC && RPC % CPC == 0 && RPC % 32 == 0, "thread mappings of the two phases");
    static_assert(BLK_BYTES % 16 == 0 && V_OFF % 128 == 0 && N_OFF % 128 == 0, "bulk and tensor copy alignment");
};

namespace {
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t addr, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *m, uint32_t parity, long long cycles)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(m, parity))
        if (clock64() - t0 > cycles) return false;
    return true;
}
}  // namespace

template <int CL, bool EXPORT>
__global__ void __launch_bounds__(PlanePsCfg<CL>::NT, PlanePsCfg<CL>::MINB)
k_plane_ps(const __grid_constant__ CUtensorMap zmap, const __grid_constant__ CUtensorMap nmap, int n_planes,
           const RotRec *rots, const ReqDev *reqs, float *Cout, int *err, int withhold)
{
    using C = PlanePsCfg<CL>;
    constexpr int M = C::M, H = C::H, CPC = C::CPC, RPC = C::RPC, BLK = C::BLK;
    extern __shared__ __align__(128) unsigned char smem[];
    cf *U = reinterpret_cast<cf *>(smem + C::U_OFF);    // [M (y)][CPC]: my packed columns
    cf *V = reinterpret_cast<cf *>(smem + C::V_OFF);    // [CL (source)][RPC (y)][CPC]; then phase 2's exchange
    cf *Nq = reinterpret_cast<cf *>(smem + C::N_OFF);   // [M][2]: kx = 128, 129
    uint64_t *tma_bar = reinterpret_cast<uint64_t *>(smem + C::MB_OFF);
    uint64_t *v_bar = tma_bar + 1;
    int *s_stop = reinterpret_cast<int *>(smem + C::MB_OFF + 16);
    unsigned long long *s_key = reinterpret_cast<unsigned long long *>(smem + C::MB_OFF + 32);   // by plane parity
    const int tid = threadIdx.x;
    const int rank = (int)cg::this_cluster().block_rank();
    const int cid = blockIdx.x / C::CL, G = gridDim.x / C::CL;
    // the tensor copies want 128-byte aligned destinations (the layout is the
    // same in every CTA, so the whole cluster returns together)
    if (smem_u32(smem) & 127) {
        if (tid == 0 && err) atomicExch(err, DOCK_E_CUDA);
        return;
    }
    auto tma_issue = [&](int p) {
        mbar_arrive_expect_tx(tma_bar, C::BOX_BYTES + (rank == 0 ? C::NYQ_BYTES : 0u));
        tma_load_2d(smem_u32(U), &zmap, 2 * CPC * rank, p * M, smem_u32(tma_bar));
        if (rank == 0) tma_load_2d(smem_u32(Nq), &nmap, 2 * H, p * M, smem_u32(tma_bar));
    };
    int tma_out = -1, v_out = -1;   // (thread 0) parity of a copy in flight that no wait has seen complete
    if (tid == 0) {
        mbar_init(tma_bar, 1);
        mbar_init(v_bar, 1);
        *s_stop = 0;
        s_key[0] = s_key[1] = 0ull;
        fence_mbar_init();
        if (cid < n_planes) {
            tma_issue(cid);
            tma_out = 0;
        }
    }
    // the barriers and the stop flag are initialised before any peer touches them
    cg::this_cluster().sync();

    bool fail = false;   // block-uniform: a wait of this CTA ran out
    int key_b = -1;      // (thread 0) rotation whose plane key waits in s_key[key_par]
    uint32_t key_par = 0;
    // the previous plane's key (every warp has added to it before the barrier
    // that precedes this call) goes to its rotation's key array
    auto flush_key = [&]() {
        if (!EXPORT && tid == 0 && key_b >= 0) {
            const unsigned long long kk = s_key[key_par];
            if (kk) atomicMax(&reqs[rots[key_b].req].keys[rots[key_b].rot], kk);
            s_key[key_par] = 0ull;
            key_b = -1;
        }
    };
    int i = 0;
#pragma unroll 1
    for (int p = cid; p < n_planes; p += G, ++i) {
        const uint32_t par = (uint32_t)(i & 1);
        if (!fail) {
            if (tid == 0) mbar_arrive_expect_tx(v_bar, C::CL * C::BLK_BYTES);
            const bool tma_ok = mbar_wait_bounded(tma_bar, par, C::WAIT_CYCLES);
            // ---- phase 1: inverse FFT along y of my packed columns ----------
            // stage 0 from U into V (idle until the pushes of this plane),
            // stage 1 from V back into U
            const int c = tid % CPC, j = tid / CPC;
            cf v[16];
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = U[(j + 16 * s) * CPC + c];
            if (rank == 0 && c == 0) {   // packed column 0: + i Z[ky][H]
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const cf u = Nq[(j + 16 * s) * 2];
                    v[s] = cmake(v[s].x - u.y, v[s].y + u.x);
                }
            }
            // stage 0: DFT over ky = j + 16 s; output r is index 16 j + r
            DFT<16, true>::run(v);
            // after this barrier every warp has left the previous plane's
            // phase 2 (V is free, its warp keys are in) and read its U inputs
            if (__syncthreads_or(!tma_ok)) {
                fail = true;
                if (tid == 0 && err) atomicExch(err, DOCK_E_TIMEOUT);
            } else {
                if (tid == 0) tma_out = -1;
                flush_key();
#pragma unroll
                for (int r = 0; r < 16; ++r) V[(16 * j + r) * CPC + c] = v[r];
                __syncthreads();
                // stage 1: inputs j + 16 r, twiddles exp(+2 pi i j r / 256);
                // output r is row y = j + 16 r
#pragma unroll
                for (int r = 0; r < 16; ++r) v[r] = V[(j + 16 * r) * CPC + c];
#pragma unroll
                for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], twc_inv(j * r));
                DFT<16, true>::run(v);
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const int y = j + 16 * r;
                    U[y * CPC + (c ^ (y & (CPC - 1)))] = v[r];
                }
            }
        }
        fence_proxy_async();   // U is read next, and V written, by the bulk-copy engine
        if (fail && tid < C::CL) st_cluster_u32(cluster_addr(smem_u32(s_stop), (uint32_t)tid), 1u);
        cg::this_cluster().sync();
        if (*reinterpret_cast<volatile int *>(s_stop)) break;   // the same decision in every CTA of the cluster

        // ---- push: U's row block q -> CTA q's V[rank] -----------------------
        // withhold (test hook of the failure path): no block is pushed, every
        // CTA's bounded wait runs out and the clusters stop at their next barrier
        if (tid == 0 && !withhold) {
            const uint32_t dst = smem_u32(V + (size_t)rank * BLK), mb = smem_u32(v_bar);
#pragma unroll 1
            for (int q = 0; q < C::CL; ++q)
                bulk_push(cluster_addr(dst, (uint32_t)q), smem_u32(U + (size_t)q * BLK), C::BLK_BYTES,
                          cluster_addr(mb, (uint32_t)q));
            bulk_commit();
        }
        const bool v_ok = mbar_wait_bounded(v_bar, par, C::WAIT_CYCLES);
        if (tid == 0) {
            bulk_wait_read();   // U has been read by the pushes
            if (v_ok && p + G < n_planes) {   // the next plane loads during phase 2
                tma_issue(p + G);
                tma_out = (int)((i + 1) & 1);
            }
        }

        // ---- phase 2: C2R along x of my rows, argmax -------------------------
        const int rowl = tid & 31, j = (tid >> 5) & 7, rr = tid >> 8;   // j, rr warp-uniform
        const int ylo = rr * 32 + rowl, y = rank * RPC + ylo;
        const int b = p >> 8, zc = p & (M - 1);
        // the rotation's best key so far (from the planes done before; a stale
        // value is only lower): a row whose maximum scores below it cannot
        // hold the rotation's peak and skips the search for its index
        const uint32_t thr = EXPORT ? 0u : (uint32_t)(__ldcg(&reqs[rots[b].req].keys[rots[b].rot]) >> 32);
        // element (kx, local row ylo) of V: source kx / CPC, column
        // (kx mod CPC) ^ (y mod CPC) (RPC is a multiple of CPC)
        auto vat = [&](int kx) -> cf { return V[(kx / CPC) * BLK + ylo * CPC + ((kx % CPC) ^ (ylo & (CPC - 1)))]; };
        cf v[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            const int k = j + 8 * s;
            cf Wk, Wm;
            if (s == 0 && j == 0) {   // packed column 0 holds W[0] + i W[H]
                const cf q0 = vat(0);
                Wk = cmake(q0.x, 0.f);
                Wm = cmake(q0.y, 0.f);
            } else {
                Wk = vat(k);
                Wm = vat(H - k);
            }
            const cf wc = cconj(Wm);
            const cf Ek = cadd(Wk, wc);
            const cf Ok = cmul(csub(Wk, wc), twc_inv(k));   // exp(+2 pi i k / M)
            v[s] = cmake(Ek.x - Ok.y, Ek.y + Ok.x);           // E + i O
        }
        if (__syncthreads_or(!v_ok)) {   // (also: every V value of these rows is in registers)
            fail = true;                 // told to the peers at the next cluster barrier
            if (tid == 0) {
                v_out = (int)par;
                if (err) atomicExch(err, DOCK_E_TIMEOUT);
            }
            continue;   // no phase 2 on missing data
        }
        // stage 0 (radix 16 over k = j + 8 s): output r to index 16 j + r,
        // stored at [index][row ^ (index mod 16)] in V
        DFT<16, true>::run(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) V[(16 * j + r) * RPC + (ylo ^ r)] = v[r];
        __syncthreads();
        // stage 1 (radix 8): butterfly jj = j + 8 bb reads jj + 16 r,
        // twiddles exp(+2 pi i 2 jj r / 256); output r is pair n = jj + 16 r
        cf w[16];
#pragma unroll
        for (int bb = 0; bb < 2; ++bb) {
            const int jj = j + 8 * bb;
#pragma unroll
            for (int r = 0; r < 8; ++r) w[bb * 8 + r] = V[(jj + 16 * r) * RPC + (ylo ^ jj)];
#pragma unroll
            for (int r = 1; r < 8; ++r) w[bb * 8 + r] = cmul(w[bb * 8 + r], twc_inv(2 * jj * r));
            DFT<8, true>::run(w + bb * 8);
        }
        const uint32_t rowbase = ((uint32_t)zc * M + (uint32_t)y) * M;
        if constexpr (EXPORT) {
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const uint32_t base = rowbase + 2u * (uint32_t)(j + 8 * (s >> 3) + 16 * (s & 7));
                Cout[base] = w[s].x;
                Cout[base + 1] = w[s].y;
            }
        } else {
            float m = w[0].x;
#pragma unroll
            for (int s = 0; s < 16; ++s) m = fmaxf(m, fmaxf(w[s].x, w[s].y));
            uint32_t bi = 0xFFFFFFFFu;
            if ((uint32_t)(pack_key(m, 0u) >> 32) >= thr) {
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const uint32_t base = rowbase + 2u * (uint32_t)(j + 8 * (s >> 3) + 16 * (s & 7));
                    if (w[s].x == m) bi = min(bi, base);
                    if (w[s].y == m) bi = min(bi, base + 1u);
                }
            }
            unsigned long long kk = (bi == 0xFFFFFFFFu) ? 0ull : pack_key(m, bi);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long k2 = __shfl_down_sync(0xFFFFFFFFu, kk, o);
                kk = k2 > kk ? k2 : kk;
            }
            // the plane's key in shared memory; thread 0 sends it on after the
            // next barrier (the next plane's, or the one after the loop)
            if ((tid & 31) == 0 && kk) atomicMax(&s_key[par], kk);
            if (tid == 0) {
                key_b = b;
                key_par = par;
            }
        }
    }
    __syncthreads();
    if (!fail) flush_key();
    // copies this CTA stopped waiting for: wait (bounded) before its shared
    // memory is released
    if (tid == 0) {
        if (tma_out >= 0) mbar_wait_bounded(tma_bar, (uint32_t)tma_out, C::WAIT_CYCLES);
        if (v_out >= 0) mbar_wait_bounded(v_bar, (uint32_t)v_out, C::WAIT_CYCLES);
        bulk_wait_read();
    }
}

// ---------------------------------------------------------------------------
// Forward x and y transforms of a slab of binary S at canvas 256 from its run
// list (Eq. (9), the first two of the three 1-D passes; the bits path of
// k_fwd2d with a footprint that lets three blocks share an SM).
//
// Block (slab jz, rotation b), 256 threads.  Each row's runs of set bits
// [a, e) are extracted once into shared memory (at most 64 per row of 128).
// Then, for each round of 16 kx columns p0 .. p0 + 15:
//   x  X[y][c] = q(kx) sum over runs (w^(kx a) - w^(kx e)), kx = p0 + c,
//      q(kx) = 1 / (1 - w^kx), w = exp(-2 pi i / 256) (kx = 0: the count of
//      set bits, with the Nyquist column, sum of (-1)^x, packed as its
//      imaginary part); a half-warp per row, lane c on kx;
//   y  forward 256-point DFT of each column (rows >= 128 are zero padding):
//      radix 16 x 16, thread (c, j) holding rows j + 16 s, one exchange
//      through shared memory, outputs ky = j + 16 r written to Y[ky][kx]
//      (a warp writes two rows of 16 consecutive kx).
// Packed column 0 is unpacked into kx = 0 and kx = 128 at the end.
// ---------------------------------------------------------------------------
struct FwdRunsCfg {
    static constexpr int M = 256, N = 128, H = 128, P = 130, NW = N / 32, NT = 256, COLS = 16;
    static constexpr size_t BITS_OFF = 0, RUNS_OFF = BITS_OFF + (size_t)N * NW * 4;
    static constexpr size_t CNT_OFF = RUNS_OFF + (size_t)N * (N / 2) * 2;
    static constexpr size_t TW_OFF = CNT_OFF + (size_t)N * 4;
    static constexpr size_t X_OFF = TW_OFF + (size_t)M * 8;
    static constexpr size_t XB_OFF = X_OFF + (size_t)N * COLS * 8;
    static constexpr size_t C0_OFF = XB_OFF + (size_t)M * COLS * 8;
    static constexpr size_t SMEM = C0_OFF + (size_t)M * 8;
    static_assert(3 * (SMEM + 1024) <= 228 * 1024, "three blocks per SM");
};

__global__ void __launch_bounds__(FwdRunsCfg::NT, 3)
k_fwd2d_runs(const uint32_t *__restrict__ bits_g, const uint32_t *__restrict__ mask_g, float2 *Y,
             const float2 *__restrict__ q_g)
{
    using C = FwdRunsCfg;
    constexpr int M = C::M, N = C::N, H = C::H, P = C::P, NW = C::NW, COLS = C::COLS;
    extern __shared__ __align__(128) unsigned char smem[];
    uint32_t *bits = reinterpret_cast<uint32_t *>(smem + C::BITS_OFF);   // [N][NW]
    uchar2 *runs = reinterpret_cast<uchar2 *>(smem + C::RUNS_OFF);       // [N][N / 2]: (a, e - 1)
    int *cnt = reinterpret_cast<int *>(smem + C::CNT_OFF);              // [N]
    cf *tw = reinterpret_cast<cf *>(smem + C::TW_OFF);                  // [M]: w^m
    cf *X = reinterpret_cast<cf *>(smem + C::X_OFF);                    // [N][COLS]
    cf *xb = reinterpret_cast<cf *>(smem + C::XB_OFF);                  // [M][COLS]
    cf *c0 = reinterpret_cast<cf *>(smem + C::C0_OFF);                  // [M]: packed column 0 after y
    const int tid = threadIdx.x, jz = blockIdx.x, b = blockIdx.y;
    const uint32_t *bg = bits_g + ((size_t)b * N + jz) * N * NW;
    if (mask_g) {
        const uint32_t *mg = mask_g + ((size_t)b * N + jz) * N * NW;
        for (int i = tid; i < N * NW; i += C::NT) bits[i] = bg[i] & ~mg[i];
    } else {
        for (int i = tid; i < N * NW; i += C::NT) bits[i] = bg[i];
    }
    for (int m = tid; m < M; m += C::NT) {
        const float2 w = c_tw256[m];
        tw[m] = cmake(w.x, w.y);
    }
    __syncthreads();
    // the runs of row y (thread y): [a, e) with e - 1 stored (e <= 128)
    if (tid < N) {
        int n = 0, open = -1;
        uint32_t prevw = 0;
        for (int w = 0; w <= NW; ++w) {
            const uint32_t cur = w < NW ? bits[tid * NW + w] : 0u;
            const uint32_t prev = (cur << 1) | (prevw >> 31);
            uint32_t ev = (cur & ~prev) | (~cur & prev);   // rises and falls
            while (ev) {
                const int bp = __ffs(ev) - 1;
                ev &= ev - 1;
                const int x = 32 * w + bp;
                if ((cur >> bp) & 1u) {
                    open = x;
                } else {
                    runs[tid * (N / 2) + n] = make_uchar2((unsigned char)open, (unsigned char)(x - 1));
                    ++n;
                }
            }
            prevw = cur;
        }
        cnt[tid] = n;
    }
    __syncthreads();

    float2 *Yb = Y + ((size_t)b * N + jz) * (size_t)M * P;
    const int hw = tid >> 4, c = tid & 15, j = tid >> 4;   // hw: half-warp (x), j: row class (y)
#pragma unroll 1
    for (int p0 = 0; p0 < H; p0 += COLS) {
        // ---- x: half-warp hw on rows hw + 16 i, lane c on kx = p0 + c ----
        const int kx = p0 + c;
        const float2 qq = q_g[kx];
        const cf q = cmake(qq.x, qq.y);
#pragma unroll 1
        for (int y = hw; y < N; y += C::NT / 16) {
            const int n = cnt[y];
            const uchar2 *rr = runs + y * (N / 2);
            cf acc = cmake(0.f, 0.f);
            if (kx == 0) {
                float ones = 0.f, nyq = 0.f;
                for (int k = 0; k < n; ++k) {
                    const int a = rr[k].x, e = rr[k].y + 1, len = e - a;
                    ones += (float)len;
                    if (len & 1) nyq += (a & 1) ? -1.f : 1.f;
                }
                acc = cmake(ones, nyq);
            } else {
                for (int k = 0; k < n; ++k) {
                    const int a = rr[k].x, e = rr[k].y + 1;
                    acc = cadd(acc, cmul(csub(tw[(kx * a) & (M - 1)], tw[(kx * e) & (M - 1)]), q));
                }
            }
            X[y * COLS + c] = acc;
        }
        __syncthreads();   // X complete; the previous round's exchange reads are done
        // ---- y: forward DFT of column c; stage 0 over rows j + 16 s --------
        cf v[16];
#pragma unroll
        for (int s = 0; s < 8; ++s) v[s] = X[(j + 16 * s) * COLS + c];
#pragma unroll
        for (int s = 8; s < 16; ++s) v[s] = cmake(0.f, 0.f);   // rows >= N: zero padding
        DFT<16, false>::run(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) xb[(16 * j + r) * COLS + c] = v[r];
        __syncthreads();
        // stage 1: inputs j + 16 r, twiddles exp(-2 pi i j r / 256); output ky = j + 16 r
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = xb[(j + 16 * r) * COLS + c];
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], cconj(twc_inv(j * r)));
        DFT<16, false>::run(v);
        if (kx == 0) {
#pragma unroll
            for (int r = 0; r < 16; ++r) c0[j + 16 * r] = v[r];
        } else {
#pragma unroll
            for (int r = 0; r < 16; ++r) Yb[(size_t)(j + 16 * r) * P + kx] = make_float2(v[r].x, v[r].y);
        }
    }
    __syncthreads();
    // packed column 0 = Y0 + i YH (both the transforms of real columns)
    for (int ky = tid; ky < M; ky += C::NT) {
        const cf val = c0[ky], oc = cconj(c0[(M - ky) & (M - 1)]);
        const cf y0 = cscale(cadd(val, oc), 0.5f);
        const cf w = csub(val, oc);
        float2 *row = Yb + (size_t)ky * P;
        row[0] = make_float2(y0.x, y0.y);
        row[H] = make_float2(0.5f * w.y, -0.5f * w.x);
        row[H + 1] = make_float2(0.f, 0.f);
    }
}

// ---------------------------------------------------------------------------
// z pass at M = 256 over 16 columns per CTA (f = ky P + kx in [16 blockIdx.x,
// + 16)): for each of the block's `group` rotations, forward FFT along z of
// the N = 128 non-zero inputs, times conj(F(O)) / M^3 (for a rotated object:
// the tile conjugated, times F(S) / M^3), inverse FFT along z.  Thread (c, j)
// (c = column, j < 16) holds z (or kz) = j + 16 s: the inputs come straight
// from global memory (the next rotation's already in flight), the forward
// output is in the inverse's input order, and both transforms exchange
// between their radix-16 stages through one [256][16] buffer.  The block's
// spectrum tile [kz][16] sits in shared memory (reloaded when the request
// changes), the stage twiddles come from the constant bank.
// ---------------------------------------------------------------------------
struct Zpass16Cfg {
    static constexpr int M = 256, N = 128, P = 130, NT = 256, COLS = 16;
    static constexpr size_t SMEM = (size_t)2 * M * COLS * 8;   // exchange + spectrum tile
};

__global__ void __launch_bounds__(Zpass16Cfg::NT, 3)
k_zpass16(int B, int group, const float2 *__restrict__ Y, const RotRec *rots, const ReqDev *reqs, float2 *Z)
{
    using C = Zpass16Cfg;
    constexpr int M = C::M, N = C::N, P = C::P, COLS = C::COLS;
    extern __shared__ __align__(16) unsigned char smem[];
    cf *xb = reinterpret_cast<cf *>(smem);      // [M][COLS]
    cf *spt = xb + M * COLS;                     // [M (kz)][COLS]
    const int tid = threadIdx.x, c = tid & 15, j = tid >> 4;
    const size_t plane = (size_t)M * P;
    const int f0 = blockIdx.x * COLS;            // first column of the block
    const int b0 = blockIdx.y * group, nb = min(group, B - b0);
    if (nb <= 0) return;
    auto load = [&](int bi, cf *v) {
        const float2 *src = Y + (size_t)(b0 + bi) * N * plane + f0 + c;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const float2 a = __ldcs(&src[(size_t)(j + 16 * s) * plane]);
            v[s] = cmake(a.x, a.y);
        }
    };
    cf nx[8];
    load(0, nx);
    int sp_req = -1;
#pragma unroll 1
    for (int bi = 0; bi < nb; ++bi) {
        cf v[16];
#pragma unroll
        for (int s = 0; s < 8; ++s) v[s] = nx[s];
#pragma unroll
        for (int s = 8; s < 16; ++s) v[s] = cmake(0.f, 0.f);   // z >= N: zero padding
        if (bi + 1 < nb) load(bi + 1, nx);
        const int req = rots[b0 + bi].req;
        if (req != sp_req) {   // block-uniform
            __syncthreads();   // the previous tile is no longer read
            const float2 *spec = reqs[req].spec;
            // tiled spectrum: ((f / 32) M + kz) 32 + f mod 32
            const float2 *src = spec + (size_t)(f0 / 32) * M * 32 + (f0 & 31) + c;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const float2 a = __ldg(&src[(size_t)(j + 16 * r) * 32]);
                spt[(j + 16 * r) * COLS + c] = cmake(a.x, a.y);
            }
            sp_req = req;
        }
        const float cj = reqs[req].rotate_object ? -1.f : 1.f;
        // forward, stage 0 (inputs z = j + 16 s) -> index 16 j + r
        DFT<16, false>::run(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) xb[(16 * j + r) * COLS + c] = v[r];
        __syncthreads();
        // forward, stage 1 -> kz = j + 16 r; multiply
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = xb[(j + 16 * r) * COLS + c];
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], cconj(twc_inv(j * r)));   // exp(-2 pi i j r / 256)
        DFT<16, false>::run(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            cf a = v[r];
            a.y *= cj;
            v[r] = cmul(a, spt[(j + 16 * r) * COLS + c]);
        }
        __syncthreads();   // every thread has read its forward stage-1 inputs
        // inverse, stage 0 (inputs kz = j + 16 r) -> index 16 j + r
        DFT<16, true>::run(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) xb[(16 * j + r) * COLS + c] = v[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = xb[(j + 16 * r) * COLS + c];
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], twc_inv(j * r));
        DFT<16, true>::run(v);
        float2 *dst = Z + (size_t)(b0 + bi) * M * plane + f0 + c;
#pragma unroll
        for (int r = 0; r < 16; ++r) __stcs(&dst[(size_t)(j + 16 * r) * plane], make_float2(v[r].x, v[r].y));
        __syncthreads();   // the exchange buffer is free for the next rotation
    }
}

// ---------------------------------------------------------------------------
// z pass with its DFT stages on the tensor cores (tcgen05, kind::tf32).
//
// The same transforms as k_zpass16 -- along z, per column of a block of 16,
// the forward 256-point DFT of the zero-padded S column, the product with
// conj(F(O)), the inverse DFT -- as four radix-16 stages, each one dense
// product of the block's 256 vectors with the 16-point DFT matrix:
//   D[v][n] = sum_k A[v][k] W[k][n],
// row v of A holding one 16-point input vector as 32 reals (re, im
// interleaved) and W the real 32 x 32 form of the DFT matrix (forward or
// inverse).  Each stage is two products of M = 128 rows (N = 32, K = 8 per
// instruction) issued by one thread; A is read from tensor memory, W from
// shared memory, D accumulates in FP32 in tensor memory.  Thread v owns row
// v: lane v mod 128 of the columns of tile v / 128, where it writes its A row
// (tcgen05.st) and reads its D row (tcgen05.ld).
// 3 x TF32: each operand is split x = hi + lo, hi = x rounded to TF32 and
// lo = (x - hi) rounded to TF32 (the tensor cores would truncate it), and
// D = Ahi Whi + Ahi Wlo + Alo Whi; x - hi - lo and the dropped Alo Wlo term
// are below 2^-22 |x| |w|.
//
// Rows v = 16 j + c (thread v: column c, index j); z = z2 + 16 z1 on the
// way in, kz = k1 + 16 k2 in the spectrum, z = b + 16 a on the way out:
//   stage  row (j, c) holds          product over   thread v then
//   F0     z2 = j;  z1 < 8 (K = 16)  z1 -> k1       twiddles w^(z2 k1), sends k1 to row (k1, c)
//   F1     k1 = j;  z2               z2 -> k2       multiplies by the spectrum at kz, keeps its row
//   I0     k1 = j;  k2               k2 -> b        twiddles w^-(b k1), sends b to row (b, c)
//   I1     b = j;   k1               k1 -> a        stores z = b + 16 a
// (w = exp(-2 pi i / 256)).  The two transposes go through shared memory
// (X[row index][K index][c], c fastest: both directions conflict-free).
//
// Shared memory: W (forward hi, lo; inverse hi, lo) in the canonical
// K-major layout without swizzle (core matrices of 8 rows x 16 bytes:
// element (n, k) at byte (k / 4) 512 + (n / 8) 128 + (n mod 8) 16 +
// (k mod 4) 4), the exchange buffer and the spectrum tile [kz][16]: 80 KB.
// Tensor memory (256 columns): D at 32 t, A hi at 64 + 32 t, A lo at
// 128 + 32 t for tile t.  Two blocks per SM fill its 512 columns.
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
// tcgen05 shared-memory matrix descriptor: start, leading- and stride-
// dimension byte offsets (16-byte units), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// D (tensor memory) (+)= A (tensor memory) . B (shared memory descriptor)
__device__ __forceinline__ void umma_tf32_ta(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
                 "r"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *m)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(m))
                 : "memory");
}
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// this warp's 32 lanes, 32 consecutive columns of tensor memory from ta
__device__ __forceinline__ void tmem_ld32(uint32_t ta, float *f)
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(ta)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) f[i] = __uint_as_float(r[i]);
}
#define DOCK_R16(a, o)                                                                                           \
    "r"(a[o + 0]), "r"(a[o + 1]), "r"(a[o + 2]), "r"(a[o + 3]), "r"(a[o + 4]), "r"(a[o + 5]), "r"(a[o + 6]),     \
        "r"(a[o + 7]), "r"(a[o + 8]), "r"(a[o + 9]), "r"(a[o + 10]), "r"(a[o + 11]), "r"(a[o + 12]),             \
        "r"(a[o + 13]), "r"(a[o + 14]), "r"(a[o + 15])
// 16 or 32 consecutive columns of this warp's lanes from ta
__device__ __forceinline__ void tmem_st16(uint32_t ta, const uint32_t *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16};" ::"r"(ta),
                 DOCK_R16(v, 0)
                 : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t ta, const uint32_t *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(ta),
                 DOCK_R16(v, 0), DOCK_R16(v, 16)
                 : "memory");
}
#undef DOCK_R16
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// a thread's A row (K = 2 NV reals) split into TF32 hi and lo, into tensor memory
template <int NV> __device__ __forceinline__ void put_row(uint32_t ta_hi, uint32_t ta_lo, const cf *v)
{
    uint32_t h[2 * NV], l[2 * NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const float hx = tf32_rna(v[i].x), hy = tf32_rna(v[i].y);
        h[2 * i] = __float_as_uint(hx);
        h[2 * i + 1] = __float_as_uint(hy);
        l[2 * i] = __float_as_uint(tf32_rna(v[i].x - hx));
        l[2 * i + 1] = __float_as_uint(tf32_rna(v[i].y - hy));
    }
    if (NV == 8) {
        tmem_st16(ta_hi, h);
        tmem_st16(ta_lo, l);
    } else {
        tmem_st32(ta_hi, h);
        tmem_st32(ta_lo, l);
    }
    tmem_wait_st();
}

}  // namespace

struct ZpassTcCfg {
    static constexpr int M = 256, N = 128, P = 130, NT = 256, COLS = 16;
    static constexpr uint32_t LBO_W = 512, SBO = 128, W_BYTES = 4096;
    static constexpr size_t X_OFF = 4 * W_BYTES, SP_OFF = X_OFF + (size_t)M * COLS * 8;
    static constexpr size_t SMEM = SP_OFF + (size_t)M * COLS * 8;
    static constexpr uint32_t TMEM_COLS = 256;
    // D FP32, A and B TF32, both K-major, N = 32, M = 128
    static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
    static constexpr long long WAIT_CYCLES = 1ll << 31;
    // two blocks per SM (their tensor memory fills the SM's 512 columns), not three
    static_assert((SMEM + 64 + 1024) * 2 <= 228 * 1024 && (SMEM + 1024) * 3 > 228 * 1024, "two blocks per SM");
};

__global__ void __launch_bounds__(ZpassTcCfg::NT, 2)
k_zpass_tc(int B, int group, const float2 *__restrict__ Y, const RotRec *rots, const ReqDev *reqs, float2 *Z,
           int *err)
{
    using C = ZpassTcCfg;
    constexpr int M = C::M, N = C::N, P = C::P, COLS = C::COLS;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ int s_fail;
    unsigned char *W = smem;                                // forward hi, forward lo, inverse hi, inverse lo
    cf *xb = reinterpret_cast<cf *>(smem + C::X_OFF);      // [16 (row index)][16 (K index)][COLS]
    cf *spt = reinterpret_cast<cf *>(smem + C::SP_OFF);    // [M (kz)][COLS]
    const int tid = threadIdx.x, c = tid & 15, j = tid >> 4, warp = tid >> 5;
    const size_t plane = (size_t)M * P;
    const int f0 = blockIdx.x * COLS;
    const int b0 = blockIdx.y * group, nb = min(group, B - b0);
    if (nb <= 0) return;

    // the real forms of the forward and inverse 16-point DFT matrices:
    // output (re, im) of index kout from input (re, im) of index kin
    for (int i = tid; i < 2048; i += C::NT) {
        const int inv = i >> 10, n = (i >> 5) & 31, k = i & 31;
        const float2 w = c_tw256[(16 * (k >> 1) * (n >> 1)) & 255];   // exp(-2 pi i kin kout / 16)
        const float wr = w.x, wi = inv ? -w.y : w.y;
        const float x = (n & 1) == 0 ? ((k & 1) == 0 ? wr : -wi) : ((k & 1) == 0 ? wi : wr);
        const float hi = tf32_rna(x);
        const uint32_t off = (k >> 2) * C::LBO_W + (n >> 3) * C::SBO + (n & 7) * 16 + (k & 3) * 4;
        *reinterpret_cast<float *>(W + 2 * inv * C::W_BYTES + off) = hi;
        *reinterpret_cast<float *>(W + (2 * inv + 1) * C::W_BYTES + off) = tf32_rna(x - hi);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "r"(C::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&mbar, 1);
        fence_mbar_init();
        s_fail = 0;
    }
    fence_proxy_async();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16, tcol = (uint32_t)(32 * (warp >> 2));
    const uint32_t t_d = tmem + lanes + tcol, t_hi = tmem + lanes + 64 + tcol, t_lo = tmem + lanes + 128 + tcol;
    const uint32_t w_u32 = smem_u32(W);
    uint32_t phase = 0;
    int lost = -1;   // parity of a product this thread stopped waiting for

    // every thread has put its A row: one thread issues the stage's products
    // (nks K-steps of 8 against the W pair `mat`), all wait for them and read
    // their D rows; false when the block gave up
    // (the issue is unrolled with the descriptors as constant offsets from one
    // base: built in the loop, the issuing thread's arithmetic doubled a
    // stage's round trip)
    const uint64_t wdesc = umma_desc(w_u32, C::LBO_W, C::SBO);
    auto stage = [&](int nks, int mat, float *d) -> bool {
        tc_before_sync();
        __syncthreads();
        tc_after_sync();
        if (s_fail) return false;
        if (tid == 0) {
#pragma unroll
            for (int t = 0; t < 2; ++t)
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks)
                        if (ks < nks)
                            umma_tf32_ta(tmem + 32 * t, tmem + (p == 2 ? 128 : 64) + 32 * t + 8 * ks,
                                         wdesc + (((mat + (p == 1)) * C::W_BYTES + ks * 2 * C::LBO_W) >> 4), C::IDESC,
                                         (p | ks) != 0);
            umma_commit(&mbar);
        }
        // every thread polls (bounded): one waiter releasing the others through
        // a block barrier measured 5 % slower
        const long long t0 = clock64();
        bool ok = true;
        while (!mbar_try_wait(&mbar, phase))
            if (clock64() - t0 > C::WAIT_CYCLES) {
                ok = false;
                break;
            }
        if (!ok) {
            lost = (int)phase;
            s_fail = 1;
            if (err) atomicExch(err, DOCK_E_TIMEOUT);
        }
        phase ^= 1;
        tc_after_sync();
        tmem_ld32(t_d, d);
        return true;
    };

    auto load = [&](int bi, cf *v) {
        const float2 *src = Y + (size_t)(b0 + bi) * N * plane + f0 + c;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const float2 a = __ldcs(&src[(size_t)(j + 16 * s) * plane]);
            v[s] = cmake(a.x, a.y);
        }
    };
    cf nx[8];
    load(0, nx);
    int sp_req = -1;
#pragma unroll 1
    for (int bi = 0; bi < nb; ++bi) {
        float d[32];
        cf v[16];
        // F0 row: x[z2 + 16 z1], z1 < 8 (z >= N is zero padding, not read by the products)
        put_row<8>(t_hi, t_lo, nx);
        if (bi + 1 < nb) load(bi + 1, nx);
        const int req = rots[b0 + bi].req;
        if (req != sp_req) {   // block-uniform; the last reads of the old tile precede three barriers
            const float2 *src = reqs[req].spec + (size_t)(f0 / 32) * M * 32 + (f0 & 31) + c;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const float2 a = __ldg(&src[(size_t)(j + 16 * r) * 32]);
                spt[(j + 16 * r) * COLS + c] = cmake(a.x, a.y);
            }
            sp_req = req;
        }
        const float cj = reqs[req].rotate_object ? -1.f : 1.f;
        if (!stage(2, 0, d)) break;
        // F0 -> F1: k1 = r goes to row (k1, c), K index z2 = j
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            cf a = cmake(d[2 * r], d[2 * r + 1]);
            if (r) a = cmul(a, cconj(twc_inv(j * r)));   // exp(-2 pi i j r / 256)
            xb[(r * 16 + j) * COLS + c] = a;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = xb[(j * 16 + k) * COLS + c];
        put_row<16>(t_hi, t_lo, v);
        if (!stage(4, 0, d)) break;
        // F1 -> I0: X[kz = j + 16 r] conj(F(O))[kz], the same row
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            cf a = cmake(d[2 * r], d[2 * r + 1]);
            a.y *= cj;
            v[r] = cmul(a, spt[(j + 16 * r) * COLS + c]);
        }
        put_row<16>(t_hi, t_lo, v);
        if (!stage(4, 2, d)) break;
        // I0 -> I1: b = r goes to row (b, c), K index k1 = j
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            cf a = cmake(d[2 * r], d[2 * r + 1]);
            if (r) a = cmul(a, twc_inv(j * r));
            xb[(r * 16 + j) * COLS + c] = a;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = xb[(j * 16 + k) * COLS + c];
        put_row<16>(t_hi, t_lo, v);
        if (!stage(4, 2, d)) break;
        float2 *dst = Z + (size_t)(b0 + bi) * M * plane + f0 + c;
#pragma unroll
        for (int r = 0; r < 16; ++r) __stcs(&dst[(size_t)(j + 16 * r) * plane], make_float2(d[2 * r], d[2 * r + 1]));
    }
    // a product still in flight after a timeout: wait for it (bounded) before
    // its tensor memory is released
    if (lost >= 0 && tid == 0) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&mbar, (uint32_t)lost) && clock64() - t0 < C::WAIT_CYCLES) {
        }
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------------------
// z pass of the label-aware score at M = 256 over 16 columns per CTA (the
// dual form of k_zpass16): per rotation the forward FFTs along z of Y (the
// contact sweep) and of Y2 (the non-contact sweep), the products with the
// object's spectrum conj(F(O)) / M^3 and with conj(F(min(O, 0))) / M^3 (the
// second only for requests with non-contact poses), summed before one inverse
// FFT.  Both spectrum tiles sit in shared memory (reloaded when the request
// changes), both inputs of the next rotation are in flight during the current
// one, and the three transforms share one [256][16] exchange buffer.
// ---------------------------------------------------------------------------
struct Zpass16DualCfg {
    static constexpr int M = 256, N = 128, P = 130, NT = 256, COLS = 16;
    static constexpr size_t SMEM = (size_t)3 * M * COLS * 8;   // exchange + two spectrum tiles
    static_assert(2 * (SMEM + 1024) <= 228 * 1024, "two blocks per SM");
};

__global__ void __launch_bounds__(Zpass16DualCfg::NT, 2)
k_zpass16_dual(int B, int group, const float2 *__restrict__ Y, const float2 *__restrict__ Y2, const RotRec *rots,
               const ReqDev *reqs, float2 *Z)
{
    using C = Zpass16DualCfg;
    constexpr int M = C::M, N = C::N, P = C::P, COLS = C::COLS;
    extern __shared__ __align__(16) unsigned char smem[];
    cf *xb = reinterpret_cast<cf *>(smem);    // [M][COLS]
    cf *spt = xb + M * COLS;                   // [M (kz)][COLS]: conj(F(O)) / M^3
    cf *ppt = spt + M * COLS;                  // [M (kz)][COLS]: conj(F(min(O, 0))) / M^3
    const int tid = threadIdx.x, c = tid & 15, j = tid >> 4;
    const size_t plane = (size_t)M * P;
    const int f0 = blockIdx.x * COLS;
    const int b0 = blockIdx.y * group, nb = min(group, B - b0);
    if (nb <= 0) return;
    auto load = [&](const float2 *src0, int bi, cf *v) {
        const float2 *src = src0 + (size_t)(b0 + bi) * N * plane + f0 + c;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const float2 a = __ldcs(&src[(size_t)(j + 16 * s) * plane]);
            v[s] = cmake(a.x, a.y);
        }
    };
    // forward DFT of the zero-padded column held as inputs z = j + 16 s
    // (s < 8): on return v[r] holds kz = j + 16 r
    auto forward = [&](cf *v) {
#pragma unroll
        for (int s = 8; s < 16; ++s) v[s] = cmake(0.f, 0.f);
        DFT<16, false>::run(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) xb[(16 * j + r) * COLS + c] = v[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = xb[(j + 16 * r) * COLS + c];
#pragma unroll
        for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], cconj(twc_inv(j * r)));   // exp(-2 pi i j r / 256)
        DFT<16, false>::run(v);
    };
    cf nx[8], nx2[8];
    load(Y, 0, nx);
    load(Y2, 0, nx2);
    int sp_req = -1;
#pragma unroll 1
    for (int bi = 0; bi < nb; ++bi) {
        cf v[16], w[16];
#pragma unroll
        for (int s = 0; s < 8; ++s) v[s] = nx[s];
        if (bi + 1 < nb) load(Y, bi + 1, nx);
        const int req = rots[b0 + bi].req;
        const bool pen = reqs[req].P_nc > 0;
        if (req != sp_req) {   // block-uniform
            __syncthreads();   // the previous tiles are no longer read
            // tiled spectra: ((f / 32) M + kz) 32 + f mod 32
            const size_t off = (size_t)(f0 / 32) * M * 32 + (f0 & 31) + c;
            const float2 *src = reqs[req].spec + off;
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                const float2 a = __ldg(&src[(size_t)(j + 16 * r) * 32]);
                spt[(j + 16 * r) * COLS + c] = cmake(a.x, a.y);
            }
            if (pen) {
                const float2 *srcp = reqs[req].spec_pen + off;
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    const float2 a = __ldg(&srcp[(size_t)(j + 16 * r) * 32]);
                    ppt[(j + 16 * r) * COLS + c] = cmake(a.x, a.y);
                }
            }
            sp_req = req;
        }
        const float cj = reqs[req].rotate_object ? -1.f : 1.f;
        // contact sweep: w = F(S) conj(F(O)) / M^3 (a rotated object: conj(F(O_R)) F(S) / M^3)
        forward(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            cf a = v[r];
            a.y *= cj;
            w[r] = cmul(a, spt[(j + 16 * r) * COLS + c]);
        }
        if (pen) {   // block-uniform
            // non-contact sweep: w += F(S_nc) conj(F(min(O, 0))) / M^3
#pragma unroll
            for (int s = 0; s < 8; ++s) v[s] = nx2[s];
            if (bi + 1 < nb) load(Y2, bi + 1, nx2);
            __syncthreads();   // every thread has read its forward stage-1 inputs
            forward(v);
#pragma unroll
            for (int r = 0; r < 16; ++r) w[r] = cadd(w[r], cmul(v[r], ppt[(j + 16 * r) * COLS + c]));
        } else if (bi + 1 < nb) {
            load(Y2, bi + 1, nx2);
        }
        __syncthreads();   // every thread has read its last forward stage-1 inputs
        // inverse, stage 0 (inputs kz = j + 16 r) -> index 16 j + r
        DFT<16, true>::run(w);
#pragma unroll
        for (int r = 0; r < 16; ++r) xb[(16 * j + r) * COLS + c] = w[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 16; ++r) w[r] = xb[(j + 16 * r) * COLS + c];
#pragma unroll
        for (int r = 1; r < 16; ++r) w[r] = cmul(w[r], twc_inv(j * r));
        DFT<16, true>::run(w);
        float2 *dst = Z + (size_t)(b0 + bi) * M * plane + f0 + c;
#pragma unroll
        for (int r = 0; r < 16; ++r) __stcs(&dst[(size_t)(j + 16 * r) * plane], make_float2(w[r].x, w[r].y));
        __syncthreads();   // the exchange buffer is free for the next rotation
    }
}

// Fills c_tw256 on the current device once (the module's constant bank is per device).
static cudaError_t ensure_twiddle_bank()
{
    static std::mutex mu;
    static bool done[256] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return cudaSuccess;
    float2 h[256];
    for (int m = 0; m < 256; ++m) {
        const double a = -2.0 * M_PI * (double)m / 256.0;
        h[m] = make_float2((float)cos(a), (float)sin(a));
    }
    e = cudaMemcpyToSymbol(c_tw256, h, sizeof(h));
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

template <int CL, bool EXPORT>
static cudaError_t launch_plane_cl_t(int B, const float2 *Z, const float2 *tw, const RotRec *rots, const ReqDev *reqs,
                                     float *Cout, int *err, cudaStream_t st, int withhold = 0)
{
    using C = PlaneClCfg<CL>;
    auto kern = k_plane_cl<CL, EXPORT>;
    cudaError_t e = ensure_twiddle_bank();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C::M * CL, B);
    cfg.blockDim = dim3(C::NT);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, Z, tw, rots, reqs, Cout, err, withhold);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

bool plane_cl_supported(int M, int cl) { return M == 256 && (cl == 4 || cl == 8); }

cudaError_t launch_zpass16(const Geo &g, int B, int group, const float2 *Y, const RotRec *rots, const ReqDev *reqs,
                           float2 *Z, cudaStream_t st)
{
    using C = Zpass16Cfg;
    if (g.M != C::M || g.P != C::P || B < 1 || group < 1) return cudaErrorInvalidValue;
    cudaError_t e = ensure_twiddle_bank();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_zpass16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid(C::M * C::P / C::COLS, (B + group - 1) / group);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    k_zpass16<<<grid, C::NT, C::SMEM, st>>>(B, group, Y, rots, reqs, Z);
    return cudaGetLastError();
}


cudaError_t launch_zpass_tc(const Geo &g, int B, int group, const float2 *Y, const RotRec *rots, const ReqDev *reqs,
                            float2 *Z, int *err, cudaStream_t st)
{
    using C = ZpassTcCfg;
    if (g.M != C::M || g.P != C::P || B < 1 || group < 1) return cudaErrorInvalidValue;
    cudaError_t e = ensure_twiddle_bank();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_zpass_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid(C::M * C::P / C::COLS, (B + group - 1) / group);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    k_zpass_tc<<<grid, C::NT, C::SMEM, st>>>(B, group, Y, rots, reqs, Z, err);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to
// the driver library)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    std::lock_guard<std::mutex> lk(mu);
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

// Z as a 2-D FP32 tensor (2 P floats per canvas row, `rows` rows), boxes of
// box_x floats x 256 rows
static cudaError_t z_tensor_map(CUtensorMap *m, const float2 *Z, size_t rows, uint32_t box_x)
{
    using C = PlanePsCfg<4>;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t gdim[2] = {2 * (cuuint64_t)C::P, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {2 * (cuuint64_t)C::P * sizeof(float)};
    const cuuint32_t box[2] = {box_x, (cuuint32_t)C::M};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2 *>(Z), gdim, gstride, box, estride,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CL, bool EXPORT>
static cudaError_t launch_plane_ps_t(int n_planes, const float2 *Z, const RotRec *rots, const ReqDev *reqs,
                                     float *Cout, int *err, cudaStream_t st, int withhold = 0)
{
    using C = PlanePsCfg<CL>;
    auto kern = k_plane_ps<CL, EXPORT>;
    if (n_planes < 1) return cudaErrorInvalidValue;
    cudaError_t e = ensure_twiddle_bank();
    if (e != cudaSuccess) return e;
    CUtensorMap zm, nm;
    if ((e = z_tensor_map(&zm, Z, (size_t)n_planes * C::M, 2 * C::CPC)) != cudaSuccess) return e;
    if ((e = z_tensor_map(&nm, Z, (size_t)n_planes * C::M, 4)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM)) != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(C::NT);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C::CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // as many clusters as are resident at once (each walks its share of planes)
    cfg.gridDim = dim3(C::CL * 1024);
    int resident = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&resident, kern, &cfg)) != cudaSuccess) return e;
    if (resident < 1) return cudaErrorInvalidConfiguration;
    cfg.gridDim = dim3(C::CL * (unsigned)std::min(resident, n_planes));
    return cudaLaunchKernelEx(&cfg, kern, zm, nm, n_planes, rots, reqs, Cout, err, withhold);
}

bool plane_ps_supported(int M, int cl) { return M == 256 && (cl == 4 || cl == 8); }

// The persistent pass refused before launching: no tensor-map encoder in the
// driver, or no cluster of its size resident on this device right now.  The
// error recorded by the failed query is cleared; the caller uses the
// one-cluster-per-plane pass instead.
bool plane_ps_unavailable(cudaError_t e)
{
    if (e != cudaErrorNotSupported && e != cudaErrorInvalidConfiguration) return false;
    (void)cudaGetLastError();
    return true;
}

cudaError_t launch_plane_ps(const Geo &g, int cl, int B, const float2 *Z, const RotRec *rots, const ReqDev *reqs,
                            int *err, cudaStream_t st)
{
    if (!plane_ps_supported(g.M, cl) || g.P != PlanePsCfg<4>::P || B < 1 || B > 65535) return cudaErrorInvalidValue;
    return cl == 4 ? launch_plane_ps_t<4, false>(B * g.M, Z, rots, reqs, nullptr, err, st)
                   : launch_plane_ps_t<8, false>(B * g.M, Z, rots, reqs, nullptr, err, st);
}

cudaError_t launch_plane_ps_export(const Geo &g, int cl, const float2 *Z, float *C, int *err, cudaStream_t st,
                                   int withhold)
{
    if (!plane_ps_supported(g.M, cl) || g.P != PlanePsCfg<4>::P) return cudaErrorInvalidValue;
    return cl == 4 ? launch_plane_ps_t<4, true>(g.M, Z, nullptr, nullptr, C, err, st, withhold)
                   : launch_plane_ps_t<8, true>(g.M, Z, nullptr, nullptr, C, err, st, withhold);
}

cudaError_t launch_fwd2d_runs(const Geo &g, int B, const uint32_t *bits, float2 *Y, const float2 *q,
                              const uint32_t *mask, cudaStream_t st)
{
    using C = FwdRunsCfg;
    if (g.M != C::M || g.N != C::N || g.P != C::P || B < 1 || B > 65535) return cudaErrorInvalidValue;
    cudaError_t e = ensure_twiddle_bank();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fwd2d_runs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    k_fwd2d_runs<<<dim3(C::N, B), C::NT, C::SMEM, st>>>(bits, mask, Y, q);
    return cudaGetLastError();
}

cudaError_t launch_zpass16_dual(const Geo &g, int B, int group, const float2 *Y, const float2 *Y2, const RotRec *rots,
                                const ReqDev *reqs, float2 *Z, cudaStream_t st)
{
    using C = Zpass16DualCfg;
    if (g.M != C::M || g.P != C::P || B < 1 || group < 1) return cudaErrorInvalidValue;
    cudaError_t e = ensure_twiddle_bank();
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_zpass16_dual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid(C::M * C::P / C::COLS, (B + group - 1) / group);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    k_zpass16_dual<<<grid, C::NT, C::SMEM, st>>>(B, group, Y, Y2, rots, reqs, Z);
    return cudaGetLastError();
}

cudaError_t launch_plane_cl(const Geo &g, int cl, int B, const float2 *Z, const float2 *tw, const RotRec *rots,
                            const ReqDev *reqs, int *err, cudaStream_t st)
{
    if (!plane_cl_supported(g.M, cl) || B < 1 || B > 65535) return cudaErrorInvalidValue;
    return cl == 4 ? launch_plane_cl_t<4, false>(B, Z, tw, rots, reqs, nullptr, err, st)
                   : launch_plane_cl_t<8, false>(B, Z, tw, rots, reqs, nullptr, err, st);
}

cudaError_t launch_plane_cl_export(const Geo &g, int cl, const float2 *Z, const float2 *tw, float *C, int *err,
                                   cudaStream_t st, int withhold)
{
    if (!plane_cl_supported(g.M, cl)) return cudaErrorInvalidValue;
    return cl == 4 ? launch_plane_cl_t<4, true>(1, Z, tw, nullptr, nullptr, C, err, st, withhold)
                   : launch_plane_cl_t<8, true>(1, Z, tw, nullptr, nullptr, C, err, st, withhold);
}

}  // namespace dock
