// Batched shared-memory radix FFT building blocks for the docking correlation
// (Sec. IV-B, Eq. (9)).  A length-M transform is split into Stockham stages of
// small radices computed in registers; between stages the data of one batch of
// columns goes through shared memory laid out [element][column], so threads
// with consecutive column indices touch consecutive words (no bank conflicts).
//
// Plan<M, V>: T threads per column, each holding E complex values; stage s has
// radix R[s] and every thread computes E / R[s] butterflies of it.  V selects
// one of the radix plans of a length (0: the default; 1: the alternative the
// autotuner may pick, canvases 64 and 128).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dock {

struct cf { float x, y; };

__device__ __forceinline__ cf cmake(float a, float b) { cf r; r.x = a; r.y = b; return r; }
__device__ __forceinline__ cf cadd(cf a, cf b) { return cmake(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cf csub(cf a, cf b) { return cmake(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cf cmul(cf a, cf b) { return cmake(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ cf cconj(cf a) { return cmake(a.x, -a.y); }
__device__ __forceinline__ cf cscale(cf a, float s) { return cmake(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ cf mul_mi(cf a) { return INV ? cmake(-a.y, a.x) : cmake(a.y, -a.x); }
// multiply by exp(-+ 2 pi i k / 8) for k = 1, 3
template <bool INV> __device__ __forceinline__ cf mul_w8_1(cf a)
{
    const float s = 0.70710678118654752f;
    return INV ? cmake((a.x - a.y) * s, (a.x + a.y) * s) : cmake((a.x + a.y) * s, (a.y - a.x) * s);
}
template <bool INV> __device__ __forceinline__ cf mul_w8_3(cf a)
{
    const float s = 0.70710678118654752f;
    return INV ? cmake(-(a.x + a.y) * s, (a.x - a.y) * s) : cmake((a.y - a.x) * s, -(a.x + a.y) * s);
}
// exp(-+ 2 pi i / 16) and exp(-+ 2 pi i 3 / 16)
template <bool INV> __device__ __forceinline__ cf mul_w16(cf a, int k)
{
    const float c1 = 0.92387953251128676f, s1 = 0.38268343236508977f;
    float c, s;
    switch (k) {
    case 1: c = c1; s = s1; break;
    case 2: c = 0.70710678118654752f; s = 0.70710678118654752f; break;
    case 3: c = s1; s = c1; break;
    case 4: c = 0.f; s = 1.f; break;
    case 6: c = -0.70710678118654752f; s = 0.70710678118654752f; break;
    case 9: c = -c1; s = -s1; break;
    default: c = 1.f; s = 0.f; break;
    }
    // forward twiddle = c - i s, inverse = c + i s
    if (INV) return cmake(a.x * c - a.y * s, a.x * s + a.y * c);
    return cmake(a.x * c + a.y * s, a.y * c - a.x * s);
}

template <bool INV> __device__ __forceinline__ void dft2(cf &a, cf &b)
{
    cf t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <bool INV> __device__ __forceinline__ void dft3(cf &a, cf &b, cf &c)
{
    const float h = -0.5f, s = INV ? 0.86602540378443865f : -0.86602540378443865f;
    cf t1 = cadd(b, c), t2 = csub(b, c);
    cf m = cmake(a.x + h * t1.x, a.y + h * t1.y);
    cf r = cmake(-s * t2.y, s * t2.x);   // i s (b - c)
    a = cadd(a, t1);
    b = cadd(m, r);
    c = csub(m, r);
}

template <bool INV> __device__ __forceinline__ void dft4(cf &a, cf &b, cf &c, cf &d)
{
    cf t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = mul_mi<INV>(csub(b, d));
    a = cadd(t0, t2);
    c = csub(t0, t2);
    b = cadd(t1, t3);
    d = csub(t1, t3);
}

// In-place DFT of R values v[0..R) (natural order in and out).
template <int R, bool INV> struct DFT;

template <bool INV> struct DFT<2, INV> {
    __device__ __forceinline__ static void run(cf *v) { dft2<INV>(v[0], v[1]); }
};
template <bool INV> struct DFT<3, INV> {
    __device__ __forceinline__ static void run(cf *v) { dft3<INV>(v[0], v[1], v[2]); }
};
template <bool INV> struct DFT<4, INV> {
    __device__ __forceinline__ static void run(cf *v) { dft4<INV>(v[0], v[1], v[2], v[3]); }
};
template <bool INV> struct DFT<8, INV> {
    __device__ __forceinline__ static void run(cf *v)
    {
        // X[k] = E[k] + w8^k O[k], X[k+4] = E[k] - w8^k O[k]
        dft4<INV>(v[0], v[2], v[4], v[6]);
        dft4<INV>(v[1], v[3], v[5], v[7]);
        cf o1 = mul_w8_1<INV>(v[3]), o2 = mul_mi<INV>(v[5]), o3 = mul_w8_3<INV>(v[7]);
        cf e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
        v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
        v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
        v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
        v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
    }
};
template <bool INV> struct DFT<16, INV> {
    __device__ __forceinline__ static void run(cf *v)
    {
        // n = n1 + 4 n2 ; k = k1 + 4 k2
        cf a[4][4];
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) {
            a[n1][0] = v[n1]; a[n1][1] = v[n1 + 4]; a[n1][2] = v[n1 + 8]; a[n1][3] = v[n1 + 12];
            dft4<INV>(a[n1][0], a[n1][1], a[n1][2], a[n1][3]);
        }
#pragma unroll
        for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) a[n1][k1] = mul_w16<INV>(a[n1][k1], n1 * k1);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            dft4<INV>(a[0][k1], a[1][k1], a[2][k1], a[3][k1]);
            v[k1] = a[0][k1]; v[k1 + 4] = a[1][k1]; v[k1 + 8] = a[2][k1]; v[k1 + 12] = a[3][k1];
        }
    }
};
template <bool INV> struct DFT<12, INV> {
    __device__ __forceinline__ static void run(cf *v)
    {
        // n = n1 + 3 n2 (n1 < 3, n2 < 4); k = k1 + 4 k2
        cf a[3][4];
#pragma unroll
        for (int n1 = 0; n1 < 3; ++n1) {
            a[n1][0] = v[n1]; a[n1][1] = v[n1 + 3]; a[n1][2] = v[n1 + 6]; a[n1][3] = v[n1 + 9];
            dft4<INV>(a[n1][0], a[n1][1], a[n1][2], a[n1][3]);
        }
        // twiddles w12^(n1 k1)
        const float c1 = 0.86602540378443865f, s1 = 0.5f;   // w12^1
#pragma unroll
        for (int n1 = 1; n1 < 3; ++n1)
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) {
                int e = n1 * k1;   // 1..6
                float c, s;
                switch (e) {
                case 1: c = c1; s = s1; break;
                case 2: c = 0.5f; s = c1; break;
                case 3: c = 0.f; s = 1.f; break;
                case 4: c = -0.5f; s = c1; break;
                default: c = -1.f; s = 0.f; break;   // 6
                }
                cf z = a[n1][k1];
                a[n1][k1] = INV ? cmake(z.x * c - z.y * s, z.x * s + z.y * c)
                                : cmake(z.x * c + z.y * s, z.y * c - z.x * s);
            }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            dft3<INV>(a[0][k1], a[1][k1], a[2][k1]);
            v[k1] = a[0][k1]; v[k1 + 4] = a[1][k1]; v[k1 + 8] = a[2][k1];
        }
    }
};

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
template <int M, int V = 0> struct Plan;
template <> struct Plan<32>  { static constexpr int T = 4,  E = 8,  S = 2; __host__ __device__ static constexpr int R(int s) { return s == 0 ? 8 : 4; } };
template <> struct Plan<64>  { static constexpr int T = 8,  E = 8,  S = 2; __host__ __device__ static constexpr int R(int s) { return 8; } };
template <> struct Plan<96>  { static constexpr int T = 8,  E = 12, S = 3; __host__ __device__ static constexpr int R(int s) { return s == 0 ? 12 : (s == 1 ? 4 : 2); } };
template <> struct Plan<128> { static constexpr int T = 8,  E = 16, S = 2; __host__ __device__ static constexpr int R(int s) { return s == 0 ? 16 : 8; } };
template <> struct Plan<192> { static constexpr int T = 16, E = 12, S = 3; __host__ __device__ static constexpr int R(int s) { return s == 0 ? 12 : 4; } };
template <> struct Plan<256> { static constexpr int T = 16, E = 16, S = 2; __host__ __device__ static constexpr int R(int s) { return 16; } };
// alternatives: 64 = 16 x 4 (4 threads per column), 128 = 8 x 8 x 2 (16 threads per column)
template <> struct Plan<64, 1>  { static constexpr int T = 4,  E = 16, S = 2; __host__ __device__ static constexpr int R(int s) { return s == 0 ? 16 : 4; } };
template <> struct Plan<128, 1> { static constexpr int T = 16, E = 8,  S = 3; __host__ __device__ static constexpr int R(int s) { return s == 2 ? 2 : 8; } };
// whether length M has plan V
template <int M, int V> struct HasPlan { static constexpr bool value = V == 0 || ((M == 64 || M == 128) && V == 1); };

template <int M, int s, int V = 0> struct Ns { static constexpr int v = Ns<M, s - 1, V>::v * Plan<M, V>::R(s - 1); };
template <int M, int V> struct Ns<M, 0, V> { static constexpr int v = 1; };

// tw[m] = exp(-2 pi i m / M) for m in [0, M)
template <bool INV> __device__ __forceinline__ cf twiddle(const cf *tw, int m)
{
    cf w = tw[m];
    return INV ? cconj(w) : w;
}

// One Stockham stage on the thread's registers.  Input element of butterfly
// j, leg r: index j + r M/R; output index (j / Ns) Ns R + (j % Ns) + r Ns.
// `v` holds E values: butterfly b (j = t + T b) occupies v[b R .. b R + R).
template <int M, int s, bool INV, int TWS = 1, int V = 0>
__device__ __forceinline__ void stage_compute(cf *v, int t, const cf *tw)
{
    constexpr int R = Plan<M, V>::R(s), E = Plan<M, V>::E, T = Plan<M, V>::T, NS = Ns<M, s, V>::v;
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
        int j = t + T * b;
        if (NS > 1) {
            int jm = j % NS;
#pragma unroll
            for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], twiddle<INV>(tw, ((jm * r * (M / (NS * R))) % M) * TWS));
        }
        DFT<R, INV>::run(v + b * R);
    }
}

// Load the inputs of stage s from an [M][ncol] buffer.
template <int M, int s, int V = 0>
__device__ __forceinline__ void stage_load(cf *v, int t, const cf *buf, int col, int ncol)
{
    constexpr int R = Plan<M, V>::R(s), E = Plan<M, V>::E, T = Plan<M, V>::T;
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
        int j = t + T * b;
#pragma unroll
        for (int r = 0; r < R; ++r) v[b * R + r] = buf[(j + r * (M / R)) * ncol + col];
    }
}

template <int M, int s, int V = 0>
__device__ __forceinline__ void stage_store(const cf *v, int t, cf *buf, int col, int ncol)
{
    constexpr int R = Plan<M, V>::R(s), E = Plan<M, V>::E, T = Plan<M, V>::T, NS = Ns<M, s, V>::v;
#pragma unroll
    for (int b = 0; b < E / R; ++b) {
        int j = t + T * b;
        int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
        for (int r = 0; r < R; ++r) buf[(base + r * NS) * ncol + col] = v[b * R + r];
    }
}

// Natural-order output index of register slot (b, r) after the last stage.
template <int M, int V = 0>
__device__ __forceinline__ int out_index(int t, int slot)
{
    constexpr int s = Plan<M, V>::S - 1, R = Plan<M, V>::R(s), T = Plan<M, V>::T, NS = Ns<M, s, V>::v;
    int b = slot / R, r = slot % R;
    int j = t + T * b;
    return (j / NS) * NS * R + (j % NS) + r * NS;
}

// True when register slot s of the first stage reads an index in [0, M/2):
// with one butterfly per thread (E = R0) and M / R0 = T, slot s reads
// j + T s, which is below M/2 exactly when s < R0/2, whatever the thread j.
// Zero-padded inputs (the upper half) then need no load.
template <int M, int V = 0>
__device__ __forceinline__ constexpr bool slot_in_lower_half(int s)
{
    static_assert(Plan<M, V>::E == Plan<M, V>::R(0) && M / Plan<M, V>::R(0) == Plan<M, V>::T, "first-stage layout");
    return s < Plan<M, V>::R(0) / 2;
}

// Input index of register slot (b, r) for the first stage.
template <int M, int V = 0>
__device__ __forceinline__ int in_index(int t, int slot)
{
    constexpr int R = Plan<M, V>::R(0), T = Plan<M, V>::T;
    int b = slot / R, r = slot % R;
    return t + T * b + r * (M / R);
}

// Full transform of one column.  On entry v holds the first stage's inputs
// (slot -> in_index); on exit v holds the outputs (slot -> out_index).  `xb`
// is the [M][ncol] exchange buffer shared by the block; all threads of the
// block must call this together (it contains __syncthreads()).  The twiddle
// table holds exp(-2 pi i m / (M TWS)); entry m TWS is used for exponent m.
template <int M, bool INV, int TWS = 1, int V = 0>
__device__ __forceinline__ void fft_column(cf *v, int t, cf *xb, int col, int ncol, const cf *tw)
{
    stage_compute<M, 0, INV, TWS, V>(v, t, tw);
    if constexpr (Plan<M, V>::S >= 2) {
        stage_store<M, 0, V>(v, t, xb, col, ncol);
        __syncthreads();
        stage_load<M, 1, V>(v, t, xb, col, ncol);
        __syncthreads();
        stage_compute<M, 1, INV, TWS, V>(v, t, tw);
    }
    if constexpr (Plan<M, V>::S >= 3) {
        stage_store<M, 1, V>(v, t, xb, col, ncol);
        __syncthreads();
        stage_load<M, 2, V>(v, t, xb, col, ncol);
        __syncthreads();
        stage_compute<M, 2, INV, TWS, V>(v, t, tw);
    }
}

}  // namespace dock
