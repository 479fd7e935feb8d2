// Search pipeline on library-owned scratch, for callers that cannot allocate
// device memory (a host framework that owns every device allocation through
// its own pool, or code running where cudaMalloc is forbidden, e.g. between
// allocations that a memory planner has fixed).  The paper has no
// counterpart: this is a systems entry point around the same kernels
// (voxeliser, forward x/y pass, z pass, plane pass) that dock_search_so3 uses.
//
// The scratch is one file-scope device array of fixed size.  Every GPU that
// loads the library holds it until the process exits.  All calls on a device
// share it, so calls that overlap on the GPU race; a call leaves its contents
// behind and the next call clears what must start at zero (the peak keys).
#include <mutex>

#include "dock_internal.h"

namespace dock {

namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t NA_M = 2 * (size_t)NOALLOC_MAX_N;
constexpr size_t NA_P = NA_M / 2 + 2;
constexpr size_t OFF_BITS = 0;
constexpr size_t OFF_Y = align256(OFF_BITS + (size_t)NOALLOC_MAX_N * NOALLOC_MAX_N * (NOALLOC_MAX_N / 32) * 4);
constexpr size_t OFF_Z = align256(OFF_Y + (size_t)NOALLOC_MAX_N * NA_M * NA_P * sizeof(float2));
constexpr size_t OFF_QUAT = align256(OFF_Z + NA_M * NA_M * NA_P * sizeof(float2));
constexpr size_t OFF_ROT = align256(OFF_QUAT + (size_t)NOALLOC_MAX_ROT * 4 * sizeof(double));
constexpr size_t OFF_KEY = align256(OFF_ROT + (size_t)NOALLOC_MAX_ROT * sizeof(RotRec));
constexpr size_t OFF_PEAK = align256(OFF_KEY + (size_t)NOALLOC_MAX_ROT * sizeof(unsigned long long));
constexpr size_t OFF_REQ = align256(OFF_PEAK + (size_t)NOALLOC_MAX_ROT * sizeof(dock_peak));
constexpr size_t NA_BYTES = align256(OFF_REQ + sizeof(ReqDev));

}  // namespace

// About 13.9 MB at N <= 64 and 4096 rotations per call.
static __device__ __align__(256) unsigned char noalloc_scratch[NA_BYTES];

size_t noalloc_scratch_bytes() { return NA_BYTES; }

// Device address of the scratch on the current device, looked up once per
// device.  On the host the name noalloc_scratch only stands in for the device
// symbol; its address is not a device pointer.
static cudaError_t scratch_address(int dev, unsigned char **out)
{
    static std::mutex mu;
    static unsigned char *addr[NOALLOC_MAX_DEVICES] = {};
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = (unsigned char *)p;
    }
    *out = addr[dev];
    return cudaSuccess;
}

cudaError_t noalloc_prepare(int device)
{
    unsigned char *p = nullptr;
    return scratch_address(device, &p);
}

// Peak key (ordered score << 32 | ~canvas index, 0 = no peak) to (score, index).
__global__ void k_keys_to_peaks(const unsigned long long *keys, int n, dock_peak *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long k = keys[i];
    dock_peak p;
    if (k == 0ull) {
        p.score = -INFINITY;
        p.canvas_idx = -1;
    } else {
        uint32_t sk = (uint32_t)(k >> 32);
        uint32_t u = (sk & 0x80000000u) ? (sk & 0x7FFFFFFFu) : ~sk;
        p.score = __uint_as_float(u);
        p.canvas_idx = (int32_t)(0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull));
    }
    out[i] = p;
}

cudaError_t noalloc_search_peaks(const NoallocJob &j)
{
    if (j.g.N > NOALLOC_MAX_N || j.n > NOALLOC_MAX_ROT || j.n < 1) return cudaErrorInvalidValue;
    unsigned char *base = nullptr;
    cudaError_t e = scratch_address(j.device, &base);
    if (e != cudaSuccess) return e;
    uint32_t *bits = (uint32_t *)(base + OFF_BITS);
    float2 *Y = (float2 *)(base + OFF_Y);
    float2 *Z = (float2 *)(base + OFF_Z);
    double *quats = (double *)(base + OFF_QUAT);
    RotRec *rots = (RotRec *)(base + OFF_ROT);
    unsigned long long *keys = (unsigned long long *)(base + OFF_KEY);
    dock_peak *peaks = (dock_peak *)(base + OFF_PEAK);
    ReqDev *req = (ReqDev *)(base + OFF_REQ);
    ReqDev r = j.req;
    r.keys = keys;
    const cudaStream_t st = j.stream;
    // pageable sources: the copies have taken the host data when they return
    if ((e = cudaMemcpyAsync(quats, j.quats, sizeof(double) * 4 * j.n, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(req, &r, sizeof(ReqDev), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * j.n, st)) != cudaSuccess) return e;
    if ((e = launch_rot_setup(quats, j.n, 0, 0, j.c_s, j.g.h, j.g.N, rots, st)) != cudaSuccess) return e;
    // one rotation per pass: the scratch holds the Y and Z arrays of one rotation
    for (int b = 0; b < j.n; ++b) {
        if ((e = launch_voxelise(j.g, req, rots + b, 1, bits, st)) != cudaSuccess) return e;
        if ((e = launch_fwd2d(j.g, 1, bits, Y, j.tw, j.qt, st)) != cudaSuccess) return e;
        if ((e = launch_zpass(j.g, 1, 1, Y, rots + b, req, Z, j.tw, st)) != cudaSuccess) return e;
        if ((e = launch_plane(j.g, 1, Z, j.tw, rots + b, req, st)) != cudaSuccess) return e;
    }
    k_keys_to_peaks<<<(j.n + 127) / 128, 128, 0, st>>>(keys, j.n, peaks);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(j.peaks, peaks, sizeof(dock_peak) * j.n, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(st);
}

}  // namespace dock
