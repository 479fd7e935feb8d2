// Internal declarations shared by the host runtime and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>
#include <map>

#include "../../include/dock.h"

namespace dock {

// Per-rotation lattice set-up, FP64 (exact operation order) and FP32 copies.
// Rotating the sweep (default): o = the swept-lattice origin o_s,R.
// Rotating the object (Sec. IV-D as printed): o = o_R, the rotated object
// lattice's origin, and ub = (R^T o_R - o_o) / h, so that voxel k of the
// rotated object samples O at the continuous index R^T k + ub.
struct RotRec {
    double R[9];   // rotation of the sample (row-major)
    double o[3];
    float Rf[9];
    float of[3];
    float ub[3];
    int32_t rot;   // sample index within its request
    int32_t req;   // request index in the launch's request table
};

// Per-pose data of a sweep: FP64 rotation/translation (exact recheck) and FP32.
struct PoseRec {
    double R[9];
    double t[3];
    float Rf[9];
    float tf[3];
};

// Geometry of one search pipeline configuration.
struct Geo {
    int N;      // lattice side
    int M;      // canvas side (2N)
    int P;      // row pitch of half-spectrum arrays in complex elements (M/2 + 2)
    double h;
    float inv_h;
    float rv;   // probe radius in voxels
    float lv;   // probe length in voxels
    double r, L;
};

// Per-request data of a search launch: the rotations of one launch may come
// from several registrations that share the lattice side N.
// Pose set 0 is (poses, P): every pose of a plain request, the contact poses
// of a label-aware one.  Pose set 1 is (poses_nc, P_nc): the non-contact
// poses of a label-aware request (P_nc = 0 otherwise), whose voxels scored
// against spec_pen count only where set 0 leaves them uncovered.
struct ReqDev {
    const PoseRec *poses;
    int P;
    double h, r, L;           // voxel size, probe radius and length (mm)
    float inv_h, rv, lv;      // FP32 copies; rv, lv in voxels
    const float2 *spec;       // tiled conj(F(O)) / M^3 of the request's object
    unsigned long long *keys; // per-rotation peak keys, indexed by RotRec::rot
    const PoseRec *poses_nc;  // label-aware: non-contact poses (else nullptr)
    int P_nc;
    const float2 *spec_pen;   // label-aware: tiled conj(F(min(O, 0))) / M^3 (else nullptr)
    // rotate_object: the object grid is rotated and resampled per rotation
    // (from its corner cells Og4, (N+1)^3) and spec holds F(S) / M^3 of the
    // fixed swept grid
    const float4 *Og4;
    int rotate_object;
};

// Kernel launchers (k_search.cu)
// o_o (nullable, device): rotate the object about its lattice instead of the
// sweep (o = o_R, ub set); c_s is then unused.
cudaError_t launch_rot_setup(const double *quats, int n, int rot0, int req, const double *c_s, double h, int N,
                             RotRec *out, cudaStream_t st, const double *o_o = nullptr);
// pose_set: 0 = (poses, P), 1 = (poses_nc, P_nc) of each rotation's request.
cudaError_t launch_voxelise(const Geo &g, const ReqDev *reqs, const RotRec *rots, int B, uint32_t *bits,
                            cudaStream_t st, int minb = 4, int pose_set = 0);
// mask (nullable, the layout of bits): bits & ~mask is transformed.  With
// rots/reqs given, rotations of rotate_object requests transform their
// resampled object grid instead of bits (and are skipped when mask is set).
// ogrids (nullable, B x N^3 floats): the rotated object grids made by
// launch_resample, read instead of resampling inside the x stage.
cudaError_t launch_fwd2d(const Geo &g, int B, const uint32_t *bits, float2 *Y, const float2 *tw, const float2 *q,
                         cudaStream_t st, const uint32_t *mask = nullptr, const RotRec *rots = nullptr,
                         const ReqDev *reqs = nullptr, const float *ogrids = nullptr, int fft_plan = 0);
// (fft_plan, here and in launch_zpass / launch_plane: the radix plan of the
// FFTs at canvases 64 and 128, 0 the default, 1 the alternative of fft.cuh;
// other canvases have one plan)
// The rotated object grids of the rotate_object rotations of a launch into out (B x N^3 floats).
cudaError_t launch_resample(const Geo &g, const ReqDev *reqs, const RotRec *rots, int B, float *out, cudaStream_t st);
// Y2 (nullable): transforms of the label-aware second grids; when given, the
// product with each request's spec_pen is added before the inverse FFT.
cudaError_t launch_zpass(const Geo &g, int B, int group, const float2 *Y, const RotRec *rots, const ReqDev *reqs,
                         float2 *Z, const float2 *tw, cudaStream_t st, const float2 *Y2 = nullptr,
                         int fft_plan = 0);
// plane_cl: CTAs per plane at M = 256 (4 or 8: the cluster kernel of
// k_fft256.cu; anything else: the 2-CTA kernel); plane_tma with plane_cl 4
// or 8: the persistent cluster kernel with TMA staging.  err (nullable, device):
// set to DOCK_E_TIMEOUT if a cluster kernel gave up waiting for its peers.
cudaError_t launch_plane(const Geo &g, int B, const float2 *Z, const float2 *tw, const RotRec *rots,
                         const ReqDev *reqs, cudaStream_t st, int plane_cl = 0, int *err = nullptr,
                         int plane_tma = 0, int fft_plan = 0);
// z pass over 16 columns per block (k_fft256.cu): M = 256, plain score only.
cudaError_t launch_zpass16(const Geo &g, int B, int group, const float2 *Y, const RotRec *rots, const ReqDev *reqs,
                           float2 *Z, cudaStream_t st);
// The cluster plane pass (k_fft256.cu): M = 256, cl = 4 or 8.
// z pass of the label-aware score over 16 columns per block: M = 256
cudaError_t launch_zpass16_dual(const Geo &g, int B, int group, const float2 *Y, const float2 *Y2, const RotRec *rots,
                                const ReqDev *reqs, float2 *Z, cudaStream_t st);
// z pass with its DFT stages as 3 x TF32 products on the tensor cores (canvas 256, plain score)
cudaError_t launch_zpass_tc(const Geo &g, int B, int group, const float2 *Y, const RotRec *rots, const ReqDev *reqs,
                            float2 *Z, int *err, cudaStream_t st);
// forward x and y passes of binary slabs at canvas 256 from their run lists
// (bits & ~mask when mask is given); no rotated-object requests
cudaError_t launch_fwd2d_runs(const Geo &g, int B, const uint32_t *bits, float2 *Y, const float2 *q,
                              const uint32_t *mask, cudaStream_t st);
// persistent cluster plane pass with TMA staging of the columns (canvas 256, 4 or 8 CTAs per plane)
bool plane_ps_supported(int M, int cl);
bool plane_ps_unavailable(cudaError_t e);
cudaError_t launch_plane_ps(const Geo &g, int cl, int B, const float2 *Z, const RotRec *rots, const ReqDev *reqs,
                            int *err, cudaStream_t st);
cudaError_t launch_plane_ps_export(const Geo &g, int cl, const float2 *Z, float *C, int *err, cudaStream_t st,
                                   int withhold = 0);
bool plane_cl_supported(int M, int cl);
cudaError_t launch_plane_cl(const Geo &g, int cl, int B, const float2 *Z, const float2 *tw, const RotRec *rots,
                            const ReqDev *reqs, int *err, cudaStream_t st);
// withhold = 1 (test hook): the peers' blocks are never pushed, so the
// bounded waits run out and set err to DOCK_E_TIMEOUT.
cudaError_t launch_plane_cl_export(const Geo &g, int cl, const float2 *Z, const float2 *tw, float *C, int *err,
                                   cudaStream_t st, int withhold = 0);
// o_s (nullable, device): the rotate_object pose T = (R, h dk + o_s - o_R);
// else T = (R, R (h dk + o_s,R - o_o)).
cudaError_t launch_topk(const unsigned long long *keys, int n, int K, int N, int M, double h, const double *o_o,
                        const double *quats, const RotRec *rots_all, dock_candidate *out, cudaStream_t st,
                        const double *o_s = nullptr);
cudaError_t launch_vox_export(const Geo &g, const ReqDev *reqs, const RotRec *rots, int B, uint8_t *bits,
                              cudaStream_t st, int pose_set = 0);
cudaError_t launch_plane_export(const Geo &g, const float2 *Z, const float2 *tw, float *C, cudaStream_t st,
                                int plane_cl = 0, int *err = nullptr, int plane_tma = 0, int fft_plan = 0);
// Corner cells of O for trilinear interpolation ((N+1)^3 float4).
cudaError_t launch_corner_cells(const float *O, int N, float4 *cells, cudaStream_t st);
// S of rotation 0 (pose set 0) as N^3 floats 0/1.
cudaError_t launch_vox_float(const Geo &g, const ReqDev *reqs, const RotRec *rots, float *out, cudaStream_t st);
// The resampled object grid of each of B rotate_object rotations (B x N^3 floats; test hook).
cudaError_t launch_rot_export(const Geo &g, const ReqDev *reqs, const RotRec *rots, int B, float *out, cudaStream_t st);

// Object grid kernels (k_object.cu)
struct ObjBins {
    const int32_t *cell3_start;  // 3-D cells, CSR
    const int32_t *cell3_items;
    const int32_t *cell2_start;  // (y,z) cells, CSR
    const int32_t *cell2_items;
    int d3[3];
    int d2[2];
    double cs;                    // cell size
};
cudaError_t launch_object_grid(const double *V, const int32_t *T, const uint8_t *touch, const ObjBins &bins,
                               int N, double h, const double *o, double tau_out, double tau_in, double deep,
                               float *O, float *f_out, int *err, cudaStream_t st);
// pen: transform min(O, 0) instead of O (the label-aware penetration part).
// conj = false stores F(O) / M^3 (the fixed swept grid of rotate_object).
cudaError_t launch_spectrum(const float *O, int N, int M, int P, double2 *work1, double2 *work2,
                            const double2 *twd, float2 *spec, cudaStream_t st, bool pen = false, bool conj = true);

// Refinement kernels (k_refine.cu)
struct BvhNode {
    float c[3];    // sphere centre (object frame)
    float rad;     // sphere radius
    int32_t left;  // child index, or -1 for a leaf
    int32_t right; // right child, or the leaf's first slot in the triangle order
    int32_t count; // leaf triangle count
    int32_t pad;
};
struct RefineDev {
    const float *Vf;          // V x 3
    const int32_t *T;         // T x 3
    const float *tri_sphere;  // T x 4 (centre, radius), object frame
    const int32_t *tri_order; // leaf slot -> triangle index
    const BvhNode *nodes;
    const PoseRec *poses;
    int P;
    float r, L;
    float tau_out, tau_in, k_slope;
    float A, B, rr;           // Eq. (18) cubic coefficients and the ratio r
    int tri_iters;
};
struct CandF;                 // per-candidate FP32 pose data (k_refine.cu)
size_t cand_bytes();
constexpr int REF_ST = 24;    // doubles of refinement state per candidate
constexpr int REF_NACC = 28;  // accumulated J, grad (6), Gauss-Newton upper triangle (21)
constexpr int REF_WARPS = 4;  // warps per block of the refinement evaluation (one partial sum each)
// hints (optional, K x nblk x 128): each query's witness triangle, read as a
// starting bound and overwritten; -1 = none.
// active (optional, K): candidates whose flag is 0 are skipped.
cudaError_t launch_refine_eval(const RefineDev *Dt, const int32_t *grp, int K, int nblk, const CandF *cands,
                               double *acc_part, bool grad, float *dist_out, float *wit_out, float *nrm_out,
                               cudaStream_t st, int32_t *hints = nullptr, const int32_t *active = nullptr);
// L-BFGS-B refinement (Sec. V-C): LB_ST doubles of solver state per candidate.
constexpr int LB_M = 8;                  // stored (s, y) pairs
constexpr int LB_ST = 32 + 13 * LB_M;
cudaError_t launch_lbfgs(int K, int nblk, double *state, const double *acc_part, const double *prm, double *lbs,
                         int32_t *active, CandF *cands, int phase, cudaStream_t st);
cudaError_t launch_refine_solve(int K, int nblk, double *state, const double *acc_part, const double *prm, int mode,
                                CandF *cands, cudaStream_t st);
cudaError_t launch_set_xi(int B, const float *xi, double *state, cudaStream_t st);
cudaError_t launch_finish_objective(int B, int nblk, const double *state, const double *acc_part, double lam, float *J,
                                    float *grad, const float *gJ, cudaStream_t st);

// Search on library-owned scratch (k_noalloc.cu): limits of that scratch.
constexpr int NOALLOC_MAX_N = 64;        // largest lattice side
constexpr int NOALLOC_MAX_ROT = 4096;    // most rotations per call
constexpr int NOALLOC_MAX_DEVICES = 64;  // device ordinals with a cached scratch address
struct NoallocJob {
    int device;             // current device
    Geo g;
    ReqDev req;             // keys are set by the callee
    const double *c_s;      // device: mean tip of the sweep
    const double *quats;    // host: n unit quaternions
    int n;
    const float2 *tw, *qt;  // device twiddle tables of the canvas side
    cudaStream_t stream;
    dock_peak *peaks;       // host: n peaks out
};
cudaError_t noalloc_search_peaks(const NoallocJob &j);
// Looks up the scratch's device address on `device` (current) once: with
// lazily loaded modules this is where the scratch is placed on the device, so
// dock_create calls it and dock_search_peaks_noalloc itself allocates nothing.
cudaError_t noalloc_prepare(int device);
size_t noalloc_scratch_bytes();

}  // namespace dock
