// pft_kernels.cuh -- data layouts and kernel declarations of libpft.
#pragma once

#include "pft_common.cuh"

namespace pft {

// ---------------------------------------------------------------------------
// Structure-of-arrays records built by the prep kernels (16-byte multiples so
// that tiles can be moved by cp.async.bulk).  All coordinates are relative to
// the bounding-box centre c of the input; the translation phase exp(iQ.c) is
// applied once per Q in the finalize kernel.
// ---------------------------------------------------------------------------

// 2D segment, FP32: midpoint and half the edge vector.
struct __align__(16) Seg32 {
  float mx, my, hx, hy;
};
// 2D segment, FP64: midpoint and half the edge vector.
struct __align__(16) Seg64 {
  double mx, my, hx, hy;
};
// 3D triangle, FP32: centroid, the first two corners relative to the centroid
// (the third is -(q0 + q1)), and N = (p1 - p0) x (p2 - p0).
struct __align__(16) Face32 {
  float gx, gy, gz, q0x, q0y, q0z, q1x, q1y, q1z, nx, ny, nz;
};
// 3D triangle, FP64: centroid, corners 0 and 1 relative to it, N.
struct __align__(16) Face64 {
  double gx, gy, gz, q0x, q0y, q0z, q1x, q1y, q1z, nx, ny, nz;
};
static_assert(sizeof(Seg32) == 16 && sizeof(Seg64) == 32, "segment record sizes");
static_assert(sizeof(Face32) == 48 && sizeof(Face64) == 96, "face record sizes");

// Threshold on |Q| * max|r - c| below which the FP64 small-|Q| pass replaces the
// boundary sum (which cancels to O(|Q|^2 R^2) of its terms there).
constexpr double kTauSmallQ = 0.25;

// sum_k i^k h_k(x) / (k + p)! for the n nodes x (FP64), K terms: the integral of exp(i Q.r)
// over a simplex divided by p! times its volume, from its corner phases x (small-|Q| passes).
template <int N, int P, int K>
__device__ __forceinline__ void simplex_series(const double* x, double& re, double& im) {
  double h[K + 1];
  h[0] = 1.0;
#pragma unroll
  for (int k = 1; k <= K; ++k) h[k] = 0.0;
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int k = 1; k <= K; ++k) h[k] = fma(x[j], h[k - 1], h[k]);
  double inv = 1.0;
#pragma unroll
  for (int k = 2; k <= P; ++k) inv /= (double)k;   // 1/P!
  re = 0.0;
  im = 0.0;
#pragma unroll
  for (int k = 0; k <= K; ++k) {
    const double t = h[k] * inv;
    switch (k & 3) { case 0: re += t; break; case 1: im += t; break; case 2: re -= t; break; default: im -= t; }
    inv /= (double)(k + P + 1);
  }
}

// Launch description computed on the host.
struct FwdLaunch {
  int r;              // Q points per thread
  int nt;             // threads per block
  int64_t q_tiles;    // blocks along x
  int k_splits;       // blocks along y (segment/face chunks)
  int64_t per_split;  // items per chunk (multiple of the tile)
};

// Host-side launchers (defined in pft_fwd.cu).  Each returns cudaSuccess or the launch error.
cudaError_t launch_init_header(WsHeader* h, cudaStream_t st);
cudaError_t launch_bbox(const float* v, int64_t n, int dim, WsHeader* h, cudaStream_t st);
cudaError_t launch_prep2d(const float* v, int64_t nv, const int64_t* off, int64_t nl, WsHeader* h,
                          void* segs, bool fp64, double* partials, int nblk, cudaStream_t st);
// pair_faces: the faces [0, pair_faces) come in pairs (2k, 2k+1) that share their first edge in
// opposite directions (face_pairs option); k_prep3d checks them, k_fwd shares the edge's sinc.
cudaError_t launch_prep3d(const float* v, int64_t nv, const int32_t* f, int64_t nf, WsHeader* h,
                          void* faces, bool fp64, double* partials, int nblk, cudaStream_t st,
                          int64_t pair_faces = 0);
// qperm: NULL, or the slot -> Q index map of launch_qorder (the kernel reads Q point qperm[slot]
// and writes its partial sums at that index).
cudaError_t launch_fwd(int dim, bool fp64, const FwdLaunch& L, const void* items, int64_t n_items,
                       const double* q, int64_t n_q, float tau, double2* partial, uint32_t* status,
                       cudaStream_t st, int64_t pair_faces = 0, const int32_t* qperm = nullptr);
cudaError_t launch_fan3d(const int32_t* idx, int64_t n_idx, const int64_t* off, int64_t n_faces, int32_t* tris,
                         int64_t n_tris, WsHeader* h, cudaStream_t st);
cudaError_t launch_finalize(int dim, const double* q, int64_t n_q, const double2* partial, int k_splits,
                            bool fp64, WsHeader* h, const double* measure_partials, int n_measure,
                            int32_t* small_list, double* out, cudaStream_t st);
cudaError_t launch_smallq2d(const float* v, int64_t nv, const int64_t* off, int64_t nl, const double* q, bool fp64,
                            const WsHeader* h, const int32_t* small_list, double* out, cudaStream_t st);
cudaError_t launch_smallq3d(const float* v, int64_t nv, const int32_t* f, int64_t nf, const double* q, bool fp64,
                            const WsHeader* h, const int32_t* small_list, double* out, cudaStream_t st);

// Prep blocks used for the per-block FP64 area/volume partial sums.
constexpr int kPrepThreads = 256;
inline int prep_blocks(int64_t n) { return (int)((n + kPrepThreads - 1) / kPrepThreads); }

// Q order (pft_qorder.cu): a slot -> Q index map that puts Q points close together in Q space
// into the same group of 32 threads of a pair kernel with r Q points per thread and nt threads
// per block.  Scratch regions (byte offsets from the scratch base, 256-byte aligned):
struct QOrderLayout {
  size_t box, keys0, keys1, vals0, vals1, hist, tot, total;
  int64_t nb, nh, nt;   // sort blocks, histogram length, scan blocks
};
QOrderLayout qorder_layout(int64_t n_q);
// Whether a call with n_q Q points and n_items segments or faces orders its Q points.
bool qorder_wanted(int64_t n_q, int64_t n_items, int r, int nt);
// perm[n_q] <- the map; q is [n_q x dim] FP64 on the device; adds its launches to *launches.
cudaError_t launch_qorder(int dim, const double* q, int64_t n_q, int r, int nt, void* scratch, int32_t* perm,
                          cudaStream_t st, int* launches);

// Occupancy query for the main kernel of a configuration (blocks per SM).
int fwd_blocks_per_sm(int dim, bool fp64, int r, int nt, bool pairs = false);
int fwd_tile(int dim, bool fp64);

}  // namespace pft
