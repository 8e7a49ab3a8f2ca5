// pft_prep.cu -- input validation, centring, segment/face records, the finalize
// pass (fixed-order FP64 split sum, 1/|Q|^2, translation phase, Q = 0 limit) and
// the FP64 small-|Q| pass.
#include "pft_kernels.cuh"

namespace pft {

namespace {


template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Fixed-order block sum (tree within warps, then warp 0 over the warp sums).
template <int NT>
__device__ double block_sum(double x, double* sh) {
  x = warp_sum(x);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = (lane < NT / 32) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;   // valid in thread 0
}

__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

__device__ __forceinline__ void load_center(const WsHeader* h, int dim, double* c) {
  for (int k = 0; k < dim; ++k)
    c[k] = 0.5 * ((double)ord2f(h->bbox_enc[k]) + (double)ord2f(h->bbox_enc[3 + k]));
}

__global__ void k_init_header(WsHeader* h) {
  uint32_t* w = reinterpret_cast<uint32_t*>(h);
  for (int i = threadIdx.x; i < (int)(sizeof(WsHeader) / 4); i += blockDim.x) w[i] = 0u;
  __syncthreads();
  if (threadIdx.x < 3) h->bbox_enc[threadIdx.x] = 0xffffffffu;   // min slots start above every code
}

template <int D>
__global__ void k_bbox(const float* __restrict__ v, int64_t n, WsHeader* h) {
  float mn[D], mx[D];
#pragma unroll
  for (int c = 0; c < D; ++c) { mn[c] = __int_as_float(0x7f800000); mx[c] = -mn[c]; }
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float x = v[i * D + c];
      if (!isfinite(x)) { bad = true; continue; }
      mn[c] = fminf(mn[c], x);
      mx[c] = fmaxf(mx[c], x);
    }
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
    mn[c] = -warp_max(-mn[c]);
    mx[c] = warp_max(mx[c]);
  }
  const bool any_bad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    for (int c = 0; c < D; ++c) {
      if (mn[c] <= mx[c]) {
        atomicMin(&h->bbox_enc[c], f2ord(mn[c]));
        atomicMax(&h->bbox_enc[3 + c], f2ord(mx[c]));
      }
    }
    if (any_bad) set_status(&h->status, ST_NONFINITE);
  }
}

// 2D: one thread per vertex j builds the segment j -> next(j) of its loop.
template <bool FP64>
__global__ void __launch_bounds__(kPrepThreads) k_prep2d(const float* __restrict__ v, int64_t nv,
                                                         const int64_t* __restrict__ off, int64_t nl, WsHeader* h,
                                                         void* items, double* partials) {
  __shared__ double sh[kPrepThreads / 32];
  const int64_t j = blockIdx.x * (int64_t)kPrepThreads + threadIdx.x;
  double c[2];
  load_center(h, 2, c);
  if (j <= nl) {   // offset validation (one thread per entry)
    bool ok = true;
    if (j == 0) ok = (off[0] == 0);
    if (j == nl) ok = ok && (off[nl] == nv);
    if (j < nl) ok = ok && (off[j] <= off[j + 1]);
    if (!ok) set_status(&h->status, ST_OFFSETS);
  }
  double area = 0.0;
  float rm = 0.0f;
  if (j < nv) {
    // loop l with off[l] <= j < off[l+1]: last l whose start is <= j
    int64_t lo = 0, hi = nl;   // search in off[0..nl-1]
    while (lo + 1 < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (off[mid] <= j) lo = mid; else hi = mid;
    }
    int64_t s0 = off[lo], s1 = off[lo + 1];
    int64_t k = (j + 1 < s1) ? j + 1 : s0;
    if (k < 0 || k >= nv || j < s0 || j >= s1) {
      set_status(&h->status, ST_OFFSETS);
      k = j;
    }
    double x0 = (double)v[2 * j] - c[0], y0 = (double)v[2 * j + 1] - c[1];
    double x1 = (double)v[2 * k] - c[0], y1 = (double)v[2 * k + 1] - c[1];
    double mx = 0.5 * (x0 + x1), my = 0.5 * (y0 + y1), hx = 0.5 * (x1 - x0), hy = 0.5 * (y1 - y0);
    area = 0.5 * (x0 * y1 - x1 * y0);
    rm = __double2float_ru(sqrt(x0 * x0 + y0 * y0));
    if (FP64) {
      reinterpret_cast<Seg64*>(items)[j] = Seg64{mx, my, hx, hy};
    } else {
      reinterpret_cast<Seg32*>(items)[j] =
          Seg32{(float)mx, (float)my, (float)hx, (float)hy};
    }
  }
  double s = block_sum<kPrepThreads>(area, sh);
  float m = warp_max(rm);
  if ((threadIdx.x & 31) == 0) atomicMax(&h->rmax_bits, __float_as_uint(m));
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) { h->center[0] = c[0]; h->center[1] = c[1]; h->center[2] = 0.0; }
}

// 3D: one thread per face.
template <bool FP64>
__global__ void __launch_bounds__(kPrepThreads) k_prep3d(const float* __restrict__ v, int64_t nv,
                                                         const int32_t* __restrict__ f, int64_t nf, WsHeader* h,
                                                         void* items, double* partials, int64_t pair_faces) {
  __shared__ double sh[kPrepThreads / 32];
  const int64_t m = blockIdx.x * (int64_t)kPrepThreads + threadIdx.x;
  double c[3];
  load_center(h, 3, c);
  double vol = 0.0;
  float rm = 0.0f;
  if (m < nf) {
    const int32_t i0 = f[3 * m], i1 = f[3 * m + 1], i2 = f[3 * m + 2];
    double g[3] = {0, 0, 0}, q0[3] = {0, 0, 0}, q1[3] = {0, 0, 0}, N[3] = {0, 0, 0};
    bool paired_ok = true;   // a face of a pair: the pair's first edges must be (a, b) and (b, a)
    if (m < pair_faces) {
      const int64_t a = m & ~(int64_t)1;
      paired_ok = f[3 * a] == f[3 * (a + 1) + 1] && f[3 * a + 1] == f[3 * (a + 1)];
    }
    if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) {
      set_status(&h->status, ST_INDEX);   // the face is skipped (all-zero record contributes 0)
    } else if (!paired_ok) {
      set_status(&h->status, ST_PAIRS);   // both faces of the pair are skipped
    } else {
      double P[3][3];
      const int32_t id[3] = {i0, i1, i2};
      for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) P[k][d] = (double)v[3 * (int64_t)id[k] + d] - c[d];
      for (int d = 0; d < 3; ++d) {
        g[d] = (P[0][d] + P[1][d] + P[2][d]) / 3.0;
        q0[d] = P[0][d] - g[d];
        q1[d] = P[1][d] - g[d];
      }
      double e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
      double e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
      N[0] = e1[1] * e2[2] - e1[2] * e2[1];
      N[1] = e1[2] * e2[0] - e1[0] * e2[2];
      N[2] = e1[0] * e2[1] - e1[1] * e2[0];
      vol = (P[0][0] * (P[1][1] * P[2][2] - P[1][2] * P[2][1]) + P[0][1] * (P[1][2] * P[2][0] - P[1][0] * P[2][2]) +
             P[0][2] * (P[1][0] * P[2][1] - P[1][1] * P[2][0])) / 6.0;
      double r2 = 0.0;
      for (int k = 0; k < 3; ++k) r2 = fmax(r2, P[k][0] * P[k][0] + P[k][1] * P[k][1] + P[k][2] * P[k][2]);
      rm = __double2float_ru(sqrt(r2));
    }
    if (FP64) {
      reinterpret_cast<Face64*>(items)[m] = Face64{g[0], g[1], g[2], q0[0], q0[1], q0[2], q1[0], q1[1], q1[2],
                                                   N[0], N[1], N[2]};
    } else {
      reinterpret_cast<Face32*>(items)[m] =
          Face32{(float)g[0], (float)g[1], (float)g[2],
                 (float)q0[0], (float)q0[1], (float)q0[2], (float)q1[0], (float)q1[1], (float)q1[2],
                 (float)N[0], (float)N[1], (float)N[2]};
    }
  }
  double s = block_sum<kPrepThreads>(vol, sh);
  float mm = warp_max(rm);
  if ((threadIdx.x & 31) == 0) atomicMax(&h->rmax_bits, __float_as_uint(mm));
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) { h->center[0] = c[0]; h->center[1] = c[1]; h->center[2] = c[2]; }
}

// Planar polygon faces (CSR) -> triangles that tile each face with signed areas (exact for
// any planar simple polygon, convex or not), so that the triangle path computes the same
// integral.  The split is by recursive halving: the chain p_i .. p_j closed by its diagonal
// is the triangle (p_i, p_m, p_j), m = (i + j)/2, plus the chains p_i .. p_m and p_m .. p_j,
// starting from p_0 .. p_{n-1}; triangles are numbered in pre-order.  The diagonals' terms
// cancel between neighbouring triangles only up to rounding, and this split keeps their
// total length near perimeter x log2(n) where a fan from p_0 has n - 3 diagonals as long as
// the face (a 65,536-gon's fan loses about 3 decimal digits).
//
// One thread per triangle: triangle t belongs to the face m with off[m] - 2m <= t <
// off[m+1] - 2(m+1), found by bisection, and the pre-order walk from the root finds its
// corners in at most log2(n) + 1 steps.  The first n_faces threads also check the offsets;
// a triangle that would fall outside its face (only with malformed offsets) is written
// degenerate (0, 0, 0), contributes nothing, and sets ST_OFFSETS.
__device__ __forceinline__ void halving_triangle(int64_t n, int64_t t, int64_t& a, int64_t& b, int64_t& c) {
  int64_t i = 0, j = n - 1;
  for (int step = 0; step < 64; ++step) {
    const int64_t m = (i + j) >> 1;
    if (t == 0 || j - i < 2) { a = i; b = m; c = j; return; }
    t -= 1;
    const int64_t nl = m - i - 1 > 0 ? m - i - 1 : 0;   // triangles of the chain i .. m
    if (t < nl) j = m;
    else { t -= nl; i = m; }
  }
  a = b = c = 0;
}

__global__ void k_fan3d(const int32_t* __restrict__ idx, int64_t n_idx, const int64_t* __restrict__ off,
                        int64_t n_faces, int32_t* __restrict__ tris, int64_t n_tris, WsHeader* h) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n_faces) {
    const int64_t a = off[t], b = off[t + 1];
    if (b - a < 3 || (t == 0 && a != 0) || (t == n_faces - 1 && b != n_idx)) set_status(&h->status, ST_OFFSETS);
  }
  if (t >= n_tris) return;
  int64_t lo = 0, hi = n_faces - 1;   // the largest m with off[m] - 2m <= t
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (off[mid] - 2 * mid <= t) lo = mid;
    else hi = mid - 1;
  }
  const int64_t base = off[lo], n = off[lo + 1] - base;
  const int64_t k = t - (base - 2 * lo);          // this face's triangle number, 0 .. n - 3
  int32_t i0 = 0, i1 = 0, i2 = 0;
  if (base >= 0 && n >= 3 && k >= 0 && k < n - 2 && base + n <= n_idx) {
    int64_t a, b, c;
    halving_triangle(n, k, a, b, c);
    i0 = idx[base + a];
    i1 = idx[base + b];
    i2 = idx[base + c];
  } else {
    set_status(&h->status, ST_OFFSETS);
  }
  tris[3 * t] = i0;
  tris[3 * t + 1] = i1;
  tris[3 * t + 2] = i2;
}

// Finalize: out(Q) = exp(iQ.c) * scale / |Q|^2 * sum_splits partial (fixed order, FP64).
__global__ void k_finalize(int dim, const double* __restrict__ q, int64_t n_q, const double2* __restrict__ partial,
                           int ks, int fp64, WsHeader* h, const double* __restrict__ mparts, int nm,
                           int32_t* small_list, double* __restrict__ out, double scale) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_q) return;
  double Q[3] = {0, 0, 0};
  for (int d = 0; d < dim; ++d) {
    double x = q[dim * i + d];
    // the caller's Q: the FP32 pair sums ran at Q rounded to float in coordinates centred on the
    // bounding box, where that moves them by ~1e-7 of |S|; in the phase Q.c the same rounding would
    // move the result by |c| times it, which for a shape far from the origin is not small
    Q[d] = x;
  }
  const double q2 = Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2];
  if (q2 == 0.0) {
    double s = 0.0;
    for (int b = 0; b < nm; ++b) s += mparts[b];
    out[2 * i] = s;
    out[2 * i + 1] = 0.0;
    return;
  }
  const double rmax = (double)__uint_as_float(h->rmax_bits);
  if (sqrt(q2) * rmax < kTauSmallQ) {
    uint32_t slot = atomicAdd(&h->small_q_count, 1u);
    small_list[slot] = (int32_t)i;
    return;
  }
  double re = 0.0, im = 0.0;
  for (int s = 0; s < ks; ++s) {
    double2 p = partial[(int64_t)s * n_q + i];
    re += p.x;
    im += p.y;
  }
  const double k = scale / q2;
  re *= k;
  im *= k;
  const double ph = Q[0] * h->center[0] + Q[1] * h->center[1] + Q[2] * h->center[2];
  double sp, cp;
  sincos(ph, &sp, &cp);
  out[2 * i] = re * cp - im * sp;
  out[2 * i + 1] = re * sp + im * cp;
}

constexpr int kSmallThreads = 256;

// Small |Q|: the integral of exp(iQ.(r - c)) over the signed tetrahedra (c, p0, p1, p2)
// by the simplex series (|Q.(p - c)| < kTauSmallQ, so 16 terms reach FP64 rounding).
__global__ void __launch_bounds__(kSmallThreads) k_smallq3d(const float* __restrict__ v, int64_t nv,
                                                            const int32_t* __restrict__ f, int64_t nf,
                                                            const double* __restrict__ q, int fp64,
                                                            const WsHeader* h, const int32_t* list,
                                                            double* __restrict__ out) {
  __shared__ double sh[kSmallThreads / 32];
  const uint32_t count = h->small_q_count;
  const double c[3] = {h->center[0], h->center[1], h->center[2]};
  for (uint32_t e = blockIdx.x; e < count; e += gridDim.x) {
    const int64_t i = list[e];
    double Q[3];
    for (int d = 0; d < 3; ++d) Q[d] = q[3 * i + d];   // the caller's Q (FP64 series)
    double re = 0.0, im = 0.0;
    for (int64_t m = threadIdx.x; m < nf; m += kSmallThreads) {
      const int32_t id[3] = {f[3 * m], f[3 * m + 1], f[3 * m + 2]};
      if (id[0] < 0 || id[1] < 0 || id[2] < 0 || id[0] >= nv || id[1] >= nv || id[2] >= nv) continue;
      double P[3][3], x[3];
      for (int k = 0; k < 3; ++k) {
        for (int d = 0; d < 3; ++d) P[k][d] = (double)v[3 * (int64_t)id[k] + d] - c[d];
        x[k] = Q[0] * P[k][0] + Q[1] * P[k][1] + Q[2] * P[k][2];
      }
      const double det = P[0][0] * (P[1][1] * P[2][2] - P[1][2] * P[2][1]) +
                         P[0][1] * (P[1][2] * P[2][0] - P[1][0] * P[2][2]) +
                         P[0][2] * (P[1][0] * P[2][1] - P[1][1] * P[2][0]);
      double sr, si;
      simplex_series<3, 3, 16>(x, sr, si);
      re += det * sr;
      im += det * si;
    }
    re = block_sum<kSmallThreads>(re, sh);
    im = block_sum<kSmallThreads>(im, sh);
    if (threadIdx.x == 0) {
      double sp, cp;
      sincos(Q[0] * c[0] + Q[1] * c[1] + Q[2] * c[2], &sp, &cp);
      out[2 * i] = re * cp - im * sp;
      out[2 * i + 1] = re * sp + im * cp;
    }
  }
}

// Small |Q| in 2D: fan of signed triangles (c, p_j, p_{j+1}).
__global__ void __launch_bounds__(kSmallThreads) k_smallq2d(const float* __restrict__ v, int64_t nv,
                                                            const int64_t* __restrict__ off, int64_t nl,
                                                            const double* __restrict__ q, int fp64,
                                                            const WsHeader* h, const int32_t* list,
                                                            double* __restrict__ out) {
  __shared__ double sh[kSmallThreads / 32];
  const uint32_t count = h->small_q_count;
  const double c[2] = {h->center[0], h->center[1]};
  for (uint32_t e = blockIdx.x; e < count; e += gridDim.x) {
    const int64_t i = list[e];
    double Q[2];
    for (int d = 0; d < 2; ++d) Q[d] = q[2 * i + d];   // the caller's Q (FP64 series)
    double re = 0.0, im = 0.0;
    for (int64_t j = threadIdx.x; j < nv; j += kSmallThreads) {
      int64_t lo = 0, hi = nl;
      while (lo + 1 < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= j) lo = mid; else hi = mid;
      }
      int64_t s0 = off[lo], s1 = off[lo + 1];
      int64_t k = (j + 1 < s1) ? j + 1 : s0;
      if (k < 0 || k >= nv) continue;
      const double x0 = (double)v[2 * j] - c[0], y0 = (double)v[2 * j + 1] - c[1];
      const double x1 = (double)v[2 * k] - c[0], y1 = (double)v[2 * k + 1] - c[1];
      const double x[2] = {Q[0] * x0 + Q[1] * y0, Q[0] * x1 + Q[1] * y1};
      double sr, si;
      simplex_series<2, 2, 16>(x, sr, si);
      const double det = x0 * y1 - x1 * y0;
      re += det * sr;
      im += det * si;
    }
    re = block_sum<kSmallThreads>(re, sh);
    im = block_sum<kSmallThreads>(im, sh);
    if (threadIdx.x == 0) {
      double sp, cp;
      sincos(Q[0] * c[0] + Q[1] * c[1], &sp, &cp);
      out[2 * i] = re * cp - im * sp;
      out[2 * i + 1] = re * sp + im * cp;
    }
  }
}

}  // namespace

cudaError_t launch_init_header(WsHeader* h, cudaStream_t st) {
  k_init_header<<<1, 64, 0, st>>>(h);
  return cudaGetLastError();
}

cudaError_t launch_bbox(const float* v, int64_t n, int dim, WsHeader* h, cudaStream_t st) {
  int blocks = (int)std::min<int64_t>(1024, (n + 255) / 256);
  if (blocks < 1) blocks = 1;
  if (dim == 2) k_bbox<2><<<blocks, 256, 0, st>>>(v, n, h);
  else k_bbox<3><<<blocks, 256, 0, st>>>(v, n, h);
  return cudaGetLastError();
}

cudaError_t launch_prep2d(const float* v, int64_t nv, const int64_t* off, int64_t nl, WsHeader* h, void* segs,
                          bool fp64, double* partials, int nblk, cudaStream_t st) {
  // at least enough threads to validate all nl + 1 offsets
  const int need = prep_blocks(std::max<int64_t>(nv, nl + 1));
  if (need != nblk) return cudaErrorInvalidValue;
  if (fp64) k_prep2d<true><<<nblk, kPrepThreads, 0, st>>>(v, nv, off, nl, h, segs, partials);
  else k_prep2d<false><<<nblk, kPrepThreads, 0, st>>>(v, nv, off, nl, h, segs, partials);
  return cudaGetLastError();
}

cudaError_t launch_prep3d(const float* v, int64_t nv, const int32_t* f, int64_t nf, WsHeader* h, void* faces,
                          bool fp64, double* partials, int nblk, cudaStream_t st, int64_t pair_faces) {
  if (fp64) k_prep3d<true><<<nblk, kPrepThreads, 0, st>>>(v, nv, f, nf, h, faces, partials, pair_faces);
  else k_prep3d<false><<<nblk, kPrepThreads, 0, st>>>(v, nv, f, nf, h, faces, partials, pair_faces);
  return cudaGetLastError();
}

cudaError_t launch_fan3d(const int32_t* idx, int64_t n_idx, const int64_t* off, int64_t n_faces, int32_t* tris,
                         int64_t n_tris, WsHeader* h, cudaStream_t st) {
  const int64_t n = std::max(n_tris, n_faces);
  const int64_t blocks = std::max<int64_t>(1, (n + 255) / 256);
  if (blocks > INT32_MAX) return cudaErrorInvalidValue;
  k_fan3d<<<(unsigned)blocks, 256, 0, st>>>(idx, n_idx, off, n_faces, tris, n_tris, h);
  return cudaGetLastError();
}

cudaError_t launch_finalize(int dim, const double* q, int64_t n_q, const double2* partial, int k_splits, bool fp64,
                            WsHeader* h, const double* mparts, int nm, int32_t* small_list, double* out,
                            cudaStream_t st) {
  const int nt = 256;
  const int64_t blocks = (n_q + nt - 1) / nt;
  const double scale = (dim == 2) ? 2.0 : 1.0;   // 2D records hold half edge vectors
  k_finalize<<<(unsigned)blocks, nt, 0, st>>>(dim, q, n_q, partial, k_splits, fp64 ? 1 : 0, h, mparts, nm,
                                               small_list, out, scale);
  return cudaGetLastError();
}

static int small_grid() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

cudaError_t launch_smallq2d(const float* v, int64_t nv, const int64_t* off, int64_t nl, const double* q, bool fp64,
                            const WsHeader* h, const int32_t* list, double* out, cudaStream_t st) {
  k_smallq2d<<<small_grid(), kSmallThreads, 0, st>>>(v, nv, off, nl, q, fp64 ? 1 : 0, h, list, out);
  return cudaGetLastError();
}

cudaError_t launch_smallq3d(const float* v, int64_t nv, const int32_t* f, int64_t nf, const double* q, bool fp64,
                            const WsHeader* h, const int32_t* list, double* out, cudaStream_t st) {
  k_smallq3d<<<small_grid(), kSmallThreads, 0, st>>>(v, nv, f, nf, q, fp64 ? 1 : 0, h, list, out);
  return cudaGetLastError();
}

}  // namespace pft
