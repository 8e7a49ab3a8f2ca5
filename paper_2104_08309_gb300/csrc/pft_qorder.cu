// pft_qorder.cu -- the order in which the pair kernels visit the Q points.
//
// The pair kernels take some decisions once per group of 32 threads: the 3D face
// term's form (a series whose length depends on the largest phase spread P of the
// group's Q points, or the edge sum), and in 2D whether the SFU sinc runs at all.
// A group holds R Q points per thread at the slots base + r*NT + 32*w + lane of
// the Q array, so the cost of a group follows the largest |Q| and the spread of
// directions among those 32 R points.  Here the Q points are sorted along a
// Z-order (Morton) curve of their coordinates, quantised over the bounding box of
// the Q set (10 bits per axis in 3D, 16 in 2D), by a stable least-significant-digit
// radix sort (four passes of 8 bits; ties keep the caller's order, so the result is
// deterministic), and each run of 32 R consecutive sorted points is dealt to the
// slots of one group.  The pair kernel reads Q through the resulting slot -> Q index
// map and writes each Q's partial sums at the caller's index, so the finishing
// kernels and the outputs keep the caller's order.
#include <algorithm>

#include "pft_kernels.cuh"

namespace pft {
namespace {

constexpr int kST = 256;          // threads per block of the sort kernels
constexpr int kSK = 4;            // keys per thread
constexpr int kSB = kST * kSK;    // keys per block
constexpr int kBins = 256;        // 8-bit digits
static_assert(kBins == kST, "one digit per thread in the scatter's offset pass");

inline size_t al(size_t x) { return (x + 255) / 256 * 256; }

__global__ void k_qbox_init(uint32_t* box) {
  if (threadIdx.x < 3) {
    box[threadIdx.x] = 0xffffffffu;   // min of the order-preserving codes
    box[3 + threadIdx.x] = 0u;        // max
  }
}

// Bounding box of the Q points as rounded to FP32 (what the pair kernels use); NaN is skipped.
template <int D>
__global__ void __launch_bounds__(kST) k_qbox(const double* __restrict__ q, int64_t n, uint32_t* box) {
  uint32_t lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
  for (int64_t i = (int64_t)blockIdx.x * kST + threadIdx.x; i < n; i += (int64_t)gridDim.x * kST) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const float x = (float)q[i * D + d];
      if (x == x) {
        const uint32_t u = f2ord(x);
        lo[d] = min(lo[d], u);
        hi[d] = max(hi[d], u);
      }
    }
  }
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const uint32_t l = __reduce_min_sync(0xffffffffu, lo[d]), h = __reduce_max_sync(0xffffffffu, hi[d]);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&box[d], l);
      atomicMax(&box[3 + d], h);
    }
  }
}

// The low 10 (3D) or 16 (2D) bits of x moved to every third or every other bit.
__device__ __forceinline__ uint32_t spread3(uint32_t x) {
  x &= 0x3ffu;
  x = (x | (x << 16)) & 0x030000ffu;
  x = (x | (x << 8)) & 0x0300f00fu;
  x = (x | (x << 4)) & 0x030c30c3u;
  x = (x | (x << 2)) & 0x09249249u;
  return x;
}
__device__ __forceinline__ uint32_t spread2(uint32_t x) {
  x &= 0xffffu;
  x = (x | (x << 8)) & 0x00ff00ffu;
  x = (x | (x << 4)) & 0x0f0f0f0fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

// Morton key of each Q point (coordinate d's bits at positions d, d + D, d + 2D, ...) and its index.
template <int D>
__global__ void __launch_bounds__(kST) k_qkeys(const double* __restrict__ q, int64_t n, const uint32_t* __restrict__ box,
                                               uint32_t* __restrict__ keys, int32_t* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * kST + threadIdx.x;
  if (i >= n) return;
  constexpr int kBits = D == 3 ? 10 : 16;
  const float levels = (float)(1u << kBits);
  uint32_t key = 0u;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const float lo = ord2f(box[d]), hi = ord2f(box[3 + d]);
    const float t = (hi > lo) ? ((float)q[i * D + d] - lo) / (hi - lo) : 0.f;
    const uint32_t c = (t > 0.f) ? (uint32_t)fminf(t * levels, levels - 1.f) : 0u;   // NaN and t <= 0: 0
    key |= (D == 3 ? spread3(c) : spread2(c)) << d;
  }
  keys[i] = key;
  vals[i] = (int32_t)i;
}

// Digit counts of block b's kSB keys: hist[digit * nb + b] (digit-major, so that one exclusive
// scan gives every (digit, block) its first output position).
__global__ void __launch_bounds__(kST) k_rhist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                               uint32_t* __restrict__ hist, int64_t nb) {
  __shared__ uint32_t c[kBins];
  c[threadIdx.x] = 0u;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSB;
#pragma unroll
  for (int k = 0; k < kSK; ++k) {
    const int64_t i = base + (int64_t)k * kST + threadIdx.x;
    if (i < n) atomicAdd(&c[(keys[i] >> shift) & 0xffu], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nb + blockIdx.x] = c[threadIdx.x];
}

// Exclusive scan of a[0, m) in place, in three steps: per block of kSB values (block totals to
// tot), the totals (one block, in order), the block offsets added back.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* sh, uint32_t& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t s = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= o) s += y;
  }
  if (lane == 31) sh[w] = s;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < kST / 32 ? sh[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kST / 32) sh[lane] = t;
  }
  __syncthreads();
  total = sh[kST / 32 - 1];
  const uint32_t before = (w > 0 ? sh[w - 1] : 0u) + s - x;
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(kST) k_scan_a(uint32_t* __restrict__ a, int64_t m, uint32_t* __restrict__ tot) {
  __shared__ uint32_t sh[kST / 32];
  const int64_t base = (int64_t)blockIdx.x * kSB + (int64_t)threadIdx.x * kSK;
  uint32_t v[kSK], sum = 0u;
#pragma unroll
  for (int k = 0; k < kSK; ++k) {
    v[k] = base + k < m ? a[base + k] : 0u;
    sum += v[k];
  }
  uint32_t total;
  uint32_t run = block_excl_scan(sum, sh, total);
#pragma unroll
  for (int k = 0; k < kSK; ++k) {
    if (base + k < m) a[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kST) k_scan_b(uint32_t* __restrict__ tot, int64_t mt) {
  __shared__ uint32_t sh[kST / 32];
  uint32_t carry = 0u;
  for (int64_t b0 = 0; b0 < mt; b0 += kST) {   // uniform trip count over the block
    const int64_t i = b0 + threadIdx.x;
    const uint32_t x = i < mt ? tot[i] : 0u;
    uint32_t total;
    const uint32_t before = block_excl_scan(x, sh, total);
    if (i < mt) tot[i] = carry + before;
    carry += total;
  }
}

__global__ void __launch_bounds__(kST) k_scan_c(uint32_t* __restrict__ a, int64_t m, const uint32_t* __restrict__ tot) {
  const int64_t base = (int64_t)blockIdx.x * kSB + (int64_t)threadIdx.x * kSK;
  const uint32_t add = tot[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kSK; ++k)
    if (base + k < m) a[base + k] += add;
}

// Stable scatter of block b's keys by digit.  The keys go in kSK rounds of kST (round k holds
// keys base + k kST + tid), so that within a round the input order is (warp, lane): a key's
// position is its digit's running offset for this block, plus the counts of that digit in the
// round's earlier warps, plus its rank among the lanes of its own warp with the same digit.
__global__ void __launch_bounds__(kST) k_rscatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                                  int64_t n, int shift, const uint32_t* __restrict__ hist, int64_t nb,
                                                  uint32_t* __restrict__ kout, int32_t* __restrict__ vout) {
  __shared__ uint32_t run[kBins];
  __shared__ uint32_t wc[kST / 32][kBins + 1];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  run[tid] = hist[(int64_t)tid * nb + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kSB;
  for (int k = 0; k < kSK; ++k) {
#pragma unroll
    for (int j = 0; j < kST / 32; ++j) wc[j][tid] = 0u;
    __syncthreads();
    const int64_t i = base + (int64_t)k * kST + tid;
    const bool valid = i < n;
    const uint32_t key = valid ? kin[i] : 0u;
    const int32_t val = valid ? vin[i] : 0;
    const uint32_t d = valid ? ((key >> shift) & 0xffu) : (uint32_t)kBins;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0u) wc[w][d] = __popc(peers);
    __syncthreads();
    {   // digit tid: offsets of the warps' runs, in warp order
      uint32_t r = run[tid];
#pragma unroll
      for (int j = 0; j < kST / 32; ++j) {
        const uint32_t c = wc[j][tid];
        wc[j][tid] = r;
        r += c;
      }
      run[tid] = r;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = wc[w][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
  }
}

// Sorted position p -> slot.  In whole blocks of r nt slots, run g = p / (32 r) of the sorted
// points goes to group w = g mod (nt/32) of block g / (nt/32), its element o = p mod (32 r) to the
// slot of point o / 32 of lane o mod 32; the ragged last block keeps the sorted order.
__global__ void __launch_bounds__(kST) k_qslots(const int32_t* __restrict__ vals, int64_t n, int r, int nt,
                                                int32_t* __restrict__ perm) {
  const int64_t p = (int64_t)blockIdx.x * kST + threadIdx.x;
  if (p >= n) return;
  const int64_t per_block = (int64_t)r * nt, full = n / per_block * per_block;
  int64_t slot = p;
  if (p < full) {
    const int64_t g = p / (32 * r), o = p % (32 * r), wpb = nt / 32;
    slot = (g / wpb) * per_block + (o / 32) * nt + (g % wpb) * 32 + (o % 32);
  }
  perm[slot] = vals[p];
}

}  // namespace

QOrderLayout qorder_layout(int64_t n_q) {
  QOrderLayout y{};
  const int64_t n = n_q > 0 ? n_q : 1;
  y.nb = (n + kSB - 1) / kSB;
  y.nh = (int64_t)kBins * y.nb;
  y.nt = (y.nh + kSB - 1) / kSB;
  size_t o = 0;
  y.box = o;   o = al(o + 6 * sizeof(uint32_t));
  y.keys0 = o; o = al(o + sizeof(uint32_t) * (size_t)n);
  y.keys1 = o; o = al(o + sizeof(uint32_t) * (size_t)n);
  y.vals0 = o; o = al(o + sizeof(int32_t) * (size_t)n);
  y.vals1 = o; o = al(o + sizeof(int32_t) * (size_t)n);
  y.hist = o;  o = al(o + sizeof(uint32_t) * (size_t)y.nh);
  y.tot = o;   o = al(o + sizeof(uint32_t) * (size_t)y.nt);
  y.total = o;
  return y;
}

bool qorder_wanted(int64_t n_q, int64_t n_items, int r, int nt) {
  // at least two blocks' worth of Q points to group, and enough pairs (~1e9) that the ordering's
  // two dozen small launches are a negligible part of the call
  return n_q >= 2 * (int64_t)r * nt && (double)n_q * (double)n_items >= 1073741824.0;
}

cudaError_t launch_qorder(int dim, const double* q, int64_t n_q, int r, int nt, void* scratch, int32_t* perm,
                          cudaStream_t st, int* launches) {
  const QOrderLayout y = qorder_layout(n_q);
  char* s = static_cast<char*>(scratch);
  uint32_t* box = reinterpret_cast<uint32_t*>(s + y.box);
  uint32_t* keys[2] = {reinterpret_cast<uint32_t*>(s + y.keys0), reinterpret_cast<uint32_t*>(s + y.keys1)};
  int32_t* vals[2] = {reinterpret_cast<int32_t*>(s + y.vals0), reinterpret_cast<int32_t*>(s + y.vals1)};
  uint32_t* hist = reinterpret_cast<uint32_t*>(s + y.hist);
  uint32_t* tot = reinterpret_cast<uint32_t*>(s + y.tot);
  const unsigned g1 = (unsigned)((n_q + kST - 1) / kST);
  const unsigned gbox = (unsigned)std::min<int64_t>(y.nb, 1024);
  int nl = 0;
  cudaError_t e;
#define PFT_Q(expr)                                 \
  do {                                              \
    expr;                                           \
    if ((e = cudaGetLastError()) != cudaSuccess) return e; \
    ++nl;                                           \
    if (launches) ++*launches;                      \
  } while (0)
  PFT_Q((k_qbox_init<<<1, 32, 0, st>>>(box)));
  if (dim == 3) {
    PFT_Q((k_qbox<3><<<gbox, kST, 0, st>>>(q, n_q, box)));
    PFT_Q((k_qkeys<3><<<g1, kST, 0, st>>>(q, n_q, box, keys[0], vals[0])));
  } else {
    PFT_Q((k_qbox<2><<<gbox, kST, 0, st>>>(q, n_q, box)));
    PFT_Q((k_qkeys<2><<<g1, kST, 0, st>>>(q, n_q, box, keys[0], vals[0])));
  }
  int cur = 0;
  for (int shift = 0; shift < 32; shift += 8) {
    PFT_Q((k_rhist<<<(unsigned)y.nb, kST, 0, st>>>(keys[cur], n_q, shift, hist, y.nb)));
    PFT_Q((k_scan_a<<<(unsigned)y.nt, kST, 0, st>>>(hist, y.nh, tot)));
    PFT_Q((k_scan_b<<<1, kST, 0, st>>>(tot, y.nt)));
    PFT_Q((k_scan_c<<<(unsigned)y.nt, kST, 0, st>>>(hist, y.nh, tot)));
    PFT_Q((k_rscatter<<<(unsigned)y.nb, kST, 0, st>>>(keys[cur], vals[cur], n_q, shift, hist, y.nb, keys[1 - cur],
                                                      vals[1 - cur])));
    cur = 1 - cur;
  }
  PFT_Q((k_qslots<<<g1, kST, 0, st>>>(vals[cur], n_q, r, nt, perm)));
#undef PFT_Q
  (void)nl;
  return cudaSuccess;
}

}  // namespace pft
