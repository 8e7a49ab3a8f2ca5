// pft_fwd.cu -- the hot loop: every (Q, segment) or (Q, face) pair of the
// divergence-theorem sum.
//
// Mapping: each thread owns R Q points in registers; a block covers NT*R Q
// points and one chunk of the segments/faces (blockIdx.y, split-K).  Segment or
// face records stream through shared memory in tiles moved by bulk copies
// (cp.async.bulk, TMA) into a STAGES-deep ring guarded by mbarriers; one thread
// issues the copies, every thread reads each record as a broadcast.  Sums are
// per thread and in a fixed order: FP32 within a tile, error-free (TwoSum)
// compensation across tiles; the per-chunk partials are added in FP64 by the
// finalize kernel.  No atomics on data, so results are deterministic.
#include "pft_pairs.cuh"

namespace pft {
namespace {

// ---------------------------------------------------------------------------
// The main kernel: bulk-copy ring of record tiles, R Q points per thread.
//
// Ring protocol (no block-wide barrier inside the loop): full[s] completes when
// the bulk copy of the tile in slot s has landed (expect_tx by the issuing
// thread).  When a warp has finished reading slot s its lane 0 increments
// done[s]; the warp that brings the count to the number of warps resets it and
// issues the copy of the tile kStages further on into the same slot.  So no
// warp ever waits for a particular other warp: the slowest warp gates a slot's
// refill, and the others may run up to kStages - 1 tiles ahead.  Every wait is
// bounded and every stop decision is warp-uniform; a wait that gives up sets
// ST_TIMEOUT and the block stops early, after letting copies in flight land.
// ---------------------------------------------------------------------------
template <class Pol, int R, int NT>
__global__ void __launch_bounds__(NT, kMinBlocks<Pol, R, NT>) k_fwd(const typename Pol::Item* __restrict__ items, int64_t n_items,
                                            int64_t per_split, const double* __restrict__ q, int64_t n_q,
                                            Thr th, double2* __restrict__ partial, uint32_t* status,
                                            const int32_t* __restrict__ qperm) {
  using Item = typename Pol::Item;
  using QT = typename Pol::QT;
  constexpr int TILE = Pol::kTile;
  constexpr int D = Pol::kDim;
  constexpr int NW = NT / 32;
  __shared__ __align__(128) Item ring[kStages * TILE];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ int done[kStages];
  __shared__ int issued;

  const int64_t i0 = (int64_t)blockIdx.y * per_split;
  const int64_t n = max((int64_t)0, min(per_split, n_items - i0));
  const int ntiles = (int)((n + TILE - 1) / TILE);
  const Item* src = items + i0;

  // slot qbase + r NT holds Q point qperm[slot] (the caller's index; without qperm the slot itself)
  QT qr[R][3];
  const int64_t qbase = (int64_t)blockIdx.x * (NT * R) + threadIdx.x;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t iq = qbase + (int64_t)r * NT;
#pragma unroll
    for (int d = 0; d < 3; ++d) qr[r][d] = (QT)0;
    if (iq < n_q) {
      const int64_t src = qperm ? (int64_t)qperm[iq] : iq;
#pragma unroll
      for (int d = 0; d < D; ++d) qr[r][d] = (QT)q[src * D + d];
    }
  }
  typename Pol::template Acc<R> acc;
  acc.init();

  auto issue = [&](int t) {
    const int s = t % kStages;
    const int64_t cnt = min((int64_t)TILE, n - (int64_t)t * TILE);
    const uint32_t bytes = (uint32_t)(cnt * (int64_t)sizeof(Item));
    mbar_arrive_expect_tx(&full[s], bytes);
    bulk_g2s(ring + s * TILE, src + (int64_t)t * TILE, bytes, &full[s]);
    atomicAdd(&issued, 1);
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      done[s] = 0;
    }
    issued = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int t = 0; t < min(kStages, ntiles); ++t) issue(t);

  bool ok = true;
  for (int t = 0; t < ntiles; ++t) {
    const int s = t % kStages;
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[s], (uint32_t)((t / kStages) & 1)))) { ok = false; break; }
    const int cnt = (int)min((int64_t)TILE, n - (int64_t)t * TILE);
    Pol::template tile<R>(ring + s * TILE, cnt, qr, acc, th, i0 + (int64_t)t * TILE);
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
      __threadfence_block();                       // this warp's reads of slot s come first
      if (atomicAdd(&done[s], 1) == NW - 1) {      // last warp out of slot s refills it
        atomicExch(&done[s], 0);
        if (t + kStages < ntiles) {
          fence_proxy_async_smem();
          issue(t + kStages);
        }
      }
    }
  }
  if (!ok) set_status(status, ST_TIMEOUT);
  __syncthreads();   // reached by every thread: stop decisions above are per warp, never inside a warp
  if (threadIdx.x == 0) {   // no copy may still be writing into the ring when the block exits
    const int m = issued;
    for (int u = max(0, m - kStages); u < m; ++u)
      (void)mbar_wait_bounded(&full[u % kStages], (uint32_t)((u / kStages) & 1));
  }
  if (!ok) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t iq = qbase + (int64_t)r * NT;
    if (iq < n_q) partial[(int64_t)blockIdx.y * n_q + (qperm ? (int64_t)qperm[iq] : iq)] = acc.get(r);
  }
}

template <class Pol, int R, int NT>
cudaError_t launch_one(const FwdLaunch& L, const void* items, int64_t n_items, const double* q, int64_t n_q,
                       Thr th, double2* partial, uint32_t* status, cudaStream_t st, const int32_t* qperm) {
  dim3 grid((unsigned)L.q_tiles, (unsigned)L.k_splits);
  k_fwd<Pol, R, NT><<<grid, NT, 0, st>>>(static_cast<const typename Pol::Item*>(items), n_items, L.per_split, q,
                                         n_q, th, partial, status, qperm);
  return cudaGetLastError();
}

template <class Pol, int R, int NT>
int occupancy_one() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fwd<Pol, R, NT>, NT, 0) != cudaSuccess) return 1;
  return b > 0 ? b : 1;
}

// Dispatch over the instantiated configurations (FP64 paths keep R <= 2).
template <class Pol, class F>
cudaError_t dispatch(int r, int nt, F&& f) {
  constexpr bool kBig = sizeof(typename Pol::QT) == 4;
#define PFT_CASE(RR, NN) \
  if (r == RR && nt == NN) return f.template operator()<Pol, RR, NN>();
  PFT_CASE(1, 128) PFT_CASE(2, 128) PFT_CASE(1, 256) PFT_CASE(2, 256)
  if constexpr (kBig) {
    PFT_CASE(4, 128) PFT_CASE(8, 128) PFT_CASE(4, 256) PFT_CASE(8, 256)
  }
#undef PFT_CASE
  return cudaErrorInvalidConfiguration;
}

// The paired-face policy: the FP32 launch shapes with R <= 4.
template <class F>
cudaError_t dispatch_pairs(int r, int nt, F&& f) {
#define PFT_CASE(RR, NN) \
  if (r == RR && nt == NN) return f.template operator()<Pol3F32Pair, RR, NN>();
  PFT_CASE(1, 128) PFT_CASE(2, 128) PFT_CASE(4, 128) PFT_CASE(1, 256) PFT_CASE(2, 256) PFT_CASE(4, 256)
#undef PFT_CASE
  return cudaErrorInvalidConfiguration;
}

struct LaunchF {
  const FwdLaunch& L; const void* items; int64_t n_items; const double* q; int64_t n_q; Thr th;
  double2* partial; uint32_t* status; cudaStream_t st; const int32_t* qperm;
  template <class Pol, int R, int NT>
  cudaError_t operator()() const {
    return launch_one<Pol, R, NT>(L, items, n_items, q, n_q, th, partial, status, st, qperm);
  }
};

struct OccF {
  int* out;
  template <class Pol, int R, int NT>
  cudaError_t operator()() const { *out = occupancy_one<Pol, R, NT>(); return cudaSuccess; }
};

}  // namespace

cudaError_t launch_fwd(int dim, bool fp64, const FwdLaunch& L, const void* items, int64_t n_items, const double* q,
                       int64_t n_q, float tau, double2* partial, uint32_t* status, cudaStream_t st,
                       int64_t pair_faces, const int32_t* qperm) {
  // the FP64 path keeps its series (through k = 16) for P < 9/4, where it truncates below 1e-14
  if (fp64) tau = fminf(tau, 3.0f);
  const float tau_lo = fminf(tau, kTauLo);
  const Thr th{0.25f * tau * tau, 0.25f * tau_lo * tau_lo, tau > 1.0f ? 1 : 0, tau > 3.0f ? 1 : 0,
               dim == 3 && !fp64 ? pair_faces : 0};
  LaunchF f{L, items, n_items, q, n_q, th, partial, status, st, qperm};
  if (dim == 2) return fp64 ? dispatch<Pol2F64>(L.r, L.nt, f) : dispatch<Pol2F32>(L.r, L.nt, f);
  if (!fp64 && th.pair_end > 0) return dispatch_pairs(L.r, L.nt, f);
  return fp64 ? dispatch<Pol3F64>(L.r, L.nt, f) : dispatch<Pol3F32>(L.r, L.nt, f);
}

int fwd_blocks_per_sm(int dim, bool fp64, int r, int nt, bool pairs) {
  int b = 1;
  OccF f{&b};
  cudaError_t e;
  if (dim == 2) e = fp64 ? dispatch<Pol2F64>(r, nt, f) : dispatch<Pol2F32>(r, nt, f);
  else if (!fp64 && pairs) e = dispatch_pairs(r, nt, f);
  else e = fp64 ? dispatch<Pol3F64>(r, nt, f) : dispatch<Pol3F32>(r, nt, f);
  return e == cudaSuccess ? b : 1;
}

int fwd_tile(int dim, bool fp64) {
  if (dim == 2) return fp64 ? Pol2F64::kTile : Pol2F32::kTile;
  return fp64 ? Pol3F64::kTile : Pol3F32::kTile;
}

}  // namespace pft
