// pft_batched.cu -- many polygons (2D) or closed triangle meshes (3D) in one
// persistent launch.
//
// Host (pft2d_batched_prepare / pft3d_batched_prepare): every shape i is cut into
// work items (shape, chunk of segments or faces, Q tile) whose cost is items x Q
// points (+ a fixed per-item charge for the finalize arithmetic).  Items are sorted by cost and
// dealt to the G = SMs x resident-blocks persistent blocks, each to the least
// loaded one so far (longest-processing-time first); every block gets a fixed
// list, so the schedule, and with it every floating-point sum, is the same on
// every call.  The plan is copied once into the workspace.
//
// Device (pft2d_polygons_batched / pft3d_meshes_batched, kernels only, so a CUDA
// graph can capture and replay it): k_bprep / k_bprep3 build per-shape centres,
// areas or volumes and segment or face records; k_batched walks each block's
// item list with the same bulk-copy ring as the single-shape kernel (the tile
// stream runs across item boundaries) and finishes single-chunk shapes in
// place; k_bfinal adds the chunk partials of multi-chunk shapes; k_bsmall /
// k_bsmall3 redo points with |Q| R < 0.25 in FP64.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <queue>
#include <vector>

#include "pft_pairs.cuh"

namespace pft {
namespace {

constexpr uint64_t kPlanMagic = 0x706674626174636bULL;   // "pftbatck"
constexpr int64_t kChunk = 4096;                          // segments or faces per item at most
constexpr int kBThreads = 256;                            // prep / finalize block size
constexpr double kTwoPiD = 6.283185307179586477;          // 2 pi (FP64)
constexpr double kInvTwoPiD = 0.1591549430918953358;      // 1 / (2 pi) (FP64)

struct BPlanHeader {
  uint64_t magic;
  int64_t n_polys, n_verts, n_q, n_items, n_cta, n_mc, part_rows, n_out;   // n_verts: segments or faces
  int32_t r, nt, shared_q, fp64, dim;
  float tau;
  int32_t q_tiled, pad1;   // q_tiled: the pair kernel visits the shared Q set in the library's order
  uint8_t pad[256 - 8 * 9 - 4 * 8];
};
static_assert(sizeof(BPlanHeader) == 256, "plan header is 256 bytes");

struct PolyPlan {       // per shape; "seg" counts segments (2D) or faces (3D)
  int64_t seg_begin, q_begin, out_base, part_base;
  int32_t n_seg, n_q, n_chunks, pad;
};
struct BItem {          // per work item
  int32_t poly, chunk, qtile, pad;
};
struct PolyInfo {       // written by k_bprep / k_bprep3: centre, area or volume, max radius
  double cx, cy, cz, measure;
  float rmax;
  uint32_t pad;
};

struct BLayout {
  size_t plan_hdr, cta_off, items, pplan, mc, info, segs, partial, small, qperm, qscratch, qlo, total;
};

inline size_t al(size_t x) { return (x + 255) / 256 * 256; }
// q - (float)q per Q coordinate (FP32 policies): the FP32 finish's phase Q.c takes the caller's Q
inline size_t qlo_bytes(int64_t dim, int64_t n_q) { return sizeof(float) * (size_t)dim * (size_t)std::max<int64_t>(n_q, 1); }

BLayout layout(int dim, int64_t n_polys, int64_t n_verts, int64_t n_items, int64_t n_cta, int64_t n_mc,
               int64_t part_rows, int64_t n_out, bool fp64, int64_t n_q, bool q_tiled) {
  const size_t rec = dim == 2 ? (fp64 ? sizeof(Seg64) : sizeof(Seg32)) : (fp64 ? sizeof(Face64) : sizeof(Face32));
  BLayout y{};
  size_t o = al(sizeof(WsHeader));
  y.plan_hdr = o; o = al(o + sizeof(BPlanHeader));
  y.cta_off = o;  o = al(o + sizeof(int32_t) * (size_t)(n_cta + 1));
  y.items = o;    o = al(o + sizeof(BItem) * (size_t)std::max<int64_t>(n_items, 1));
  y.pplan = o;    o = al(o + sizeof(PolyPlan) * (size_t)std::max<int64_t>(n_polys, 1));
  y.mc = o;       o = al(o + sizeof(int32_t) * (size_t)std::max<int64_t>(n_mc, 1));
  y.info = o;     o = al(o + sizeof(PolyInfo) * (size_t)std::max<int64_t>(n_polys, 1));
  y.segs = o;     o = al(o + rec * (size_t)std::max<int64_t>(n_verts, 1));
  y.partial = o;  o = al(o + sizeof(double2) * (size_t)std::max<int64_t>(part_rows, 1));
  y.small = o;    o = al(o + sizeof(uint32_t) * (size_t)std::max<int64_t>(n_out, 1));
  if (q_tiled) {
    y.qperm = o;    o = al(o + sizeof(int32_t) * (size_t)n_q);
    y.qscratch = o; o = al(o + qorder_layout(n_q).total);
  }
  if (!fp64) {   // the last region, so that its offset follows from the total: the low parts of Q
    y.qlo = o;  o = al(o + qlo_bytes(dim, n_q));
  }
  y.total = o;
  return y;
}

template <typename T>
T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

// ---------------------------------------------------------------------------
// Host plan.
// ---------------------------------------------------------------------------
struct HostPlan {
  BPlanHeader h{};
  std::vector<int32_t> cta_off;
  std::vector<BItem> items;
  std::vector<PolyPlan> pplan;
  std::vector<int32_t> mc;
};

bool batched_config(int dim, bool fp64, int r, int nt);

// Default launch shape: one block of 512 threads per SM on a shared Q set that fills its Q tiles
// (r x 512 points or more), else blocks of 128.  Two or more resident blocks of the persistent
// kernel do not share an SM evenly (the warps of the block that started first keep the issue
// priority), so with a static schedule the later blocks ran up to a third longer than the first
// ones while the SM sat half empty; the warps of one block walk the same tile ring and finish
// together.
int resolve_batched(int dim, const pft_options* o, bool shared_q, int64_t n_q, bool& fp64, int& r, int& nt,
                    float& tau, int& q_order) {
  pft_options z;
  std::memset(&z, 0, sizeof(z));
  const pft_options& p = o ? *o : z;
  if (p.precision != PFT_FP32_COMPENSATED && p.precision != PFT_FP64) return PFT_ERR_INVALID_ARG;
  fp64 = p.precision == PFT_FP64;
  r = p.q_per_thread ? p.q_per_thread : (fp64 ? 1 : 4);
  nt = p.block_threads ? p.block_threads
                       : (shared_q && n_q >= (int64_t)r * 512 && batched_config(dim, fp64, r, 512) ? 512 : 128);
  if (!batched_config(dim, fp64, r, nt) || p.tile_items != 0 || p.k_splits != 0) return PFT_ERR_UNSUPPORTED;
  tau = p.face_series_tau == 0.f ? 6.0f : p.face_series_tau;
  if (!(tau > 0.f && tau <= 6.0f)) return PFT_ERR_INVALID_ARG;
  if (fp64) tau = std::min(tau, 3.0f);   // the FP64 series is kept for P < 9/4 (as in the single-shape path)
  if (p.q_order != PFT_Q_TILED && p.q_order != PFT_Q_AS_GIVEN) return PFT_ERR_INVALID_ARG;
  q_order = p.q_order;
  return PFT_OK;
}

int batched_blocks_per_sm(int dim, bool fp64, int r, int nt);

int build_plan(int dim, const int64_t* poly_off, int64_t n_polys, const int64_t* q_off, int64_t n_q,
               const pft_options* opts, HostPlan& P) {
  bool fp64;
  int r, nt, q_order;
  float tau;
  if (int e = resolve_batched(dim, opts, q_off == nullptr, n_q, fp64, r, nt, tau, q_order)) return e;
  if (n_polys < 0 || n_q < 0 || (n_polys > 0 && poly_off == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_polys > 0 && poly_off[0] != 0) return PFT_ERR_OFFSETS;
  for (int64_t i = 0; i < n_polys; ++i)
    if (poly_off[i + 1] < poly_off[i] || poly_off[i + 1] - poly_off[i] > INT32_MAX) return PFT_ERR_OFFSETS;
  if (q_off) {
    if (n_polys > 0 && (q_off[0] != 0 || q_off[n_polys] != n_q)) return PFT_ERR_OFFSETS;
    for (int64_t i = 0; i < n_polys; ++i)
      if (q_off[i + 1] < q_off[i] || q_off[i + 1] - q_off[i] > INT32_MAX) return PFT_ERR_OFFSETS;
  } else if (n_q > INT32_MAX) {
    return PFT_ERR_UNSUPPORTED;
  }
  const int64_t n_out = q_off ? n_q : n_polys * n_q;
  if (n_out > (int64_t)UINT32_MAX) return PFT_ERR_UNSUPPORTED;
  const int64_t qt = (int64_t)r * nt;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t G = std::max(1, sms) * (int64_t)batched_blocks_per_sm(dim, fp64, r, nt);

  P.pplan.resize((size_t)n_polys);
  std::vector<int64_t> cost;
  int64_t part_rows = 0;
  for (int64_t i = 0; i < n_polys; ++i) {
    PolyPlan& pp = P.pplan[(size_t)i];
    pp.seg_begin = poly_off[i];
    pp.n_seg = (int32_t)(poly_off[i + 1] - poly_off[i]);
    pp.q_begin = q_off ? q_off[i] : 0;
    pp.n_q = (int32_t)(q_off ? q_off[i + 1] - q_off[i] : n_q);
    pp.out_base = q_off ? q_off[i] : i * n_q;
    pp.n_chunks = pp.n_seg > 0 ? (int32_t)((pp.n_seg + kChunk - 1) / kChunk) : 1;
    pp.part_base = 0;
    pp.pad = 0;
    if (pp.n_chunks > 1) {
      pp.part_base = part_rows;
      part_rows += (int64_t)pp.n_chunks * pp.n_q;
      P.mc.push_back((int32_t)i);
    }
    const int64_t n_qt = (pp.n_q + qt - 1) / qt;
    for (int32_t c = 0; c < pp.n_chunks; ++c) {
      const int64_t segs = std::min<int64_t>(kChunk, std::max<int64_t>(0, pp.n_seg - (int64_t)c * kChunk));
      for (int64_t t = 0; t < n_qt; ++t) {
        const int64_t nq = std::min<int64_t>(qt, pp.n_q - t * qt);
        P.items.push_back(BItem{(int32_t)i, c, (int32_t)t, 0});
        cost.push_back(nq * (segs + 64));   // pairs plus the per-Q finalize charge
      }
    }
  }
  // longest processing time first onto the least loaded block (ties: lowest index)
  const int64_t n_items = (int64_t)P.items.size();
  std::vector<int64_t> order((size_t)n_items);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
  using Slot = std::pair<int64_t, int64_t>;   // (load, block)
  std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
  for (int64_t b = 0; b < G; ++b) heap.push({0, b});
  std::vector<std::vector<int64_t>> lists((size_t)G);
  for (int64_t k : order) {
    Slot s = heap.top();
    heap.pop();
    lists[(size_t)s.second].push_back(k);
    heap.push({s.first + cost[k], s.second});
  }
  std::vector<BItem> sorted;
  sorted.reserve((size_t)n_items);
  P.cta_off.assign((size_t)G + 1, 0);
  for (int64_t b = 0; b < G; ++b) {
    for (int64_t k : lists[(size_t)b]) sorted.push_back(P.items[(size_t)k]);
    P.cta_off[(size_t)b + 1] = (int32_t)sorted.size();
  }
  P.items.swap(sorted);
  std::memset(&P.h, 0, sizeof(P.h));
  P.h.magic = kPlanMagic;
  P.h.n_polys = n_polys;
  P.h.n_verts = n_polys > 0 ? poly_off[n_polys] : 0;
  P.h.n_q = n_q;
  P.h.n_items = n_items;
  P.h.n_cta = G;
  P.h.n_mc = (int64_t)P.mc.size();
  P.h.part_rows = part_rows;
  P.h.n_out = n_out;
  P.h.r = r;
  P.h.nt = nt;
  P.h.shared_q = q_off ? 0 : 1;
  // per-shape Q lists keep their order; a shared Q set is ordered once for every shape
  P.h.q_tiled = (!q_off && q_order == PFT_Q_TILED && qorder_wanted(n_q, P.h.n_verts, r, nt)) ? 1 : 0;
  P.h.fp64 = fp64 ? 1 : 0;
  P.h.dim = dim;
  P.h.tau = tau;
  return PFT_OK;
}

BLayout layout_of(const BPlanHeader& h) {
  return layout(h.dim, h.n_polys, h.n_verts, h.n_items, h.n_cta, h.n_mc, h.part_rows, h.n_out, h.fp64 != 0, h.n_q,
                h.q_tiled != 0);
}

// ---------------------------------------------------------------------------
// Device kernels.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double bsum(double x, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

__device__ __forceinline__ float bminmax(float x, bool is_max, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float y = __shfl_xor_sync(0xffffffffu, x, o);
    x = is_max ? fmaxf(x, y) : fminf(x, y);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  float r = sh[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = is_max ? fmaxf(r, sh[w]) : fminf(r, sh[w]);
  __syncthreads();
  return r;
}

// One block per polygon: plan check, bounding-box centre, records, FP64 area, max radius.
template <bool FP64>
__global__ void __launch_bounds__(kBThreads) k_bprep(const float* __restrict__ v, const int64_t* __restrict__ poly_off,
                                                     const BPlanHeader* ph, const PolyPlan* __restrict__ pplan,
                                                     PolyInfo* info, void* segs, WsHeader* h) {
  __shared__ double shd[kBThreads / 32];
  __shared__ float shf[kBThreads / 32];
  const int64_t i = blockIdx.x;
  const PolyPlan pp = pplan[i];
  const int64_t s0 = poly_off[i], s1 = poly_off[i + 1];
  if (threadIdx.x == 0 && (s0 != pp.seg_begin || s1 - s0 != pp.n_seg || ph->magic != kPlanMagic))
    set_status(&h->status, ST_OFFSETS);   // offsets differ from the prepared plan
  const int64_t n = min((int64_t)pp.n_seg, max((int64_t)0, s1 - s0));
  float mn[2] = {3.4e38f, 3.4e38f}, mx[2] = {-3.4e38f, -3.4e38f};
  bool bad = false;
  for (int64_t j = threadIdx.x; j < n; j += kBThreads)
    for (int d = 0; d < 2; ++d) {
      const float x = v[2 * (pp.seg_begin + j) + d];
      if (!isfinite(x)) { bad = true; continue; }
      mn[d] = fminf(mn[d], x);
      mx[d] = fmaxf(mx[d], x);
    }
  if (bad) set_status(&h->status, ST_NONFINITE);
  double c[2];
  for (int d = 0; d < 2; ++d) {
    const float lo = bminmax(mn[d], false, shf), hi = bminmax(mx[d], true, shf);
    c[d] = (n > 0 && lo <= hi) ? 0.5 * ((double)lo + (double)hi) : 0.0;
  }
  double area = 0.0;
  float rm = 0.f;
  if constexpr (FP64) {
    for (int64_t j = threadIdx.x; j < n; j += kBThreads) {
      const int64_t a = pp.seg_begin + j, b = pp.seg_begin + (j + 1 < n ? j + 1 : 0);
      const double x0 = (double)v[2 * a] - c[0], y0 = (double)v[2 * a + 1] - c[1];
      const double x1 = (double)v[2 * b] - c[0], y1 = (double)v[2 * b + 1] - c[1];
      area += 0.5 * (x0 * y1 - x1 * y0);
      rm = fmaxf(rm, __double2float_ru(sqrt(x0 * x0 + y0 * y0)));
      reinterpret_cast<Seg64*>(segs)[a] = Seg64{0.5 * (x0 + x1), 0.5 * (y0 + y1), 0.5 * (x1 - x0), 0.5 * (y1 - y0)};
    }
  } else {
    // FP32 records without FP64 arithmetic (GB300's FP64 pipe is a small fraction of its FP32
    // rate): with the centre c = c_hi + c_lo as floats, v - c_hi = s + e exactly (TwoSum), so a
    // centred coordinate is the float pair s + (e - c_lo); m and h are each rounded once from the
    // float-pair sum or difference of two such pairs.  The area is the record polygon's own
    // (p0 x p1 / 2 = mx hy - my hx for p0,1 = m -/+ h), each product split exactly by its FMA and
    // summed with compensation: within ~1e-7 of the vertex polygon's, as the records are.  The
    // radius bound comes from the centred vertex in FP32, raised by a relative 1e-6 to stay above
    // the exact value.
    float chi[2], clo[2];
    for (int d = 0; d < 2; ++d) {
      chi[d] = __double2float_rn(c[d]);
      clo[d] = __double2float_rn(c[d] - (double)chi[d]);
    }
    auto centred = [&](float x, int d, float& s, float& t) {
      float e;
      two_sum(x, -chi[d], s, e);
      t = e - clo[d];
    };
    auto half_sum = [](float s0, float t0, float s1, float t1) {   // (s0 + t0 + s1 + t1) / 2
      float s, e;
      two_sum(s0, s1, s, e);
      return 0.5f * (s + (e + (t0 + t1)));
    };
    CAcc ar;
    ar.init();
    for (int64_t j = threadIdx.x; j < n; j += kBThreads) {
      const int64_t a = pp.seg_begin + j, b = pp.seg_begin + (j + 1 < n ? j + 1 : 0);
      float s0x, t0x, s0y, t0y, s1x, t1x, s1y, t1y;
      centred(v[2 * a], 0, s0x, t0x);
      centred(v[2 * a + 1], 1, s0y, t0y);
      centred(v[2 * b], 0, s1x, t1x);
      centred(v[2 * b + 1], 1, s1y, t1y);
      const float mx = half_sum(s0x, t0x, s1x, t1x), my = half_sum(s0y, t0y, s1y, t1y);
      const float hx = half_sum(s1x, t1x, -s0x, -t0x), hy = half_sum(s1y, t1y, -s0y, -t0y);
      reinterpret_cast<Seg32*>(segs)[a] = Seg32{mx, my, hx, hy};
      const float p = mx * hy, pe = fmaf(mx, hy, -p), q = my * hx, qe = fmaf(my, hx, -q);
      float d, de;
      two_sum(p, -q, d, de);
      ar.add(d);
      ar.add(de + (pe - qe));
      rm = fmaxf(rm, sqrtf(fmaf(s0x, s0x, s0y * s0y)) * 1.000001f);
    }
    area = (double)ar.hi + (double)ar.lo;
  }
  area = bsum(area, shd);
  rm = bminmax(rm, true, shf);
  if (threadIdx.x == 0) info[i] = PolyInfo{c[0], c[1], 0.0, area, rm, 0u};
}

// One block per mesh (3D): plan check, bounding-box centre of the face corners, face records
// (as k_prep3d: centroid, corners 0 and 1 relative to it, N, all relative to the centre),
// FP64 volume from the signed tetrahedra, max radius.  Bad indices or coordinates set the
// status and the face is written empty (it contributes 0).
template <bool FP64>
__global__ void __launch_bounds__(kBThreads) k_bprep3(const float* __restrict__ v, int64_t nv,
                                                      const int32_t* __restrict__ f,
                                                      const int64_t* __restrict__ mesh_off, const BPlanHeader* ph,
                                                      const PolyPlan* __restrict__ pplan, PolyInfo* info,
                                                      void* recs, WsHeader* h) {
  __shared__ double shd[kBThreads / 32];
  __shared__ float shf[kBThreads / 32];
  const int64_t i = blockIdx.x;
  const PolyPlan pp = pplan[i];
  const int64_t s0 = mesh_off[i], s1 = mesh_off[i + 1];
  if (threadIdx.x == 0 && (s0 != pp.seg_begin || s1 - s0 != pp.n_seg || ph->magic != kPlanMagic))
    set_status(&h->status, ST_OFFSETS);   // offsets differ from the prepared plan
  const int64_t n = min((int64_t)pp.n_seg, max((int64_t)0, s1 - s0));
  auto corner_ok = [&](int64_t m) {
    const int32_t a = f[3 * m], b = f[3 * m + 1], c = f[3 * m + 2];
    return a >= 0 && b >= 0 && c >= 0 && a < nv && b < nv && c < nv;
  };
  float mn[3] = {3.4e38f, 3.4e38f, 3.4e38f}, mx[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
  bool bad_idx = false, bad_val = false;
  for (int64_t j = threadIdx.x; j < n; j += kBThreads) {
    const int64_t m = pp.seg_begin + j;
    if (!corner_ok(m)) { bad_idx = true; continue; }
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) {
        const float x = v[3 * (int64_t)f[3 * m + k] + d];
        if (!isfinite(x)) { bad_val = true; continue; }
        mn[d] = fminf(mn[d], x);
        mx[d] = fmaxf(mx[d], x);
      }
  }
  if (bad_idx) set_status(&h->status, ST_INDEX);
  if (bad_val) set_status(&h->status, ST_NONFINITE);
  double c[3];
  for (int d = 0; d < 3; ++d) {
    const float lo = bminmax(mn[d], false, shf), hi = bminmax(mx[d], true, shf);
    c[d] = (n > 0 && lo <= hi) ? 0.5 * ((double)lo + (double)hi) : 0.0;
  }
  double vol = 0.0;
  float rm = 0.f;
  if constexpr (FP64) {
    for (int64_t j = threadIdx.x; j < n; j += kBThreads) {
      const int64_t m = pp.seg_begin + j;
      double g[3] = {0, 0, 0}, q0[3] = {0, 0, 0}, q1[3] = {0, 0, 0}, N[3] = {0, 0, 0};
      if (corner_ok(m)) {
        double P[3][3];
        bool fin = true;
        for (int k = 0; k < 3; ++k)
          for (int d = 0; d < 3; ++d) {
            P[k][d] = (double)v[3 * (int64_t)f[3 * m + k] + d] - c[d];
            fin = fin && isfinite(P[k][d]);
          }
        if (fin) {
          for (int d = 0; d < 3; ++d) {
            g[d] = (P[0][d] + P[1][d] + P[2][d]) / 3.0;
            q0[d] = P[0][d] - g[d];
            q1[d] = P[1][d] - g[d];
          }
          const double e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
          const double e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
          N[0] = e1[1] * e2[2] - e1[2] * e2[1];
          N[1] = e1[2] * e2[0] - e1[0] * e2[2];
          N[2] = e1[0] * e2[1] - e1[1] * e2[0];
          vol += (P[0][0] * (P[1][1] * P[2][2] - P[1][2] * P[2][1]) +
                  P[0][1] * (P[1][2] * P[2][0] - P[1][0] * P[2][2]) +
                  P[0][2] * (P[1][0] * P[2][1] - P[1][1] * P[2][0])) / 6.0;
          double r2 = 0.0;
          for (int k = 0; k < 3; ++k) r2 = fmax(r2, P[k][0] * P[k][0] + P[k][1] * P[k][1] + P[k][2] * P[k][2]);
          rm = fmaxf(rm, __double2float_ru(sqrt(r2)));
        }
      }
      reinterpret_cast<Face64*>(recs)[m] = Face64{g[0], g[1], g[2], q0[0], q0[1], q0[2], q1[0], q1[1], q1[2],
                                                  N[0], N[1], N[2]};
    }
  } else {
    // FP32 records without FP64 arithmetic, as k_bprep: each centred corner is a float pair
    // s + t (TwoSum of the vertex and the centre's high part, less its low part); the centroid is
    // rounded once from the pair sum over 3 (the remainder of the rounded quotient is exact through
    // its FMA), q0, q1 and the edges from TwoSum differences, N = e1 x e2 with Kahan's FMA form of
    // each 2 x 2 determinant.  The volume is the records' own: det(P0, P1, P2) = g . N for the
    // centroid g and N = (P1 - P0) x (P2 - P0), so it is the compensated sum of g . N over 6, each
    // product split exactly by its FMA.  Radius bound as in 2D.
    float chi[3], clo[3];
    for (int d = 0; d < 3; ++d) {
      chi[d] = __double2float_rn(c[d]);
      clo[d] = __double2float_rn(c[d] - (double)chi[d]);
    }
    auto det2 = [](float a, float b, float cc, float dd) {   // a b - cc dd
      const float w = cc * dd;
      return fmaf(a, b, -w) + fmaf(-cc, dd, w);
    };
    CAcc va;
    va.init();
    for (int64_t j = threadIdx.x; j < n; j += kBThreads) {
      const int64_t m = pp.seg_begin + j;
      float G[3] = {0.f, 0.f, 0.f}, Q0[3] = {0.f, 0.f, 0.f}, Q1[3] = {0.f, 0.f, 0.f}, Nn[3] = {0.f, 0.f, 0.f};
      if (corner_ok(m)) {
        float sp[3][3], tp[3][3];
        bool fin = true;
        for (int k = 0; k < 3; ++k)
          for (int d = 0; d < 3; ++d) {
            const float x = v[3 * (int64_t)f[3 * m + k] + d];
            fin = fin && isfinite(x);
            float e;
            two_sum(x, -chi[d], sp[k][d], e);
            tp[k][d] = e - clo[d];
          }
        if (fin) {
          float e1[3], e2[3];
          for (int d = 0; d < 3; ++d) {
            float a, ea, b, eb;
            two_sum(sp[0][d], sp[1][d], a, ea);
            two_sum(a, sp[2][d], b, eb);
            const float lo = (ea + eb) + (tp[0][d] + tp[1][d] + tp[2][d]);
            const float gh = b / 3.0f;
            G[d] = gh + (fmaf(-gh, 3.0f, b) + lo) / 3.0f;
            float x, ex;
            two_sum(sp[0][d], -G[d], x, ex);
            Q0[d] = x + (ex + tp[0][d]);
            two_sum(sp[1][d], -G[d], x, ex);
            Q1[d] = x + (ex + tp[1][d]);
            two_sum(sp[1][d], -sp[0][d], x, ex);
            e1[d] = x + (ex + (tp[1][d] - tp[0][d]));
            two_sum(sp[2][d], -sp[0][d], x, ex);
            e2[d] = x + (ex + (tp[2][d] - tp[0][d]));
          }
          Nn[0] = det2(e1[1], e2[2], e1[2], e2[1]);
          Nn[1] = det2(e1[2], e2[0], e1[0], e2[2]);
          Nn[2] = det2(e1[0], e2[1], e1[1], e2[0]);
          for (int d = 0; d < 3; ++d) {
            const float pr = G[d] * Nn[d];
            va.add(pr);
            va.add(fmaf(G[d], Nn[d], -pr));
          }
          for (int k = 0; k < 3; ++k)
            rm = fmaxf(rm, sqrtf(fmaf(sp[k][0], sp[k][0], fmaf(sp[k][1], sp[k][1], sp[k][2] * sp[k][2]))) * 1.000001f);
        }
      }
      reinterpret_cast<Face32*>(recs)[m] = Face32{G[0], G[1], G[2], Q0[0], Q0[1], Q0[2], Q1[0], Q1[1], Q1[2],
                                                  Nn[0], Nn[1], Nn[2]};
    }
    vol = ((double)va.hi + (double)va.lo) / 6.0;
  }
  vol = bsum(vol, shd);
  rm = bminmax(rm, true, shf);
  if (threadIdx.x == 0) info[i] = PolyInfo{c[0], c[1], c[2], vol, rm, 0u};
}

// Shared finish of one output: s/|Q|^2 * exp(iQ.c) * sum (s = 2 in 2D, where the records hold
// half the cross product; 1 in 3D), Q = 0 -> area or volume, small |Q| -> FP64 list.
// kF32: the sums come from the FP32 policies (relative error ~1e-7), so the factor 2/|Q|^2 (1/|Q|^2
// in 3D) is an FP32 division and the translation phase an FP32 sincos of Q.c less its nearest
// multiple of 2 pi (both taken in FP64): about 15 FP64 operations per output instead of about 65,
// which keeps GB300's narrow FP64 pipe from stalling the warps at the end of every item, for at
// most ~3e-7 of |F| more error.  The FP64 policies keep FP64 throughout.
template <int D, bool kF32>
__device__ __forceinline__ void finish_out(const double* Q, double re, double im, const PolyInfo& pi, int64_t row,
                                           double* out, uint32_t* small, WsHeader* h) {
  double q2 = 0.0, ph = 0.0;
  const double c[3] = {pi.cx, pi.cy, pi.cz};
#pragma unroll
  for (int d = 0; d < D; ++d) {
    q2 += Q[d] * Q[d];
    ph += Q[d] * c[d];
  }
  if (q2 == 0.0) {
    out[2 * row] = pi.measure;
    out[2 * row + 1] = 0.0;
    return;
  }
  if (q2 * ((double)pi.rmax * (double)pi.rmax) < kTauSmallQ * kTauSmallQ) {   // |Q| r_max < tau_small
    small[atomicAdd(&h->small_q_count, 1u)] = (uint32_t)row;
    return;
  }
  double k, sp, cp;
  if constexpr (kF32) {
    const float pr = (float)fma(-rint(ph * kInvTwoPiD), kTwoPiD, ph);
    float sf, cf;
    sincosf(pr, &sf, &cf);
    sp = sf;
    cp = cf;
    k = (double)((D == 2 ? 2.0f : 1.0f) / (float)q2);
  } else {
    sincos(ph, &sp, &cp);
    k = (D == 2 ? 2.0 : 1.0) / q2;
  }
  out[2 * row] = k * (re * cp - im * sp);
  out[2 * row + 1] = k * (re * sp + im * cp);
}

// The centre as float pairs c = hi + lo (to ~2^-48 of |c|), taken once per item.
struct CenterF {
  float hi[3], lo[3];
};
__device__ __forceinline__ CenterF center_f(const PolyInfo& pi) {
  const double c[3] = {pi.cx, pi.cy, pi.cz};
  CenterF f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    f.hi[d] = __double2float_rn(c[d]);
    f.lo[d] = __double2float_rn(c[d] - (double)f.hi[d]);
  }
  return f;
}

constexpr float kTwoPiHi = 6.28318548202514648438f;       // 2 pi rounded to FP32
constexpr float kTwoPiLo = -1.7484555314695172e-07f;        // 2 pi - kTwoPiHi, rounded to FP32

// The same finish for the FP32 policies' single-chunk outputs, without FP64 arithmetic: GB300 runs
// FP64 at a small fraction of its FP32 rate, and all warps of a block reach this together at the end
// of every item.  The phase takes the caller's Q, Q + Qlo (Q rounded to float, as the pair sums used
// it, and the low part q - (float)q from k_bqlo): a shape far from the origin would otherwise see
// its phase moved by |c| times the rounding of Q.  Q.c is carried as s + t (the products Q c_hi exact
// through their FMA residuals; Q c_lo, Qlo c_hi and the residuals in t), k = rint(s / 2 pi), and s - k 2pi_hi is exact in FP32 (both
// are multiples of 2^-21 and the difference is below 4 in magnitude), so the reduced phase carries one
// rounding, as the FP64 reduction cast to FP32 does; sincosf of it, the factor s/|Q|^2 and the
// rotation of hi + lo in FP32: about 3e-7 of |F| against ~1e-7 for the sums themselves.  Phases
// beyond 2^20 rad take the FP64 finish.
template <int D>
__device__ __forceinline__ void finish_out_f32(const float* Q, const float* Qlo, const CAcc& re, const CAcc& im,
                                               const PolyInfo& pi,
                                               const CenterF& cf, int64_t row, double* out, uint32_t* small,
                                               WsHeader* h) {
  bool zero = true;
  float q2 = 0.f;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    zero = zero && Q[d] == 0.f;
    q2 = fmaf(Q[d], Q[d], q2);
  }
  if (zero) {
    out[2 * row] = pi.measure;
    out[2 * row + 1] = 0.0;
    return;
  }
  if (q2 * (pi.rmax * pi.rmax) < (float)(kTauSmallQ * kTauSmallQ)) {   // |Q| r_max < tau_small
    small[atomicAdd(&h->small_q_count, 1u)] = (uint32_t)row;
    return;
  }
  float s = Q[0] * cf.hi[0];
  float t = fmaf(Q[0], cf.hi[0], -s);
#pragma unroll
  for (int d = 1; d < D; ++d) {
    const float p = Q[d] * cf.hi[d];
    const float e = fmaf(Q[d], cf.hi[d], -p);
    float s2, e2;
    two_sum(s, p, s2, e2);
    s = s2;
    t += e2 + e;
  }
#pragma unroll
  for (int d = 0; d < D; ++d) t = fmaf(Qlo[d], cf.hi[d], fmaf(Q[d], cf.lo[d], t));
  if (!(fabsf(s) < 1048576.f)) {
    const double Qd[3] = {(double)Q[0] + (double)Qlo[0], (double)Q[1] + (double)Qlo[1],
                          D == 3 ? (double)Q[2] + (double)Qlo[2] : 0.0};
    finish_out<D, true>(Qd, (double)re.hi + (double)re.lo, (double)im.hi + (double)im.lo, pi, row, out, small, h);
    return;
  }
  const float k = rintf(s * kInvTwoPi);
  const float ph = fmaf(-k, kTwoPiHi, s) + fmaf(-k, kTwoPiLo, t);
  float sp, cp;
  sincosf(ph, &sp, &cp);
  const float f = (D == 2 ? 2.0f : 1.0f) / q2;
  const float a = re.hi + re.lo, b = im.hi + im.lo;
  out[2 * row] = (double)(f * fmaf(a, cp, -b * sp));
  out[2 * row + 1] = (double)(f * fmaf(a, sp, b * cp));
}

// Persistent kernel: block b runs items [cta_off[b], cta_off[b+1]) in order.  The
// segment tiles of consecutive items form one stream through the ring; the last
// warp to finish a slot issues the tile kStages further on (as in k_fwd).
// Register budget: as the single-shape kernel, except that the 3D FP32 shapes with 128 threads
// keep one block per SM fewer here (4 at 4 Q points, 5 at 2), where the item loop and the
// in-place finish would otherwise spill, and that 512 threads are one block per SM (up to 128
// registers: 16 warps, as 2 x 256 or 4 x 128).
// Records per tile of the batched kernel's ring.  With one block of 16 warps per SM walking it (the
// 512-thread shapes), 256 segments ran faster than 128 (4,096 polygons: 7.63 against 7.70 ms) and
// 128 faces faster than 64 (1,024 meshes: 67.2 against 68.2 ms): a 16 KB or 24 KB ring.  The other
// launch shapes take the policy's tile.
template <class Pol, int NT>
constexpr int kBTile = NT >= 512 ? (Pol::kDim == 2 ? 256 : 128) : Pol::kTile;

template <class Pol, int R, int NT>
constexpr int kBatchedMinBlocks = NT >= 512 ? 1
                                  : (Pol::kDim == 3 && R == 4 && NT == 128) ? 4
                                  : (Pol::kDim == 3 && R == 2 && NT == 128 && sizeof(typename Pol::QT) == 4)
                                      ? 5
                                      : kMinBlocks<Pol, R, NT>;

template <class Pol, int R, int NT>
__global__ void __launch_bounds__(NT, kBatchedMinBlocks<Pol, R, NT>) k_batched(
    const BPlanHeader* __restrict__ ph, const int32_t* __restrict__ cta_off, const BItem* __restrict__ items,
    const PolyPlan* __restrict__ pplan, const PolyInfo* __restrict__ info, const typename Pol::Item* __restrict__ segs,
    const double* __restrict__ q, double2* __restrict__ partial, double* __restrict__ out, uint32_t* small,
    WsHeader* h, Thr th, const int32_t* __restrict__ qperm, const float* __restrict__ qlo) {
  using Item = typename Pol::Item;
  using QT = typename Pol::QT;
  constexpr int TILE = kBTile<Pol, NT>;
  constexpr int D = Pol::kDim;
  constexpr int NW = NT / 32;
  __shared__ __align__(128) Item ring[kStages * TILE];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ int done[kStages];
  __shared__ int issued;

  const int k0 = cta_off[blockIdx.x], k1 = cta_off[blockIdx.x + 1];
  auto seg_range = [&](int k, int64_t& begin, int& count) {
    const BItem it = items[k];
    const PolyPlan& pp = pplan[it.poly];
    const int64_t off = (int64_t)it.chunk * kChunk;
    begin = pp.seg_begin + off;
    count = (int)max((int64_t)0, min((int64_t)kChunk, (int64_t)pp.n_seg - off));
  };
  auto n_tiles = [&](int k) {
    int64_t b;
    int c;
    seg_range(k, b, c);
    return (c + TILE - 1) / TILE;
  };
  // copy tile tt of item kk into slot s
  auto issue = [&](int kk, int tt, int s) {
    int64_t b;
    int c;
    seg_range(kk, b, c);
    const int m = min(TILE, c - tt * TILE);
    const uint32_t bytes = (uint32_t)(m * (int)sizeof(Item));
    mbar_arrive_expect_tx(&full[s], bytes);
    bulk_g2s(ring + s * TILE, segs + b + (int64_t)tt * TILE, bytes, &full[s]);
    atomicAdd(&issued, 1);
  };
  // the position `steps` tiles after (kk, tt) in this block's stream; false past the end
  auto advance = [&](int& kk, int& tt, int steps) {
    while (steps-- > 0) {
      if (tt + 1 < n_tiles(kk)) {
        ++tt;
        continue;
      }
      do { ++kk; } while (kk < k1 && n_tiles(kk) == 0);
      if (kk >= k1) return false;
      tt = 0;
    }
    return true;
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
  if (threadIdx.x == 0) {   // the first kStages tiles of the stream
    int kk = k0, tt = 0;
    while (kk < k1 && n_tiles(kk) == 0) ++kk;
    for (int s = 0; s < kStages && kk < k1; ++s) {
      issue(kk, tt, s);
      if (!advance(kk, tt, 1)) break;
    }
  }

  bool ok = true;
  int64_t g = 0;   // position of the current tile in this block's stream
  for (int k = k0; k < k1 && ok; ++k) {
    const BItem it = items[k];
    const PolyPlan pp = pplan[it.poly];
    int64_t sb;
    int cnt;
    seg_range(k, sb, cnt);
    const int64_t q0 = pp.q_begin + (int64_t)it.qtile * (NT * R);
    const int64_t qend = pp.q_begin + pp.n_q;
    // slot iq holds Q row qperm[iq] (shared Q set, q_begin = 0), else row iq itself
    QT qr[R][3];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t iq = q0 + (int64_t)r * NT + threadIdx.x;
      qr[r][0] = qr[r][1] = qr[r][2] = (QT)0;
      if (iq < qend) {
        const int64_t src = qperm ? (int64_t)qperm[iq] : iq;
#pragma unroll
        for (int d = 0; d < D; ++d) qr[r][d] = (QT)q[D * src + d];
      }
    }
    typename Pol::template Acc<R> acc;
    acc.init();
    const int ntk = (cnt + TILE - 1) / TILE;
    for (int t = 0; t < ntk; ++t, ++g) {
      const int s = (int)(g % kStages);
      // stop decisions are warp-uniform (see k_fwd)
      if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[s], (uint32_t)((g / kStages) & 1)))) {
        ok = false;
        break;
      }
      Pol::template tile<R>(ring + s * TILE, min(TILE, cnt - t * TILE), qr, acc, th, 0);
      __syncwarp();
      if ((threadIdx.x & 31) == 0) {
        __threadfence_block();
        if (atomicAdd(&done[s], 1) == NW - 1) {   // last warp out of slot s refills it
          atomicExch(&done[s], 0);
          int kk = k, tt = t;
          if (advance(kk, tt, kStages)) {
            fence_proxy_async_smem();
            issue(kk, tt, s);
          }
        }
      }
    }
    if (!ok) break;
    const PolyInfo pi = info[it.poly];
    constexpr bool kF32 = sizeof(QT) == 4;
    CenterF cf{};
    if constexpr (kF32) {
      if (pp.n_chunks == 1) cf = center_f(pi);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t iq = q0 + (int64_t)r * NT + threadIdx.x;
      if (iq >= qend) continue;
      const int64_t local = (qperm ? (int64_t)qperm[iq] : iq) - pp.q_begin;
      if (pp.n_chunks > 1) {
        const int64_t pidx = pp.part_base + (int64_t)it.chunk * pp.n_q + local;
        if constexpr (kF32)   // the compensated sums as they are: (re hi, re lo, im hi, im lo)
          reinterpret_cast<float4*>(partial)[pidx] =
              make_float4(acc.re[r].hi, acc.re[r].lo, acc.im[r].hi, acc.im[r].lo);
        else
          partial[pidx] = acc.get(r);
      } else if constexpr (kF32) {
        float ql[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int d = 0; d < D; ++d) ql[d] = qlo[D * (pp.q_begin + local) + d];
        finish_out_f32<D>(qr[r], ql, acc.re[r], acc.im[r], pi, cf, pp.out_base + local, out, small, h);
      } else {
        const double2 f = acc.get(r);
        const double Qd[3] = {(double)qr[r][0], (double)qr[r][1], (double)qr[r][2]};
        finish_out<D, false>(Qd, f.x, f.y, pi, pp.out_base + local, out, small, h);
      }
    }
  }
  if (!ok) set_status(&h->status, ST_TIMEOUT);
  __syncthreads();
  if (threadIdx.x == 0) {   // no copy may still be writing into the ring when the block exits
    const int m = issued;
    for (int u = max(0, m - kStages); u < m; ++u)
      (void)mbar_wait_bounded(&full[u % kStages], (uint32_t)((u / kStages) & 1));
  }
}

// The low parts q - (float)q of the caller's Q coordinates (FP32 policies), for the finish's phase.
__global__ void __launch_bounds__(kBThreads) k_bqlo(const double* __restrict__ q, int64_t n, float* __restrict__ qlo) {
  const int64_t i = blockIdx.x * (int64_t)kBThreads + threadIdx.x;
  if (i < n) qlo[i] = __double2float_rn(q[i] - (double)__double2float_rn(q[i]));
}

// Multi-chunk shapes: fixed-order sum of their chunk partials, then the finish.  The FP32
// policies' partials are compensated float pairs, added in the same compensated accumulator and
// finished in FP32 (as the single-chunk outputs are); the FP64 policies' are doubles.
__global__ void __launch_bounds__(kBThreads) k_bfinal(const BPlanHeader* ph, const int32_t* __restrict__ mc,
                                                      const PolyPlan* __restrict__ pplan,
                                                      const PolyInfo* __restrict__ info, const double* __restrict__ q,
                                                      const double2* __restrict__ partial, double* out,
                                                      uint32_t* small, WsHeader* h, const float* __restrict__ qlo) {
  const int i = mc[blockIdx.x];
  const PolyPlan pp = pplan[i];
  const PolyInfo pi = info[i];
  const bool fp64 = ph->fp64 != 0;
  const int D = ph->dim;
  if (!fp64) {
    const CenterF cf = center_f(pi);
    const float4* pf = reinterpret_cast<const float4*>(partial);
    for (int64_t l = threadIdx.x; l < pp.n_q; l += kBThreads) {
      CAcc re, im;
      re.init();
      im.init();
      for (int c = 0; c < pp.n_chunks; ++c) {
        const float4 p = pf[pp.part_base + (int64_t)c * pp.n_q + l];
        re.add(p.x);
        re.add(p.y);
        im.add(p.z);
        im.add(p.w);
      }
      const int64_t iq = pp.q_begin + l;
      float Q[3], ql[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        Q[d] = d < D ? (float)q[D * iq + d] : 0.f;
        ql[d] = d < D ? qlo[D * iq + d] : 0.f;
      }
      if (D == 2) finish_out_f32<2>(Q, ql, re, im, pi, cf, pp.out_base + l, out, small, h);
      else finish_out_f32<3>(Q, ql, re, im, pi, cf, pp.out_base + l, out, small, h);
    }
    return;
  }
  for (int64_t l = threadIdx.x; l < pp.n_q; l += kBThreads) {
    double re = 0.0, im = 0.0;
    for (int c = 0; c < pp.n_chunks; ++c) {
      const double2 p = partial[pp.part_base + (int64_t)c * pp.n_q + l];
      re += p.x;
      im += p.y;
    }
    const int64_t iq = pp.q_begin + l;
    double Q[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < D; ++d) Q[d] = q[D * iq + d];
    if (D == 2) finish_out<2, false>(Q, re, im, pi, pp.out_base + l, out, small, h);
    else finish_out<3, false>(Q, re, im, pi, pp.out_base + l, out, small, h);
  }
}

// FP64 small-|Q| pass: fan of signed triangles (c, p_j, p_{j+1}) with the simplex series.
__global__ void __launch_bounds__(kBThreads) k_bsmall(const float* __restrict__ v, const BPlanHeader* ph,
                                                      const PolyPlan* __restrict__ pplan,
                                                      const PolyInfo* __restrict__ info, const int64_t* q_off,
                                                      const double* __restrict__ q, const uint32_t* small,
                                                      double* out, const WsHeader* h) {
  __shared__ double sh[kBThreads / 32];
  const uint32_t count = h->small_q_count;
  const int64_t n_q = ph->n_q, n_polys = ph->n_polys;
  for (uint32_t e = blockIdx.x; e < count; e += gridDim.x) {
    const int64_t row = small[e];
    int64_t i, iq;
    if (ph->shared_q) {
      i = row / n_q;
      iq = row % n_q;
    } else {
      int64_t lo = 0, hi = n_polys;   // last polygon whose Q range starts at or before row
      while (lo + 1 < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (q_off[mid] <= row) lo = mid; else hi = mid;
      }
      i = lo;
      iq = row;
    }
    const PolyPlan pp = pplan[i];
    const PolyInfo pi = info[i];
    const double qx = q[2 * iq], qy = q[2 * iq + 1];   // the caller's Q (FP64 series, either precision)
    double re = 0.0, im = 0.0;
    for (int64_t j = threadIdx.x; j < pp.n_seg; j += kBThreads) {
      const int64_t a = pp.seg_begin + j, b = pp.seg_begin + (j + 1 < pp.n_seg ? j + 1 : 0);
      const double x0 = (double)v[2 * a] - pi.cx, y0 = (double)v[2 * a + 1] - pi.cy;
      const double x1 = (double)v[2 * b] - pi.cx, y1 = (double)v[2 * b + 1] - pi.cy;
      const double n0 = qx * x0 + qy * y0, n1 = qx * x1 + qy * y1;
      // sum_k i^k h_k(n0, n1) / (k+2)!, 16 terms (|n| < 0.25)
      double hk = 1.0, p1 = 1.0, inv = 0.5, sr = 0.0, si = 0.0;
      for (int k = 0; k <= 16; ++k) {
        if (k > 0) {
          p1 *= n1;
          hk = n0 * hk + p1;   // h_k(n0, n1) = n0 h_{k-1} + n1^k
        }
        const double t = hk * inv;
        switch (k & 3) { case 0: sr += t; break; case 1: si += t; break; case 2: sr -= t; break; default: si -= t; }
        inv /= (double)(k + 3);
      }
      const double det = x0 * y1 - x1 * y0;
      re += det * sr;
      im += det * si;
    }
    re = bsum(re, sh);
    im = bsum(im, sh);
    if (threadIdx.x == 0) {
      double sp, cp;
      sincos(qx * pi.cx + qy * pi.cy, &sp, &cp);
      out[2 * row] = re * cp - im * sp;
      out[2 * row + 1] = re * sp + im * cp;
    }
  }
}

// FP64 small-|Q| pass in 3D: the mesh's signed tetrahedra (c, p0, p1, p2) with the simplex
// series (as k_smallq3d for one mesh).
__global__ void __launch_bounds__(kBThreads) k_bsmall3(const float* __restrict__ v, int64_t nv,
                                                       const int32_t* __restrict__ f, const BPlanHeader* ph,
                                                       const PolyPlan* __restrict__ pplan,
                                                       const PolyInfo* __restrict__ info,
                                                       const int64_t* __restrict__ q_off,
                                                       const double* __restrict__ q, const uint32_t* small,
                                                       double* out, const WsHeader* h) {
  __shared__ double sh[kBThreads / 32];
  const uint32_t count = h->small_q_count;
  const int64_t n_q = ph->n_q, n_polys = ph->n_polys;
  for (uint32_t e = blockIdx.x; e < count; e += gridDim.x) {
    const int64_t row = small[e];
    int64_t i, iq;
    if (ph->shared_q) {
      i = row / n_q;
      iq = row % n_q;
    } else {
      int64_t lo = 0, hi = n_polys;   // last mesh whose Q range starts at or before row
      while (lo + 1 < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (q_off[mid] <= row) lo = mid; else hi = mid;
      }
      i = lo;
      iq = row;
    }
    const PolyPlan pp = pplan[i];
    const PolyInfo pi = info[i];
    const double c[3] = {pi.cx, pi.cy, pi.cz};
    double Q[3];
    for (int d = 0; d < 3; ++d) Q[d] = q[3 * iq + d];   // the caller's Q (FP64 series, either precision)
    double re = 0.0, im = 0.0;
    for (int64_t j = threadIdx.x; j < pp.n_seg; j += kBThreads) {
      const int64_t m = pp.seg_begin + j;
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
    re = bsum(re, sh);
    im = bsum(im, sh);
    if (threadIdx.x == 0) {
      double sp, cp;
      sincos(Q[0] * c[0] + Q[1] * c[1] + Q[2] * c[2], &sp, &cp);
      out[2 * row] = re * cp - im * sp;
      out[2 * row + 1] = re * sp + im * cp;
    }
  }
}

template <class Pol, int R, int NT>
int occ_batched() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batched<Pol, R, NT>, NT, 0) != cudaSuccess) return 1;
  return b > 0 ? b : 1;
}

template <class Pol, int R, int NT>
cudaError_t launch_batched_one(int grid, const BPlanHeader* ph, const int32_t* cta_off, const BItem* items,
                               const PolyPlan* pplan, const PolyInfo* info, const void* segs, const double* q,
                               double2* partial, double* out, uint32_t* small, WsHeader* h, Thr th, cudaStream_t st,
                               const int32_t* qperm, const float* qlo) {
  k_batched<Pol, R, NT><<<grid, NT, 0, st>>>(ph, cta_off, items, pplan, info,
                                             static_cast<const typename Pol::Item*>(segs), q, partial, out, small, h,
                                             th, qperm, qlo);
  return cudaGetLastError();
}

// Instantiated configurations: (policy, Q points per thread, threads per block).
#define PFT_BATCHED_CASES(X)                                                                          \
  X(Pol2F32, 1, 128) X(Pol2F32, 2, 128) X(Pol2F32, 4, 128) X(Pol2F32, 8, 128) X(Pol2F32, 1, 256)      \
  X(Pol2F32, 2, 256) X(Pol2F32, 4, 256) X(Pol2F32, 8, 256) X(Pol2F64, 1, 128) X(Pol2F64, 2, 128)      \
  X(Pol2F64, 1, 256) X(Pol2F64, 2, 256) X(Pol3F32, 2, 128) X(Pol3F32, 4, 128) X(Pol3F64, 1, 128)      \
  X(Pol2F32, 4, 512) X(Pol3F32, 4, 512)

#define PFT_BATCHED_MATCH(P, RR, NN) \
  (P::kDim == dim && (sizeof(P::QT) == 8) == fp64 && r == RR && nt == NN)

bool batched_config(int dim, bool fp64, int r, int nt) {
#define X(P, RR, NN) \
  if (PFT_BATCHED_MATCH(P, RR, NN)) return true;
  PFT_BATCHED_CASES(X)
#undef X
  return false;
}

int batched_blocks_per_sm(int dim, bool fp64, int r, int nt) {
#define X(P, RR, NN) \
  if (PFT_BATCHED_MATCH(P, RR, NN)) return occ_batched<P, RR, NN>();
  PFT_BATCHED_CASES(X)
#undef X
  return 1;
}

cudaError_t launch_batched(int dim, bool fp64, int r, int nt, int grid, const BPlanHeader* ph, const int32_t* cta_off,
                           const BItem* items, const PolyPlan* pplan, const PolyInfo* info, const void* segs,
                           const double* q, double2* partial, double* out, uint32_t* small, WsHeader* h, Thr th,
                           cudaStream_t st, const int32_t* qperm, const float* qlo) {
#define X(P, RR, NN)                                                                                      \
  if (PFT_BATCHED_MATCH(P, RR, NN))                                                                      \
    return launch_batched_one<P, RR, NN>(grid, ph, cta_off, items, pplan, info, segs, q, partial, out, small, h, \
                                         th, st, qperm, qlo);
  PFT_BATCHED_CASES(X)
#undef X
  return cudaErrorInvalidConfiguration;
}

thread_local int g_batched_launches = 0;

// Host-side copy of what a batched call needs (kept in the caller's pft_batched_plan).
struct PlanHandle {
  int64_t magic, n_polys, n_verts, n_q, shared_q, fp64, r, nt, grid, n_mc;
  int64_t plan_hdr, cta_off, items, pplan, mc, info, segs, partial, small, total;
  int64_t dim;
  double tau;
  int64_t qperm, qscratch;   // 0: the caller's Q order
};
static_assert(sizeof(PlanHandle) <= sizeof(pft_batched_plan), "plan handle fits the public struct");

size_t workspace_impl(int dim, int64_t n_items, const int64_t* off_host, int64_t n_shapes, const int64_t* q_off_host,
                      int64_t n_q, const pft_options* opts) {
  HostPlan P;
  if (n_items < 0 || build_plan(dim, off_host, n_shapes, q_off_host, n_q, opts, P) != PFT_OK) return 0;
  if (P.h.n_verts != n_items) return 0;
  return layout_of(P.h).total;
}

int prepare_impl(int dim, const int64_t* off_host, int64_t n_shapes, const int64_t* q_off_host, int64_t n_q,
                 void* ws, size_t ws_bytes, const pft_options* opts, pft_batched_plan* plan, void* stream) {
  if (plan == nullptr) return PFT_ERR_INVALID_ARG;
  std::memset(plan, 0, sizeof(*plan));
  HostPlan P;
  if (int e = build_plan(dim, off_host, n_shapes, q_off_host, n_q, opts, P)) return e;
  const BLayout y = layout_of(P.h);
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < y.total) return PFT_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto put = [&](size_t off, const void* src, size_t bytes) {
    return bytes == 0 || cudaMemcpyAsync(at<char>(ws, off), src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  bool ok = put(y.plan_hdr, &P.h, sizeof(P.h)) &&
            put(y.cta_off, P.cta_off.data(), sizeof(int32_t) * P.cta_off.size()) &&
            put(y.items, P.items.data(), sizeof(BItem) * P.items.size()) &&
            put(y.pplan, P.pplan.data(), sizeof(PolyPlan) * P.pplan.size()) &&
            put(y.mc, P.mc.data(), sizeof(int32_t) * P.mc.size());
  ok = ok && cudaStreamSynchronize(st) == cudaSuccess;   // the host vectors die on return
  if (!ok) return PFT_ERR_CUDA;
  PlanHandle ph{};
  ph.magic = (int64_t)kPlanMagic;
  ph.n_polys = n_shapes;
  ph.n_verts = P.h.n_verts;
  ph.n_q = n_q;
  ph.shared_q = P.h.shared_q;
  ph.fp64 = P.h.fp64;
  ph.r = P.h.r;
  ph.nt = P.h.nt;
  ph.grid = P.h.n_cta;
  ph.n_mc = P.h.n_mc;
  ph.plan_hdr = (int64_t)y.plan_hdr; ph.cta_off = (int64_t)y.cta_off; ph.items = (int64_t)y.items;
  ph.pplan = (int64_t)y.pplan; ph.mc = (int64_t)y.mc; ph.info = (int64_t)y.info; ph.segs = (int64_t)y.segs;
  ph.partial = (int64_t)y.partial; ph.small = (int64_t)y.small; ph.total = (int64_t)y.total;
  ph.dim = dim;
  ph.tau = P.h.tau;
  ph.qperm = P.h.q_tiled ? (int64_t)y.qperm : 0;
  ph.qscratch = P.h.q_tiled ? (int64_t)y.qscratch : 0;
  std::memcpy(plan, &ph, sizeof(ph));
  return PFT_OK;
}

// Checks shared by both batched calls; on success fills p and the header pointer.
int check_call(int dim, const pft_batched_plan* plan, int64_t n_items, int64_t n_shapes, int64_t n_q,
               const int64_t* q_off, const void* verts, const int64_t* off, const double* q, double* out, void* ws,
               size_t ws_bytes, PlanHandle& p) {
  if (plan == nullptr) return PFT_ERR_INVALID_ARG;
  std::memcpy(&p, plan, sizeof(p));
  if (p.magic != (int64_t)kPlanMagic || p.dim != dim) return PFT_ERR_INVALID_ARG;
  if (n_items != p.n_verts || n_shapes != p.n_polys || n_q != p.n_q || (q_off == nullptr) != (p.shared_q != 0))
    return PFT_ERR_INVALID_ARG;   // not the shape the plan was prepared for
  if (n_shapes > 0 && (off == nullptr || verts == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_q > 0 && (q == nullptr || out == nullptr)) return PFT_ERR_INVALID_ARG;
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < (size_t)p.total)
    return PFT_ERR_WORKSPACE;
  return PFT_OK;
}

Thr plan_thr(const PlanHandle& p) {
  const float tau = (float)p.tau, lo = std::min(tau, kTauLo);
  return Thr{0.25f * tau * tau, 0.25f * lo * lo, tau > 1.f ? 1 : 0, tau > 3.f ? 1 : 0};
}

// Pair kernel, multi-chunk finish and the small-|Q| pass (the last is dimension-specific).
int run_rest(const PlanHandle& p, void* ws, const double* q, double* out, WsHeader* h, cudaStream_t st) {
  const BPlanHeader* phd = at<BPlanHeader>(ws, (size_t)p.plan_hdr);
  const PolyPlan* pplan = at<PolyPlan>(ws, (size_t)p.pplan);
  PolyInfo* info = at<PolyInfo>(ws, (size_t)p.info);
  uint32_t* small = at<uint32_t>(ws, (size_t)p.small);
  double2* partial = at<double2>(ws, (size_t)p.partial);
  int32_t* qperm = nullptr;
  if (p.qperm != 0) {
    qperm = at<int32_t>(ws, (size_t)p.qperm);
    if (launch_qorder((int)p.dim, q, p.n_q, (int)p.r, (int)p.nt, at<void>(ws, (size_t)p.qscratch), qperm, st,
                      &g_batched_launches) != cudaSuccess)
      return PFT_ERR_CUDA;
  }
  float* qlo = nullptr;
  if (p.fp64 == 0) {   // the last region of the workspace
    qlo = at<float>(ws, (size_t)p.total - qlo_bytes(p.dim, p.n_q));
    const int64_t n = p.dim * p.n_q;
    if (n > 0) {
      k_bqlo<<<(unsigned)((n + kBThreads - 1) / kBThreads), kBThreads, 0, st>>>(q, n, qlo);
      if (cudaGetLastError() != cudaSuccess) return PFT_ERR_CUDA;
      ++g_batched_launches;
    }
  }
  if (launch_batched((int)p.dim, p.fp64 != 0, (int)p.r, (int)p.nt, (int)p.grid, phd,
                     at<int32_t>(ws, (size_t)p.cta_off), at<BItem>(ws, (size_t)p.items), pplan, info,
                     at<void>(ws, (size_t)p.segs), q, partial, out, small, h, plan_thr(p), st, qperm,
                     qlo) != cudaSuccess)
    return PFT_ERR_CUDA;
  ++g_batched_launches;
  if (p.n_mc > 0) {
    k_bfinal<<<(unsigned)p.n_mc, kBThreads, 0, st>>>(phd, at<int32_t>(ws, (size_t)p.mc), pplan, info, q, partial,
                                                      out, small, h, qlo);
    if (cudaGetLastError() != cudaSuccess) return PFT_ERR_CUDA;
    ++g_batched_launches;
  }
  return PFT_OK;
}

int sm_count() {
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, sms);
}

}  // namespace
}  // namespace pft

using namespace pft;

extern "C" {

size_t pft2d_batched_workspace_size(int64_t n_verts, const int64_t* poly_off_host, int64_t n_polys,
                                    const int64_t* q_off_host, int64_t n_q, const pft_options* opts) {
  return workspace_impl(2, n_verts, poly_off_host, n_polys, q_off_host, n_q, opts);
}

int pft2d_batched_prepare(const int64_t* poly_off_host, int64_t n_polys, const int64_t* q_off_host, int64_t n_q,
                          void* ws, size_t ws_bytes, const pft_options* opts, pft_batched_plan* plan,
                          void* stream) {
  return prepare_impl(2, poly_off_host, n_polys, q_off_host, n_q, ws, ws_bytes, opts, plan, stream);
}

int pft2d_polygons_batched(const float* verts, int64_t n_verts, const int64_t* poly_off, int64_t n_polys,
                           const double* q, const int64_t* q_off, int64_t n_q, double* out, void* ws,
                           size_t ws_bytes, const pft_batched_plan* plan, void* stream) {
  g_batched_launches = 0;
  PlanHandle p;
  if (int e = check_call(2, plan, n_verts, n_polys, n_q, q_off, verts, poly_off, q, out, ws, ws_bytes, p)) return e;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* h = at<WsHeader>(ws, 0);
  if (launch_init_header(h, st) != cudaSuccess) return PFT_ERR_CUDA;
  ++g_batched_launches;
  if (n_polys == 0 || n_q == 0) return PFT_OK;
  const BPlanHeader* phd = at<BPlanHeader>(ws, (size_t)p.plan_hdr);
  const PolyPlan* pplan = at<PolyPlan>(ws, (size_t)p.pplan);
  PolyInfo* info = at<PolyInfo>(ws, (size_t)p.info);
  void* segs = at<void>(ws, (size_t)p.segs);
  if (p.fp64) k_bprep<true><<<(unsigned)n_polys, kBThreads, 0, st>>>(verts, poly_off, phd, pplan, info, segs, h);
  else k_bprep<false><<<(unsigned)n_polys, kBThreads, 0, st>>>(verts, poly_off, phd, pplan, info, segs, h);
  if (cudaGetLastError() != cudaSuccess) return PFT_ERR_CUDA;
  ++g_batched_launches;
  if (int e = run_rest(p, ws, q, out, h, st)) return e;
  k_bsmall<<<sm_count(), kBThreads, 0, st>>>(verts, phd, pplan, info, q_off, q, at<uint32_t>(ws, (size_t)p.small),
                                              out, h);
  if (cudaGetLastError() != cudaSuccess) return PFT_ERR_CUDA;
  ++g_batched_launches;
  return PFT_OK;
}

size_t pft3d_batched_workspace_size(int64_t n_faces, const int64_t* mesh_off_host, int64_t n_meshes,
                                    const int64_t* q_off_host, int64_t n_q, const pft_options* opts) {
  return workspace_impl(3, n_faces, mesh_off_host, n_meshes, q_off_host, n_q, opts);
}

int pft3d_batched_prepare(const int64_t* mesh_off_host, int64_t n_meshes, const int64_t* q_off_host, int64_t n_q,
                          void* ws, size_t ws_bytes, const pft_options* opts, pft_batched_plan* plan,
                          void* stream) {
  return prepare_impl(3, mesh_off_host, n_meshes, q_off_host, n_q, ws, ws_bytes, opts, plan, stream);
}

int pft3d_meshes_batched(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
                         const int64_t* mesh_off, int64_t n_meshes, const double* q, const int64_t* q_off,
                         int64_t n_q, double* out, void* ws, size_t ws_bytes, const pft_batched_plan* plan,
                         void* stream) {
  g_batched_launches = 0;
  PlanHandle p;
  if (int e = check_call(3, plan, n_faces, n_meshes, n_q, q_off, verts, mesh_off, q, out, ws, ws_bytes, p)) return e;
  if (n_verts < 0 || (n_faces > 0 && (faces == nullptr || n_verts == 0))) return PFT_ERR_INVALID_ARG;
  if (n_verts > INT32_MAX) return PFT_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* h = at<WsHeader>(ws, 0);
  if (launch_init_header(h, st) != cudaSuccess) return PFT_ERR_CUDA;
  ++g_batched_launches;
  if (n_meshes == 0 || n_q == 0) return PFT_OK;
  const BPlanHeader* phd = at<BPlanHeader>(ws, (size_t)p.plan_hdr);
  const PolyPlan* pplan = at<PolyPlan>(ws, (size_t)p.pplan);
  PolyInfo* info = at<PolyInfo>(ws, (size_t)p.info);
  void* recs = at<void>(ws, (size_t)p.segs);
  if (p.fp64)
    k_bprep3<true><<<(unsigned)n_meshes, kBThreads, 0, st>>>(verts, n_verts, faces, mesh_off, phd, pplan, info, recs, h);
  else
    k_bprep3<false><<<(unsigned)n_meshes, kBThreads, 0, st>>>(verts, n_verts, faces, mesh_off, phd, pplan, info, recs,
                                                              h);
  if (cudaGetLastError() != cudaSuccess) return PFT_ERR_CUDA;
  ++g_batched_launches;
  if (int e = run_rest(p, ws, q, out, h, st)) return e;
  k_bsmall3<<<sm_count(), kBThreads, 0, st>>>(verts, n_verts, faces, phd, pplan, info, q_off, q,
                                              at<uint32_t>(ws, (size_t)p.small), out, h);
  if (cudaGetLastError() != cudaSuccess) return PFT_ERR_CUDA;
  ++g_batched_launches;
  return PFT_OK;
}

int pft_batched_last_launch_count(void) { return g_batched_launches; }

}  // extern "C"
