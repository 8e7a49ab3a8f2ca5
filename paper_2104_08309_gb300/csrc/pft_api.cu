// pft_api.cu -- the C ABI (include/pft.h): argument checks, workspace layout,
// launch planning and the kernel sequence of each call.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <vector>

#include "pft_kernels.cuh"

namespace pft {
namespace {

thread_local int g_last_launches = 0;

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Opts {
  bool fp64;
  int r, nt, k_splits;
  float tau;
  cudaEvent_t ev_start, ev_stop;
  int64_t face_pairs;
  int q_order;
};

int resolve(const pft_options* o, int dim, Opts& out) {
  pft_options z;
  std::memset(&z, 0, sizeof(z));
  const pft_options& p = o ? *o : z;
  if (p.precision != PFT_FP32_COMPENSATED && p.precision != PFT_FP64) return PFT_ERR_INVALID_ARG;
  out.fp64 = (p.precision == PFT_FP64);
  out.r = p.q_per_thread ? p.q_per_thread : (out.fp64 ? 1 : 4);
  out.nt = p.block_threads ? p.block_threads : ((out.fp64 || dim == 3) ? 128 : 256);
  const bool r_ok = out.fp64 ? (out.r == 1 || out.r == 2) : (out.r == 1 || out.r == 2 || out.r == 4 || out.r == 8);
  if (!r_ok || (out.nt != 128 && out.nt != 256)) return PFT_ERR_UNSUPPORTED;
  if (p.k_splits < 0) return PFT_ERR_INVALID_ARG;
  out.k_splits = p.k_splits;
  if (p.tile_items != 0) return PFT_ERR_UNSUPPORTED;
  float tau = p.face_series_tau;
  if (tau == 0.f) tau = 6.0f;
  if (!(tau > 0.f && tau <= 6.0f)) return PFT_ERR_INVALID_ARG;
  out.tau = tau;
  out.ev_start = static_cast<cudaEvent_t>(p.main_start_event);
  out.ev_stop = static_cast<cudaEvent_t>(p.main_stop_event);
  if (p.face_pairs < 0) return PFT_ERR_INVALID_ARG;
  if (p.face_pairs > 0 && dim == 3 && !out.fp64 && out.r > 4) return PFT_ERR_UNSUPPORTED;
  out.face_pairs = dim == 3 ? p.face_pairs : 0;
  if (p.q_order != PFT_Q_TILED && p.q_order != PFT_Q_AS_GIVEN) return PFT_ERR_INVALID_ARG;
  out.q_order = p.q_order;
  return PFT_OK;
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

// Split-K choice: the smallest number of chunks that fills the GPU in whole
// waves (the last wave >= 97 % as full as the others), each chunk at least two
// tiles long; then, for launches of fewer than 40 waves with chunks to spare,
// more chunks (below).
FwdLaunch plan_fwd(int dim, const Opts& o, int64_t n_items, int64_t n_q) {
  FwdLaunch L{};
  L.r = o.r;
  L.nt = o.nt;
  const int tile = fwd_tile(dim, o.fp64);
  const int64_t q_per_block = (int64_t)o.r * o.nt;
  L.q_tiles = std::max<int64_t>(1, (n_q + q_per_block - 1) / q_per_block);
  const int64_t item_tiles = std::max<int64_t>(1, (n_items + tile - 1) / tile);
  int k = o.k_splits;
  if (k == 0) {
    const int64_t slots = (int64_t)device_sms() * fwd_blocks_per_sm(dim, o.fp64, o.r, o.nt, o.face_pairs > 0);
    const int kmax = (int)std::max<int64_t>(1, std::min<int64_t>(64, item_tiles / 2));
    double best_eff = -1.0;
    int best_k = 1;
    k = 0;
    for (int c = 1; c <= kmax; ++c) {
      const double waves = (double)(L.q_tiles * c) / (double)slots;
      const double eff = waves / std::ceil(waves);
      if (L.q_tiles * c >= slots && eff >= 0.97) { k = c; break; }
      if (eff > best_eff + 1e-9) { best_eff = eff; best_k = c; }
    }
    if (k == 0) k = best_k;
    // Long launches: more chunks, up to about 40 waves (chunks of at least 4,096 faces or 8,192
    // segments, the last wave still >= 97 % full).  Blocks do not finish in waves: the resident
    // blocks of an SM share it unevenly, and the last blocks to start leave SMs partly idle for about
    // a third of a block's run (a 1.3M-face mesh on 2M Q points: 10.8 waves lost 2 % of the launch
    // against 43).
    const int kw_max = (int)std::min<int64_t>(64, n_items / (dim == 3 ? 4096 : 8192));
    if ((double)(L.q_tiles * k) / (double)slots < 40.0) {
      for (int c = k + 1; c <= kw_max; ++c) {
        const double waves = (double)(L.q_tiles * c) / (double)slots;
        if (waves / std::ceil(waves) < 0.97) continue;
        k = c;
        if (waves >= 40.0) break;
      }
    }
  }
  k = (int)std::min<int64_t>(k, item_tiles);
  const int64_t tiles_per = (item_tiles + k - 1) / k;
  L.per_split = tiles_per * tile;
  L.k_splits = (int)((item_tiles + tiles_per - 1) / tiles_per);
  return L;
}

struct FwdLayout {
  size_t mparts, items, partial, small, qperm, qscratch, total;
  int nblk;
  bool tiled;   // the main kernel visits the Q points in the library's order (q_order option)
  FwdLaunch L;
};

FwdLayout layout_fwd(int dim, const Opts& o, int64_t n_items, int64_t n_prep, int64_t n_q) {
  FwdLayout y{};
  y.L = plan_fwd(dim, o, n_items, n_q);
  y.nblk = std::max(1, prep_blocks(n_prep));
  const size_t item_bytes = dim == 2 ? (o.fp64 ? sizeof(Seg64) : sizeof(Seg32)) : (o.fp64 ? sizeof(Face64) : sizeof(Face32));
  size_t off = align_up(sizeof(WsHeader));
  y.mparts = off;  off = align_up(off + sizeof(double) * (size_t)y.nblk);
  y.items = off;   off = align_up(off + item_bytes * (size_t)std::max<int64_t>(n_items, 1));
  y.partial = off; off = align_up(off + sizeof(double2) * (size_t)y.L.k_splits * (size_t)std::max<int64_t>(n_q, 1));
  y.small = off;   off = align_up(off + sizeof(int32_t) * (size_t)std::max<int64_t>(n_q, 1));
  y.tiled = o.q_order == PFT_Q_TILED && qorder_wanted(n_q, n_items, o.r, o.nt);
  if (y.tiled) {
    y.qperm = off;    off = align_up(off + sizeof(int32_t) * (size_t)n_q);
    y.qscratch = off; off = align_up(off + qorder_layout(n_q).total);
  }
  y.total = off;
  return y;
}


template <typename T>
T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

bool bad_ws(const void* ws, size_t bytes, size_t need) {
  return ws == nullptr || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0 || bytes < need;
}

// The slot -> Q map of the main kernel (NULL: the caller's order), computed on the stream.
int fwd_qorder(int dim, const FwdLayout& y, const double* q, int64_t n_q, void* ws, cudaStream_t st,
               const int32_t*& qperm) {
  qperm = nullptr;
  if (!y.tiled) return PFT_OK;
  int32_t* perm = at<int32_t>(ws, y.qperm);
  if (launch_qorder(dim, q, n_q, y.L.r, y.L.nt, at<void>(ws, y.qscratch), perm, st, &g_last_launches) != cudaSuccess)
    return PFT_ERR_CUDA;
  qperm = perm;
  return PFT_OK;
}

// Records an optional caller event on the stream (timing of the main kernel alone).
inline cudaError_t mark(cudaEvent_t ev, cudaStream_t st) { return ev ? cudaEventRecord(ev, st) : cudaSuccess; }

#define PFT_LAUNCH(expr)                        \
  do {                                          \
    if ((expr) != cudaSuccess) return PFT_ERR_CUDA; \
    ++g_last_launches;                          \
  } while (0)

}  // namespace
}  // namespace pft

using namespace pft;

extern "C" {

size_t pft2d_workspace_size(int64_t n_verts, int64_t n_loops, int64_t n_q, const pft_options* opts) {
  Opts o;
  if (n_verts < 0 || n_loops < 0 || n_q < 0 || resolve(opts, 2, o) != PFT_OK) return 0;
  return layout_fwd(2, o, n_verts, std::max<int64_t>(n_verts, n_loops + 1), n_q).total;
}

size_t pft3d_workspace_size(int64_t n_verts, int64_t n_faces, int64_t n_q, const pft_options* opts) {
  Opts o;
  if (n_verts < 0 || n_faces < 0 || n_q < 0 || resolve(opts, 3, o) != PFT_OK) return 0;
  return layout_fwd(3, o, n_faces, n_faces, n_q).total;
}

int pft2d_polygons(const float* verts, int64_t n_verts, const int64_t* loop_off, int64_t n_loops, const double* q,
                   int64_t n_q, double* out, void* ws, size_t ws_bytes, const pft_options* opts, void* stream) {
  g_last_launches = 0;
  Opts o;
  if (int e = resolve(opts, 2, o)) return e;
  if (n_verts < 0 || n_loops < 0 || n_q < 0) return PFT_ERR_INVALID_ARG;
  if (n_q > 0 && (q == nullptr || out == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_verts > 0 && (verts == nullptr || loop_off == nullptr || n_loops == 0)) return PFT_ERR_INVALID_ARG;
  if (n_q > INT32_MAX) return PFT_ERR_UNSUPPORTED;
  const FwdLayout y = layout_fwd(2, o, n_verts, std::max<int64_t>(n_verts, n_loops + 1), n_q);
  if (bad_ws(ws, ws_bytes, y.total)) return PFT_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* h = at<WsHeader>(ws, 0);
  PFT_LAUNCH(launch_init_header(h, st));
  if (n_q == 0) return PFT_OK;
  if (n_verts == 0) {
    if (cudaMemsetAsync(out, 0, sizeof(double) * 2 * (size_t)n_q, st) != cudaSuccess) return PFT_ERR_CUDA;
    return PFT_OK;
  }
  double* mp = at<double>(ws, y.mparts);
  PFT_LAUNCH(launch_bbox(verts, n_verts, 2, h, st));
  PFT_LAUNCH(launch_prep2d(verts, n_verts, loop_off, n_loops, h, at<void>(ws, y.items), o.fp64, mp, y.nblk, st));
  const int32_t* qperm;
  if (int e = fwd_qorder(2, y, q, n_q, ws, st, qperm)) return e;
  if (mark(o.ev_start, st) != cudaSuccess) return PFT_ERR_CUDA;
  PFT_LAUNCH(launch_fwd(2, o.fp64, y.L, at<void>(ws, y.items), n_verts, q, n_q, o.tau, at<double2>(ws, y.partial),
                        &h->status, st, 0, qperm));
  if (mark(o.ev_stop, st) != cudaSuccess) return PFT_ERR_CUDA;
  PFT_LAUNCH(launch_finalize(2, q, n_q, at<double2>(ws, y.partial), y.L.k_splits, o.fp64, h, mp, y.nblk,
                             at<int32_t>(ws, y.small), out, st));
  PFT_LAUNCH(launch_smallq2d(verts, n_verts, loop_off, n_loops, q, o.fp64, h, at<int32_t>(ws, y.small), out, st));
  return PFT_OK;
}

int pft3d_mesh(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces, const double* q,
               int64_t n_q, double* out, void* ws, size_t ws_bytes, const pft_options* opts, void* stream) {
  g_last_launches = 0;
  Opts o;
  if (int e = resolve(opts, 3, o)) return e;
  if (n_verts < 0 || n_faces < 0 || n_q < 0) return PFT_ERR_INVALID_ARG;
  if (n_q > 0 && (q == nullptr || out == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_faces > 0 && (faces == nullptr || verts == nullptr || n_verts == 0)) return PFT_ERR_INVALID_ARG;
  if (n_q > INT32_MAX || n_verts > INT32_MAX) return PFT_ERR_UNSUPPORTED;
  if (2 * o.face_pairs > n_faces) return PFT_ERR_INVALID_ARG;
  const FwdLayout y = layout_fwd(3, o, n_faces, n_faces, n_q);
  if (bad_ws(ws, ws_bytes, y.total)) return PFT_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* h = at<WsHeader>(ws, 0);
  PFT_LAUNCH(launch_init_header(h, st));
  if (n_q == 0) return PFT_OK;
  if (n_faces == 0) {
    if (cudaMemsetAsync(out, 0, sizeof(double) * 2 * (size_t)n_q, st) != cudaSuccess) return PFT_ERR_CUDA;
    return PFT_OK;
  }
  double* mp = at<double>(ws, y.mparts);
  PFT_LAUNCH(launch_bbox(verts, n_verts, 3, h, st));
  PFT_LAUNCH(launch_prep3d(verts, n_verts, faces, n_faces, h, at<void>(ws, y.items), o.fp64, mp, y.nblk, st,
                           2 * o.face_pairs));
  const int32_t* qperm;
  if (int e = fwd_qorder(3, y, q, n_q, ws, st, qperm)) return e;
  if (mark(o.ev_start, st) != cudaSuccess) return PFT_ERR_CUDA;
  PFT_LAUNCH(launch_fwd(3, o.fp64, y.L, at<void>(ws, y.items), n_faces, q, n_q, o.tau, at<double2>(ws, y.partial),
                        &h->status, st, 2 * o.face_pairs, qperm));
  if (mark(o.ev_stop, st) != cudaSuccess) return PFT_ERR_CUDA;
  PFT_LAUNCH(launch_finalize(3, q, n_q, at<double2>(ws, y.partial), y.L.k_splits, o.fp64, h, mp, y.nblk,
                             at<int32_t>(ws, y.small), out, st));
  PFT_LAUNCH(launch_smallq3d(verts, n_verts, faces, n_faces, q, o.fp64, h, at<int32_t>(ws, y.small), out, st));
  return PFT_OK;
}

size_t pft3d_polymesh_workspace_size(int64_t n_verts, int64_t n_idx, int64_t n_faces, int64_t n_q,
                                     const pft_options* opts) {
  Opts o;
  if (n_verts < 0 || n_idx < 0 || n_faces < 0 || n_q < 0 || n_idx < 3 * n_faces || resolve(opts, 3, o) != PFT_OK)
    return 0;
  const int64_t n_tris = n_idx - 2 * n_faces;
  return layout_fwd(3, o, n_tris, n_tris, n_q).total + align_up(sizeof(int32_t) * 3 * (size_t)std::max<int64_t>(n_tris, 1));
}

int pft3d_polymesh(const float* verts, int64_t n_verts, const int32_t* face_idx, int64_t n_idx,
                   const int64_t* face_off, int64_t n_faces, const double* q, int64_t n_q, double* out,
                   void* ws, size_t ws_bytes, const pft_options* opts, void* stream) {
  g_last_launches = 0;
  Opts o;
  if (int e = resolve(opts, 3, o)) return e;
  if (n_verts < 0 || n_idx < 0 || n_faces < 0 || n_q < 0 || n_idx < 3 * n_faces) return PFT_ERR_INVALID_ARG;
  if (n_q > 0 && (q == nullptr || out == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_faces > 0 && (face_idx == nullptr || face_off == nullptr || verts == nullptr || n_verts == 0))
    return PFT_ERR_INVALID_ARG;
  if (n_q > INT32_MAX || n_verts > INT32_MAX) return PFT_ERR_UNSUPPORTED;
  const int64_t n_tris = n_idx - 2 * n_faces;
  const FwdLayout y = layout_fwd(3, o, n_tris, n_tris, n_q);
  const size_t tri_off = y.total;
  if (bad_ws(ws, ws_bytes, tri_off + align_up(sizeof(int32_t) * 3 * (size_t)std::max<int64_t>(n_tris, 1))))
    return PFT_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* h = at<WsHeader>(ws, 0);
  PFT_LAUNCH(launch_init_header(h, st));
  if (n_q == 0) return PFT_OK;
  if (n_faces == 0) {
    if (cudaMemsetAsync(out, 0, sizeof(double) * 2 * (size_t)n_q, st) != cudaSuccess) return PFT_ERR_CUDA;
    return PFT_OK;
  }
  int32_t* tris = at<int32_t>(ws, tri_off);
  double* mp = at<double>(ws, y.mparts);
  PFT_LAUNCH(launch_fan3d(face_idx, n_idx, face_off, n_faces, tris, n_tris, h, st));
  PFT_LAUNCH(launch_bbox(verts, n_verts, 3, h, st));
  PFT_LAUNCH(launch_prep3d(verts, n_verts, tris, n_tris, h, at<void>(ws, y.items), o.fp64, mp, y.nblk, st));
  const int32_t* qperm;
  if (int e = fwd_qorder(3, y, q, n_q, ws, st, qperm)) return e;
  if (mark(o.ev_start, st) != cudaSuccess) return PFT_ERR_CUDA;
  PFT_LAUNCH(launch_fwd(3, o.fp64, y.L, at<void>(ws, y.items), n_tris, q, n_q, o.tau, at<double2>(ws, y.partial),
                        &h->status, st, 0, qperm));
  if (mark(o.ev_stop, st) != cudaSuccess) return PFT_ERR_CUDA;
  PFT_LAUNCH(launch_finalize(3, q, n_q, at<double2>(ws, y.partial), y.L.k_splits, o.fp64, h, mp, y.nblk,
                             at<int32_t>(ws, y.small), out, st));
  PFT_LAUNCH(launch_smallq3d(verts, n_verts, tris, n_tris, q, o.fp64, h, at<int32_t>(ws, y.small), out, st));
  return PFT_OK;
}

int pft_status(const void* ws, void* stream) {
  if (ws == nullptr) return PFT_ERR_INVALID_ARG;
  uint32_t word = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&word, ws, sizeof(word), cudaMemcpyDeviceToHost, st) != cudaSuccess) return PFT_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PFT_ERR_CUDA;
  if (word & ST_INDEX) return PFT_ERR_INDEX_RANGE;
  if (word & ST_NONFINITE) return PFT_ERR_NONFINITE;
  if (word & ST_OFFSETS) return PFT_ERR_OFFSETS;
  if (word & ST_PAIRS) return PFT_ERR_PAIRS;
  if (word & ST_TIMEOUT) return PFT_ERR_TIMEOUT;
  return PFT_OK;
}

const char* pft_status_string(int code) {
  switch (code) {
    case PFT_OK: return "ok";
    case PFT_ERR_INVALID_ARG: return "invalid argument";
    case PFT_ERR_INDEX_RANGE: return "face index out of range";
    case PFT_ERR_NONFINITE: return "non-finite vertex coordinate";
    case PFT_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case PFT_ERR_CUDA: return "CUDA launch or copy failed";
    case PFT_ERR_TIMEOUT: return "bounded wait on a bulk copy timed out";
    case PFT_ERR_UNSUPPORTED: return "unsupported option combination";
    case PFT_ERR_OFFSETS: return "malformed CSR offsets";
    case PFT_ERR_SCRATCH_LIMIT: return "problem exceeds the 32 MiB static scratch of pft3d_mesh_noalloc";
    case PFT_ERR_PAIRS: return "faces given as pairs do not share their first edge";
    default: return "unknown status code";
  }
}

size_t pft_q_order_workspace_size(int64_t n_q) {
  if (n_q < 0 || n_q > INT32_MAX) return 0;
  return qorder_layout(n_q).total;
}

int pft_q_order(const double* q, int64_t n_q, int dim, int q_per_thread, int block_threads, int32_t* perm, void* ws,
                size_t ws_bytes, void* stream) {
  g_last_launches = 0;
  if (n_q < 0 || (dim != 2 && dim != 3)) return PFT_ERR_INVALID_ARG;
  if (n_q > INT32_MAX) return PFT_ERR_UNSUPPORTED;
  const int r = q_per_thread, nt = block_threads;
  if (!(r == 1 || r == 2 || r == 4 || r == 8) || (nt != 128 && nt != 256 && nt != 512)) return PFT_ERR_UNSUPPORTED;
  if (n_q == 0) return PFT_OK;
  if (q == nullptr || perm == nullptr) return PFT_ERR_INVALID_ARG;
  if (bad_ws(ws, ws_bytes, qorder_layout(n_q).total)) return PFT_ERR_WORKSPACE;
  return launch_qorder(dim, q, n_q, r, nt, ws, perm, static_cast<cudaStream_t>(stream), &g_last_launches) ==
                 cudaSuccess
             ? PFT_OK
             : PFT_ERR_CUDA;
}

int pft3d_pair_faces(const int32_t* f, int64_t nf, int32_t* out, int64_t* n_pairs) {
  if (nf < 0 || n_pairs == nullptr || (nf > 0 && (f == nullptr || out == nullptr || f == out)))
    return PFT_ERR_INVALID_ARG;
  for (int64_t i = 0; i < 3 * nf; ++i)
    if (f[i] < 0) return PFT_ERR_INVALID_ARG;
  // undirected edge -> the first two (face, slot) that hold it, and how many faces do
  struct Uses {
    int64_t face[2];
    int8_t slot[2];
    int32_t count;
  };
  auto key = [](uint32_t u, uint32_t v) {
    return u < v ? ((uint64_t)u << 32) | v : ((uint64_t)v << 32) | u;
  };
  std::unordered_map<uint64_t, Uses> edges;
  edges.reserve((size_t)(3 * nf / 2 + 1));
  for (int64_t m = 0; m < nf; ++m)
    for (int l = 0; l < 3; ++l) {
      Uses& e = edges[key((uint32_t)f[3 * m + l], (uint32_t)f[3 * m + (l + 1) % 3])];
      if (e.count < 2) {
        e.face[e.count] = m;
        e.slot[e.count] = (int8_t)l;
      }
      ++e.count;
    }
  // pairable neighbours: faces that hold a common edge (of exactly two faces) the other way round
  std::vector<int64_t> nb((size_t)(3 * nf), -1);
  std::vector<int8_t> nb_slot((size_t)(3 * nf), 0);
  for (int64_t m = 0; m < nf; ++m)
    for (int l = 0; l < 3; ++l) {
      const int32_t u = f[3 * m + l], v = f[3 * m + (l + 1) % 3];
      if (u == v) continue;
      const Uses& e = edges.at(key((uint32_t)u, (uint32_t)v));
      if (e.count != 2) continue;
      const int j = (e.face[0] == m && e.slot[0] == l) ? 1 : 0;
      const int64_t o = e.face[j];
      const int lo = e.slot[j];
      if (o == m || f[3 * o + lo] != v || f[3 * o + (lo + 1) % 3] != u) continue;
      nb[(size_t)(3 * m + l)] = o;
      nb_slot[(size_t)(3 * m + l)] = (int8_t)lo;
    }
  // maximum-cardinality-seeking matching (Karp-Sipser): a face with one free neighbour is matched
  // to it first; otherwise the lowest-numbered free face with a free neighbour is matched to its
  // first free neighbour.  Deterministic.
  std::vector<int64_t> partner((size_t)nf, -1);
  std::vector<int8_t> first((size_t)nf, 0);
  std::vector<int8_t> deg((size_t)nf, 0);
  for (int64_t m = 0; m < nf; ++m)
    for (int l = 0; l < 3; ++l) deg[(size_t)m] += nb[(size_t)(3 * m + l)] >= 0;
  std::vector<int64_t> ones;
  for (int64_t m = nf - 1; m >= 0; --m)
    if (deg[(size_t)m] == 1) ones.push_back(m);
  auto match = [&](int64_t m, int l) {
    const int64_t o = nb[(size_t)(3 * m + l)];
    partner[(size_t)m] = o;
    partner[(size_t)o] = m;
    first[(size_t)m] = (int8_t)l;
    first[(size_t)o] = nb_slot[(size_t)(3 * m + l)];
    for (const int64_t x : {m, o})
      for (int c = 0; c < 3; ++c) {
        const int64_t y = nb[(size_t)(3 * x + c)];
        if (y >= 0 && partner[(size_t)y] < 0 && --deg[(size_t)y] == 1) ones.push_back(y);
      }
  };
  auto free_slot = [&](int64_t m) {
    for (int l = 0; l < 3; ++l) {
      const int64_t o = nb[(size_t)(3 * m + l)];
      if (o >= 0 && partner[(size_t)o] < 0) return l;
    }
    return -1;
  };
  int64_t scan = 0;
  for (;;) {
    int64_t m = -1;
    while (!ones.empty() && m < 0) {
      const int64_t c = ones.back();
      ones.pop_back();
      if (partner[(size_t)c] < 0 && free_slot(c) >= 0) m = c;
    }
    while (m < 0 && scan < nf) {
      if (partner[(size_t)scan] < 0 && free_slot(scan) >= 0) m = scan;
      ++scan;
    }
    if (m < 0) break;
    match(m, free_slot(m));
  }
  int64_t k = 0;
  auto put = [&](int64_t dst, int64_t m, int l) {
    for (int c = 0; c < 3; ++c) out[3 * dst + c] = f[3 * m + (l + c) % 3];
  };
  for (int64_t m = 0; m < nf; ++m)
    if (partner[(size_t)m] > m) {
      put(2 * k, m, first[(size_t)m]);
      put(2 * k + 1, partner[(size_t)m], first[(size_t)partner[(size_t)m]]);
      ++k;
    }
  int64_t w = 2 * k;
  for (int64_t m = 0; m < nf; ++m)
    if (partner[(size_t)m] < 0) put(w++, m, 0);
  *n_pairs = k;
  return PFT_OK;
}

int pft_version(void) { return 10000 * 0 + 100 * 1 + 0; }

int pft_last_launch_count(void) { return g_last_launches; }

}  // extern "C"
