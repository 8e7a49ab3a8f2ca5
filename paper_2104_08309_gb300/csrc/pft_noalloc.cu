// pft_noalloc.cu -- pft3d_mesh for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they need a transform: code that runs while a CUDA stream is being
// captured into a graph (allocation is not a capturable operation), plug-ins
// hosted by an application that owns every device allocation and hands out no
// scratch, and real-time loops that forbid allocation after start-up.  For them
// this file keeps the scratch space of pft3d_mesh in a fixed, file-scope device
// array instead of a caller-supplied workspace.
//
// Costs and rules:
//  - Every GPU that loads this module holds kScratchBytes of device memory for
//    the scratch array until the process exits.
//  - All calls on a device share the one array, and it keeps the last call's
//    contents.  Calls whose GPU work overlaps (other streams, other host threads)
//    race on it and corrupt each other's results: serialise them.
//  - The first call on each device looks up the array's device address with
//    cudaGetSymbolAddress (with that device current) and caches it; make that
//    first call before any stream capture begins.  Every later call made while
//    its stream is not capturing looks the address up again, so that a context
//    torn down and recreated (cudaDeviceReset) is picked up; a call made during
//    capture uses the cached address, which such a reset in between would leave
//    stale.
#include <mutex>

#include "pft_kernels.cuh"

namespace pft {
namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB per device
constexpr int kMaxDevices = 64;

// The scratch array.  In host code this name is only a stand-in for the device
// symbol, never a usable address: the address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  Outside stream capture it
// is looked up afresh (cheap, and right after a context reset); during capture
// the address cached by an earlier call is used.
int scratch_address(cudaStream_t st, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PFT_ERR_CUDA;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    (void)cudaGetLastError();   // not decidable (e.g. legacy stream under global capture): use the cache
    cs = cudaStreamCaptureStatusActive;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[dev] == nullptr || cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return PFT_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return PFT_OK;
}

}  // namespace
}  // namespace pft

extern "C" int pft3d_mesh_noalloc(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
                                  const double* q, int64_t n_q, double* out, const pft_options* opts,
                                  void* stream) {
  const size_t need = pft3d_workspace_size(n_verts, n_faces, n_q, opts);
  // Sizes or options that pft3d_workspace_size rejects: pft3d_mesh refuses them
  // before it looks at the workspace, with the code it would give any caller.
  if (need == 0) return pft3d_mesh(verts, n_verts, faces, n_faces, q, n_q, out, nullptr, 0, opts, stream);
  if (need > pft::kScratchBytes) return PFT_ERR_SCRATCH_LIMIT;
  void* scratch = nullptr;
  if (int e = pft::scratch_address(static_cast<cudaStream_t>(stream), &scratch)) return e;
  // The header at the start of the scratch (status word, counters, bounding box)
  // is re-initialised on the GPU by every call before anything reads it.
  return pft3d_mesh(verts, n_verts, faces, n_faces, q, n_q, out, scratch, pft::kScratchBytes, opts, stream);
}
