// pft_selftest.cu -- a self-test of the bounded mbarrier wait and of the status word.
//
// Every wait of the library's kernels on an mbarrier polls a bounded number of
// times; when the phase never completes, the kernel sets the timeout bit of the
// status word at the start of the workspace and the block leaves, so the
// context stays usable and the host learns of it through pft_status().  In
// correct use no wait runs out, so this entry point exercises that path on
// purpose: one block initialises an mbarrier that nothing arrives on and polls
// it `polls` times (arrive = 0), or arrives on it first and then waits
// (arrive = 1, the phase completes and the status stays clear).  The paper has
// no counterpart; it is a check of the failure handling around the copies.
#include "pft_kernels.cuh"

namespace pft {
namespace {

__global__ void k_wait_selftest(uint32_t* status, uint32_t polls, int arrive) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (arrive) mbar_arrive(&bar);   // the one expected arrival: phase 0 completes
  bool done = false;
  for (uint32_t i = 0; i < polls && !done; ++i) done = mbar_try_wait(&bar, 0u);
  if (!done) set_status(status, ST_TIMEOUT);
}

}  // namespace
}  // namespace pft

extern "C" int pft_selftest_wait(void* ws, size_t ws_bytes, uint32_t polls, int arrive, void* stream) {
  using namespace pft;
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < sizeof(WsHeader))
    return PFT_ERR_WORKSPACE;
  if (polls == 0 || polls > (1u << 20) || (arrive != 0 && arrive != 1)) return PFT_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(ws, 0, sizeof(WsHeader), st) != cudaSuccess) return PFT_ERR_CUDA;
  k_wait_selftest<<<1, 32, 0, st>>>(static_cast<uint32_t*>(ws), polls, arrive);
  return cudaGetLastError() == cudaSuccess ? PFT_OK : PFT_ERR_CUDA;
}
