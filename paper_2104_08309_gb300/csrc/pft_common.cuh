// pft_common.cuh -- device helpers shared by the libpft kernels (sm_103a).
//
// Status word, FP32 phase and sinc evaluation, compensated accumulation, and the
// bulk-copy (TMA, cp.async.bulk) + mbarrier pipeline used to stage segment and
// face tiles into shared memory.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pft.h"

namespace pft {

// ---------------------------------------------------------------------------
// Status word (first 4 bytes of the workspace): one bit per error class.
// ---------------------------------------------------------------------------
enum : uint32_t {
  ST_INDEX = 1u << 0,
  ST_NONFINITE = 1u << 1,
  ST_TIMEOUT = 1u << 2,
  ST_OFFSETS = 1u << 3,
  ST_PAIRS = 1u << 4,
};

__device__ __forceinline__ void set_status(uint32_t* st, uint32_t bit) { atomicOr(st, bit); }

// Bound on mbarrier polls before a wait is declared lost (~seconds at most).
constexpr uint32_t kWaitLimit = 1u << 22;

// ---------------------------------------------------------------------------
// Workspace header (256 bytes), filled by the prep kernels.
// ---------------------------------------------------------------------------
struct WsHeader {
  uint32_t status;
  uint32_t small_q_count;   // number of Q points routed to the FP64 small-|Q| pass
  uint32_t bbox_enc[6];     // order-preserving encodings: min x,y,z then max x,y,z
  uint32_t rmax_bits;       // max |v - c| as float bits (non-negative floats order as ints)
  uint32_t pad0;
  double center[3];         // bounding-box midpoint c (all coordinates are taken relative to c)
  double measure;           // area (2D) or volume (3D), FP64, fixed-order sum
  uint8_t pad[256 - 4 * 10 - 8 * 4];
};
static_assert(sizeof(WsHeader) == 256, "header must stay 256 bytes");

// Order-preserving float <-> uint32 map (for exact atomic min/max).
__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// ---------------------------------------------------------------------------
// FP32 arithmetic helpers.
// ---------------------------------------------------------------------------
constexpr float kTwoPi = 6.28318530717958647692f;
constexpr float kInvTwoPi = 0.15915494309189533577f;

// 1/x on the SFU (rcp.approx: about 1 ulp; x is never a denormal here).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// exp(2 pi i t) for a phase t given in turns.  t - rint(t) is exact in FP32, so
// the reduction adds no error; sin/cos then run on the SFU over [-pi, pi].
__device__ __forceinline__ void sincos_turns(float t, float* s, float* c) {
  float r = t - rintf(t);
  __sincosf(kTwoPi * r, s, c);
}

// Scalar (float) and packed (float2: two values in one register pair) arithmetic.  The packed
// forms are the sm_100+ paired FP32 instructions (one issue slot for two fused multiply-adds,
// each rounded as fmaf), so a function written once with these helpers gives bit-identical
// results in either form.
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
template <class V> __device__ __forceinline__ V vs(float c);
template <> __device__ __forceinline__ float vs<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 vs<float2>(float c) { return make_float2(c, c); }
// Element r of a thread's R per-Q values, stored as R floats or, for even R, as R/2 float2 pairs.
__device__ __forceinline__ float& el(float* a, int r) { return a[r]; }
__device__ __forceinline__ float& el(float2* a, int r) { return (r & 1) ? a[r >> 1].y : a[r >> 1].x; }
__device__ __forceinline__ float el(const float* a, int r) { return a[r]; }
__device__ __forceinline__ float el(const float2* a, int r) { return (r & 1) ? a[r >> 1].y : a[r >> 1].x; }

// sinc(u) = sin(u)/u from v = u^2 <= pi^2: the degree-6 polynomial in v that
// interpolates sinc(sqrt(v)) at the 7 Chebyshev nodes of [0, pi^2] (our own fit;
// max abs error 7.5e-10 in exact arithmetic, ~1.6e-7 after FP32 rounding, the
// same as the 8-term Taylor series it replaces at two fewer FMAs).
template <class V>
__device__ __forceinline__ V sinc_poly_v(V u2) {
  V p = vfma(u2, vs<V>(1.361159657e-10f), vs<V>(-2.472836691e-8f));
  p = vfma(u2, p, vs<V>(2.753580020e-6f));
  p = vfma(u2, p, vs<V>(-1.984053088e-4f));
  p = vfma(u2, p, vs<V>(8.333321661e-3f));
  p = vfma(u2, p, vs<V>(-1.666666567e-1f));
  return vfma(u2, p, vs<V>(1.0f));
}
__device__ __forceinline__ float sinc_poly(float u2) { return sinc_poly_v(u2); }

constexpr float kPi2 = 9.86960440108935861883f;   // pi^2

// sin(u)/u for |u| > pi: sin of the turn-reduced argument on the SFU times 1/u
// (relative error ~1e-7).
__device__ __forceinline__ float sinc_large(float u) {
  float s, c;
  sincos_turns(u * kInvTwoPi, &s, &c);
  return s * rcp_approx(u);
}


// Error-free sum a + b = s + e (Knuth TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Compensated accumulator: value = hi + lo.
struct CAcc {
  float hi, lo;
  __device__ __forceinline__ void init() { hi = 0.f; lo = 0.f; }
  __device__ __forceinline__ void add(float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
  }
};

// ---------------------------------------------------------------------------
// Bulk copy (TMA, non-tensor) + mbarrier helpers.  One elected thread issues the
// copy; every consumer waits on the barrier's phase with a bounded poll.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Global -> shared bulk copy completing on `bar`.  dst, src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase completed, false after kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace pft
