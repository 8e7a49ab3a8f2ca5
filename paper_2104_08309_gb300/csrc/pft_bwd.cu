// pft_bwd.cu -- adjoints of the forward transforms (vertex gradients of a loss on F).
//
// For g_Q = dL/dRe F(Q) + i dL/dIm F(Q) the calls return
//   dL/dv = sum_Q Re(conj(g_Q) dF(Q)/dv).
// The segment / face terms are recomputed, not stored by the forward call, and
// differentiated in reverse mode exactly as the forward kernels evaluate them
// (the same branches, phases and polynomials), in FP32 with compensated sums:
//  * k_bq: per Q, the weight gt = g exp(-iQ.c) * scale / |Q|^2 that carries the
//    finalize factors onto each pair (scale 2 in 2D for the half vectors), and
//    the list of Q = 0 / small-|Q| points, which take an FP64 path instead;
//  * k_bwd2d / k_bwd3d: thread <-> segment or face, Q records streamed through
//    shared memory by the same bulk-copy ring as the forward kernels, adjoints
//    of the record fields accumulated per thread, FP64 partials per Q chunk;
//  * FP64 small-|Q| contributions from the boundary-flux (shape derivative)
//    series, then a fixed-order gather to the vertices (3D through a vertex ->
//    face-corner CSR built on the device and sorted, so sums are reproducible).
#include <algorithm>
#include <cstring>

#include "pft_pairs.cuh"

namespace pft {
namespace {

constexpr int kBwdNT = 128;        // threads per block of the pair kernels (one item each)
constexpr int kBbSegs = 2 * kBwdNT;  // segments per pair block of the batched 2D adjoint (two a thread)
constexpr int kQTile = 128;        // Q records per shared-memory tile
constexpr int kAux = 256;          // threads per block of the auxiliary kernels
constexpr double kTwoPiD = 6.283185307179586477;      // 2 pi (FP64)
constexpr double kInvTwoPiD = 0.1591549430918953358;  // 1 / (2 pi) (FP64)

struct __align__(16) QRec {
  float qx, qy, qz, gr, gi, pad0, pad1, pad2;
};
static_assert(sizeof(QRec) == 32, "Q record is two float4");

// ---------------------------------------------------------------------------
// Generic bulk-copy ring over an array of records (same protocol as k_fwd: the
// last warp out of a slot issues the tile kStages further on).
// ---------------------------------------------------------------------------
template <class Item, int TILE, int NT>
struct Ring {
  Item* slots;
  uint64_t* full;
  int* done;
  int* issued;
  const Item* src;
  int64_t n;
  int ntiles;

  __device__ void issue(int t) {
    const int s = t % kStages;
    const int64_t c = min((int64_t)TILE, n - (int64_t)t * TILE);
    const uint32_t bytes = (uint32_t)(c * (int64_t)sizeof(Item));
    mbar_arrive_expect_tx(&full[s], bytes);
    bulk_g2s(slots + s * TILE, src + (int64_t)t * TILE, bytes, &full[s]);
    atomicAdd(issued, 1);
  }
  __device__ void start() {   // every thread; contains a block barrier
    if (threadIdx.x == 0) {
      for (int s = 0; s < kStages; ++s) {
        mbar_init(&full[s], 1);
        done[s] = 0;
      }
      *issued = 0;
      fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int t = 0; t < min(kStages, ntiles); ++t) issue(t);
  }
  // warp-uniform: true when tile t is in its slot
  __device__ bool wait(int t) {
    return __all_sync(0xffffffffu, mbar_wait_bounded(&full[t % kStages], (uint32_t)((t / kStages) & 1)));
  }
  __device__ const Item* tile(int t) const { return slots + (t % kStages) * TILE; }
  __device__ int count(int t) const { return (int)min((int64_t)TILE, n - (int64_t)t * TILE); }
  __device__ void release(int t) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
      __threadfence_block();
      const int s = t % kStages;
      if (atomicAdd(&done[s], 1) == NT / 32 - 1) {
        atomicExch(&done[s], 0);
        if (t + kStages < ntiles) {
          fence_proxy_async_smem();
          issue(t + kStages);
        }
      }
    }
  }
  __device__ void finish() {   // every thread; contains a block barrier
    __syncthreads();
    if (threadIdx.x == 0) {
      const int m = *issued;
      for (int u = max(0, m - kStages); u < m; ++u)
        (void)mbar_wait_bounded(&full[u % kStages], (uint32_t)((u / kStages) & 1));
    }
  }
};

// sinc(u) and its derivative: the Chebyshev polynomial and its derivative on
// |u| <= pi, sin and cos of the turn-reduced argument beyond.  V = float2 takes two
// arguments through the same (paired) instructions.
template <class V>
__device__ __forceinline__ void sinc_d(V u, V& S, V& dS) {
  const V v = vmul(u, u);
  V p = vfma(v, vs<V>(1.361159657e-10f), vs<V>(-2.472836691e-8f));
  p = vfma(v, p, vs<V>(2.753580020e-6f));
  p = vfma(v, p, vs<V>(-1.984053088e-4f));
  p = vfma(v, p, vs<V>(8.333321661e-3f));
  p = vfma(v, p, vs<V>(-1.666666567e-1f));
  S = vfma(v, p, vs<V>(1.0f));
  V d = vfma(v, vs<V>(6.0f * 1.361159657e-10f), vs<V>(5.0f * -2.472836691e-8f));   // p'(v)
  d = vfma(v, d, vs<V>(4.0f * 2.753580020e-6f));
  d = vfma(v, d, vs<V>(3.0f * -1.984053088e-4f));
  d = vfma(v, d, vs<V>(2.0f * 8.333321661e-3f));
  d = vfma(v, d, vs<V>(-1.666666567e-1f));
  dS = vmul(vmul(vs<V>(2.0f), u), d);
  constexpr int kE = sizeof(V) / sizeof(float);
  bool big = false;
#pragma unroll
  for (int e = 0; e < kE; ++e) big = big || (el(&v, e) > kPi2);
  if (__any_sync(__activemask(), big)) {   // warp-uniform: the SFU work only where some lane needs it
#pragma unroll
    for (int e = 0; e < kE; ++e) {
      if (el(&v, e) > kPi2) {
        const float ue = el(&u, e);
        float s, c;
        sincos_turns(ue * kInvTwoPi, &s, &c);
        const float r = rcp_approx(ue);
        const float Se = s * r;
        el(&S, e) = Se;
        el(&dS, e) = (c - Se) * r;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Per-pair adjoints.
// ---------------------------------------------------------------------------

// 2D: term -i w S(u) exp(i ph) of one (Q, segment) pair with weight gt; adds the
// adjoints of the record fields s = (m.x, m.y, h.x, h.y).  V = float2 holds two
// segments (one Q record feeds both).
template <class V>
__device__ __forceinline__ void seg_adj(const QRec& Q, const V (&s)[4], V (&a)[4]) {
  const V qx = vs<V>(Q.qx), qy = vs<V>(Q.qy);
  const V ph = vfma(qx, s[0], vmul(qy, s[1]));
  const V u = vfma(qx, s[2], vmul(qy, s[3]));
  const V w = vfma(qx, s[3], vmul(vneg(qy), s[2]));
  V sn, cs;
  sincos_v(ph, sn, cs);
  V S, dS;
  sinc_d(u, S, dS);
  const V A = vfma(vs<V>(Q.gr), sn, vmul(vs<V>(-Q.gi), cs));   // Re(conj(gt)(sin - i cos))
  const V B = vfma(vs<V>(Q.gr), cs, vmul(vs<V>(Q.gi), sn));    // dA/dph
  const V wb = vmul(S, A), Sb = vmul(w, A), phb = vmul(vmul(w, S), B);
  const V ub = vmul(Sb, dS);
  a[0] = vfma(phb, qx, a[0]);
  a[1] = vfma(phb, qy, a[1]);
  a[2] = vfma(ub, qx, vfma(vneg(wb), qy, a[2]));
  a[3] = vfma(ub, qy, vfma(wb, qx, a[3]));
}

// 3D: face term J = -s exp(i mu) Z (series or edge branch, chosen as in the
// forward kernel, warp-uniform over the lanes) with weight gt, differentiated in
// reverse mode.  The adjoints of the projections mu = Q.g, a0 = Q.q0, a1 = Q.q1,
// s = Q.N (and, in the edge branch, of X = N x Q and b_k = q_k.X) go to `out`,
// which turns them into record adjoints (RecAdj) or Q adjoints (QAdj): the
// projections are bilinear in Q and the record, so the two are mirror images.
template <class Out>
__device__ __forceinline__ void face_adj_t(const QRec& Q, const float4 A, const float4 B, const float4 C, Thr th,
                                           Out& out) {
  const float qx = Q.qx, qy = Q.qy, qz = Q.qz;
  float mu, a0, a1, s, P;
  face_common(qx, qy, qz, A, B, C, mu, a0, a1, s, P);
  // the forward kernel's rule over the warp's faces: short series when all have
  // P < 1/4 (or this one is below p_lo), the k <= 9 form when all are below 1, long
  // series when all are below 9/4 (and p_hi), extra-long series when all are below
  // p_hi, else the edge sum.  All the tests read the
  // warp's largest |P|, taken by every lane before any of them branches.  Here P can
  // be -0 or a tiny negative subnormal (a1 a1 underflows before the fused add when
  // the phases are below ~1e-20, as for a tiny Q beside large ones in k_qgrad), so
  // the sign bit is cleared: the bits of |P| (and of NaN, above +inf) order as
  // unsigned integers, and one reduction serves all three tests.
  const float wmax =
      __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(P) & 0x7fffffffu));
  const bool all_hi = wmax < th.hi;
  const bool all_short = wmax < kPShort;
  const bool all_long = wmax < kPLong;
  const bool shorts = (th.longs ? all_short : all_hi) || (P < th.lo);
  const bool k9s = !shorts && all_hi && wmax < kP9;   // tau > 1 here (else every series lane is short)
  const bool longs = !shorts && !k9s && all_hi && (!th.xlongs || all_long);
  const bool series = shorts || all_hi;
  float sm, cm;
  __sincosf(mu, &sm, &cm);
  float zr, zi;
  // forward Z, then (after the common adjoints below) its reverse pass
  float dGre_dP = 0.f, dGre_dT = 0.f, dGim_dP = 0.f, dGim_dT = 0.f, T = 0.f;
  float Xx = 0.f, Xy = 0.f, Xz = 0.f, x2 = 0.f, inv = 0.f, w[3] = {0.f, 0.f, 0.f}, S[3], dS[3], sp[3], cp[3];
  if (shorts) {               // short series (P < 1/4, k <= 7), as face_series
    T = -(a0 * a1) * (a0 + a1);
    float gre = fmaf(P, -2.48015873e-5f, 1.38888889e-3f);
    gre = fmaf(P, gre, -4.16666667e-2f);
    gre = fmaf(P, gre, 0.5f);
    gre = fmaf(T * T, -2.48015873e-5f, gre);
    const float r = fmaf(P, fmaf(P, -8.26719577e-6f, 3.96825397e-4f), -8.33333333e-3f);
    zr = -T * r;
    zi = gre;
    dGre_dP = fmaf(P, fmaf(P, 3.0f * -2.48015873e-5f, 2.0f * 1.38888889e-3f), -4.16666667e-2f);
    dGre_dT = 2.0f * T * -2.48015873e-5f;
    dGim_dP = T * fmaf(P, 2.0f * -8.26719577e-6f, 3.96825397e-4f);
    dGim_dT = r;
  } else if (k9s) {          // k <= 9 series (P < 1), as face_series_k9
    T = -(a0 * a1) * (a0 + a1);
    const float T2 = T * T;
    float A0 = fmaf(P, 2.755731922e-07f, -2.480158730e-05f);
    A0 = fmaf(P, A0, 1.388888889e-03f);
    A0 = fmaf(P, A0, -4.166666667e-02f);
    A0 = fmaf(P, A0, 0.5f);
    const float A2 = fmaf(P, 8.267195767e-07f, -2.480158730e-05f);
    float D1 = fmaf(P, 1.002084335e-07f, -8.267195767e-06f);
    D1 = fmaf(P, D1, 3.968253968e-04f);
    D1 = fmaf(P, D1, -8.333333333e-03f);
    zr = -T * fmaf(T2, 2.505210839e-08f, D1);
    zi = fmaf(T2, A2, A0);
    // derivatives of A0, A2, D1 in P (coefficients i c_i); the T^3 coefficient is constant
    float dA0 = fmaf(P, 4.0f * 2.755731922e-07f, 3.0f * -2.480158730e-05f);
    dA0 = fmaf(P, dA0, 2.0f * 1.388888889e-03f);
    dA0 = fmaf(P, dA0, -4.166666667e-02f);
    float dD1 = fmaf(P, 3.0f * 1.002084335e-07f, 2.0f * -8.267195767e-06f);
    dD1 = fmaf(P, dD1, 3.968253968e-04f);
    dGre_dP = fmaf(T2, 8.267195767e-07f, dA0);
    dGre_dT = 2.0f * T * A2;
    dGim_dP = T * dD1;
    dGim_dT = fmaf(3.0f * T2, 2.505210839e-08f, D1);
  } else if (longs) {         // long series (P < 9/4, k <= 11), as face_series_long
    T = -(a0 * a1) * (a0 + a1);
    const float T2 = T * T;
    float A = fmaf(P, -2.087675588e-9f, 2.75573192e-7f);
    A = fmaf(P, A, -2.48015873e-5f);
    A = fmaf(P, A, 1.38888889e-3f);
    A = fmaf(P, A, -4.16666667e-2f);
    A = fmaf(P, A, 0.5f);
    float Bp = fmaf(P, -1.252605397e-8f, 8.26719577e-7f);
    Bp = fmaf(P, Bp, -2.48015873e-5f);
    float D = fmaf(P, -8.029522047e-10f, 1.002084318e-7f);
    D = fmaf(P, D, -8.26719577e-6f);
    D = fmaf(P, D, 3.96825397e-4f);
    D = fmaf(P, D, -8.33333333e-3f);
    const float E = fmaf(P, -6.423617749e-10f, 2.505210794e-8f);
    zr = -T * fmaf(T2, E, D);
    zi = fmaf(T2, Bp, A);
    // derivatives of A, B, D, E in P
    float dA = fmaf(P, 5.0f * -2.087675588e-9f, 4.0f * 2.75573192e-7f);
    dA = fmaf(P, dA, 3.0f * -2.48015873e-5f);
    dA = fmaf(P, dA, 2.0f * 1.38888889e-3f);
    dA = fmaf(P, dA, -4.16666667e-2f);
    const float dB = fmaf(P, 2.0f * -1.252605397e-8f, 8.26719577e-7f);
    float dD = fmaf(P, 4.0f * -8.029522047e-10f, 3.0f * 1.002084318e-7f);
    dD = fmaf(P, dD, 2.0f * -8.26719577e-6f);
    dD = fmaf(P, dD, 3.96825397e-4f);
    dGre_dP = fmaf(T2, dB, dA);
    dGre_dT = 2.0f * T * Bp;
    dGim_dP = T * fmaf(T2, -6.423617749e-10f, dD);
    dGim_dT = fmaf(3.0f * T2, E, D);
  } else if (series) {        // extra-long series (P < 9, k <= 17), as face_series_xlong
    T = -(a0 * a1) * (a0 + a1);
    const float T2 = T * T;
    float A0 = fmaf(P, 1.561920697e-16f, -4.779477332e-14f);
    A0 = fmaf(P, A0, 1.147074560e-11f);
    A0 = fmaf(P, A0, -2.087675699e-09f);
    A0 = fmaf(P, A0, 2.755731922e-07f);
    A0 = fmaf(P, A0, -2.480158730e-05f);
    A0 = fmaf(P, A0, 1.388888889e-03f);
    A0 = fmaf(P, A0, -4.166666667e-02f);
    A0 = fmaf(P, A0, 0.5f);
    float A2 = fmaf(P, 3.280033463e-15f, -7.169215999e-13f);
    A2 = fmaf(P, A2, 1.147074560e-10f);
    A2 = fmaf(P, A2, -1.252605419e-08f);
    A2 = fmaf(P, A2, 8.267195767e-07f);
    A2 = fmaf(P, A2, -2.480158730e-05f);
    float A4 = fmaf(P, 2.342881045e-15f, -2.389738666e-13f);
    A4 = fmaf(P, A4, 1.147074560e-11f);
    float D1 = fmaf(P, 6.576508197e-17f, -1.968020078e-14f);
    D1 = fmaf(P, D1, 4.588298239e-12f);
    D1 = fmaf(P, D1, -8.029521918e-10f);
    D1 = fmaf(P, D1, 1.002084335e-07f);
    D1 = fmaf(P, D1, -8.267195767e-06f);
    D1 = fmaf(P, D1, 3.968253968e-04f);
    D1 = fmaf(P, D1, -8.333333333e-03f);
    float D3 = fmaf(P, 2.877222336e-16f, -5.622914509e-14f);
    D3 = fmaf(P, D3, 7.647163732e-12f);
    D3 = fmaf(P, D3, -6.423617535e-10f);
    D3 = fmaf(P, D3, 2.505210839e-08f);
    const float D5 = fmaf(P, 4.932381148e-17f, -2.811457254e-15f);
    const float A24 = fmaf(T2, A4, A2), D35 = fmaf(T2, D5, D3);
    zr = -T * fmaf(T2, D35, D1);
    zi = fmaf(T2, A24, A0);
    // derivatives of A_j, D_j in P (coefficients i c_i)
    float dA0 = fmaf(P, 8.0f * 1.561920697e-16f, 7.0f * -4.779477332e-14f);
    dA0 = fmaf(P, dA0, 6.0f * 1.147074560e-11f);
    dA0 = fmaf(P, dA0, 5.0f * -2.087675699e-09f);
    dA0 = fmaf(P, dA0, 4.0f * 2.755731922e-07f);
    dA0 = fmaf(P, dA0, 3.0f * -2.480158730e-05f);
    dA0 = fmaf(P, dA0, 2.0f * 1.388888889e-03f);
    dA0 = fmaf(P, dA0, -4.166666667e-02f);
    float dA2 = fmaf(P, 5.0f * 3.280033463e-15f, 4.0f * -7.169215999e-13f);
    dA2 = fmaf(P, dA2, 3.0f * 1.147074560e-10f);
    dA2 = fmaf(P, dA2, 2.0f * -1.252605419e-08f);
    dA2 = fmaf(P, dA2, 8.267195767e-07f);
    const float dA4 = fmaf(P, 2.0f * 2.342881045e-15f, -2.389738666e-13f);
    float dD1 = fmaf(P, 7.0f * 6.576508197e-17f, 6.0f * -1.968020078e-14f);
    dD1 = fmaf(P, dD1, 5.0f * 4.588298239e-12f);
    dD1 = fmaf(P, dD1, 4.0f * -8.029521918e-10f);
    dD1 = fmaf(P, dD1, 3.0f * 1.002084335e-07f);
    dD1 = fmaf(P, dD1, 2.0f * -8.267195767e-06f);
    dD1 = fmaf(P, dD1, 3.968253968e-04f);
    float dD3 = fmaf(P, 4.0f * 2.877222336e-16f, 3.0f * -5.622914509e-14f);
    dD3 = fmaf(P, dD3, 2.0f * 7.647163732e-12f);
    dD3 = fmaf(P, dD3, -6.423617535e-10f);
    const float dD5 = 4.932381148e-17f;
    dGre_dP = fmaf(T2, fmaf(T2, dA4, dA2), dA0);
    dGre_dT = 2.0f * T * fmaf(2.0f * T2, A4, A2);                  // d/dT (T^2 A2 + T^4 A4)
    dGim_dP = T * fmaf(T2, fmaf(T2, dD5, dD3), dD1);
    dGim_dT = fmaf(T2, fmaf(5.0f * T2, D5, 3.0f * D3), D1);        // d/dT (T D1 + T^3 D3 + T^5 D5)
  } else {
    const float nx = C.y, ny = C.z, nz = C.w;
    Xx = fmaf(ny, qz, -nz * qy);
    Xy = fmaf(nz, qx, -nx * qz);
    Xz = fmaf(nx, qy, -ny * qx);
    x2 = fmaf(Xx, Xx, fmaf(Xy, Xy, Xz * Xz));
    const float b0 = fmaf(A.w, Xx, fmaf(B.x, Xy, B.y * Xz));
    const float b1 = fmaf(B.z, Xx, fmaf(B.w, Xy, C.x * Xz));
    w[0] = b1 - b0;
    w[1] = fmaf(-2.0f, b1, -b0);
    w[2] = fmaf(2.0f, b0, b1);
    const float h0 = 0.5f * a0, h1 = 0.5f * a1;
    const float u[3] = {h1 - h0, fmaf(-2.0f, h1, -h0), fmaf(2.0f, h0, h1)};
    __sincosf(-h0, &sp[1], &cp[1]);
    __sincosf(-h1, &sp[2], &cp[2]);
    cp[0] = fmaf(cp[1], cp[2], -sp[1] * sp[2]);
    sp[0] = -fmaf(sp[1], cp[2], cp[1] * sp[2]);
    float sr = 0.f, si = 0.f;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      sinc_d(u[l], S[l], dS[l]);
      const float ws = w[l] * S[l];
      sr = fmaf(ws, cp[l], sr);
      si = fmaf(ws, sp[l], si);
    }
    inv = (x2 > 0.f) ? rcp_approx(x2) : 0.f;
    zr = sr * inv;
    zi = si * inv;
  }
  // J = -s W, W = exp(i mu) Z
  const float Wr = fmaf(cm, zr, -sm * zi), Wi = fmaf(cm, zi, sm * zr);
  out.value(-s * Wr, -s * Wi);
  const float sb = -fmaf(Q.gr, Wr, Q.gi * Wi);       // dc/ds
  const float mub = s * fmaf(Q.gr, Wi, -Q.gi * Wr);  // dc/dmu
  const float ghr = -s * fmaf(Q.gr, cm, Q.gi * sm);  // ghat = -s gt exp(-i mu): dc = Re(conj(ghat) dZ)
  const float ghi = -s * fmaf(Q.gi, cm, -Q.gr * sm);
  float a0b, a1b;
  if (series) {
    const float Pb = fmaf(ghi, dGre_dP, -ghr * dGim_dP);
    const float Tb = fmaf(ghi, dGre_dT, -ghr * dGim_dT);
    const float e0 = fmaf(2.0f, a0, a1), e1 = fmaf(2.0f, a1, a0);
    a0b = e0 * fmaf(-Tb, a1, Pb);
    a1b = e1 * fmaf(-Tb, a0, Pb);
  } else {
    const float Sr = ghr * inv, Si = ghi * inv;        // adjoint of the edge sum
    const float x2b = -fmaf(ghr, zr, ghi * zi) * inv;
    float wb[3], psib[3], ub[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const float R = fmaf(Sr, cp[l], Si * sp[l]);
      const float I = fmaf(Sr, sp[l], -Si * cp[l]);
      wb[l] = S[l] * R;
      psib[l] = -w[l] * S[l] * I;
      ub[l] = w[l] * R * dS[l];
    }
    const float h0b = psib[0] - psib[1] - ub[0] - ub[1] + 2.0f * ub[2];
    const float h1b = psib[0] - psib[2] + ub[0] - 2.0f * ub[1] + ub[2];
    a0b = 0.5f * h0b;
    a1b = 0.5f * h1b;
    const float b0b = -wb[0] - wb[1] + 2.0f * wb[2];
    const float b1b = wb[0] - 2.0f * wb[1] + wb[2];
    const float Xbx = fmaf(b0b, A.w, fmaf(b1b, B.z, 2.0f * x2b * Xx));
    const float Xby = fmaf(b0b, B.x, fmaf(b1b, B.w, 2.0f * x2b * Xy));
    const float Xbz = fmaf(b0b, B.y, fmaf(b1b, C.x, 2.0f * x2b * Xz));
    out.edge(b0b, b1b, Xx, Xy, Xz, Xbx, Xby, Xbz);
  }
  out.common(mub, a0b, a1b, sb);
}

// Record adjoints of one (Q, face) pair: g += mub Q, q0 += a0b Q (+ b0b X), q1 += a1b Q (+ b1b X),
// N += sb Q (+ Q x Xbar), in the order of Face32's 12 fields.
struct RecAdj {
  float (&a)[12];
  float qx, qy, qz;
  __device__ __forceinline__ void value(float, float) {}
  __device__ __forceinline__ void edge(float b0b, float b1b, float Xx, float Xy, float Xz, float Xbx, float Xby,
                                       float Xbz) {
    a[3] = fmaf(b0b, Xx, a[3]);
    a[4] = fmaf(b0b, Xy, a[4]);
    a[5] = fmaf(b0b, Xz, a[5]);
    a[6] = fmaf(b1b, Xx, a[6]);
    a[7] = fmaf(b1b, Xy, a[7]);
    a[8] = fmaf(b1b, Xz, a[8]);
    a[9] = fmaf(qy, Xbz, fmaf(-qz, Xby, a[9]));    // N += Q x Xbar
    a[10] = fmaf(qz, Xbx, fmaf(-qx, Xbz, a[10]));
    a[11] = fmaf(qx, Xby, fmaf(-qy, Xbx, a[11]));
  }
  __device__ __forceinline__ void common(float mub, float a0b, float a1b, float sb) {
    a[0] = fmaf(mub, qx, a[0]);
    a[1] = fmaf(mub, qy, a[1]);
    a[2] = fmaf(mub, qz, a[2]);
    a[3] = fmaf(a0b, qx, a[3]);
    a[4] = fmaf(a0b, qy, a[4]);
    a[5] = fmaf(a0b, qz, a[5]);
    a[6] = fmaf(a1b, qx, a[6]);
    a[7] = fmaf(a1b, qy, a[7]);
    a[8] = fmaf(a1b, qz, a[8]);
    a[9] = fmaf(sb, qx, a[9]);
    a[10] = fmaf(sb, qy, a[10]);
    a[11] = fmaf(sb, qz, a[11]);
  }
};

__device__ __forceinline__ void face_adj(const QRec& Q, const float4 A, const float4 B, const float4 C, Thr th,
                                         float (&a)[12]) {
  RecAdj o{a, Q.qx, Q.qy, Q.qz};
  face_adj_t(Q, A, B, C, th, o);
}

// Q adjoint of one (Q, face) pair, and the pair's term J itself (tile sums):
// Qbar += mub g + a0b q0 + a1b q1 + sb N (+ Xbar x N, since X = N x Q).
struct QAdj {
  float jr, ji, bx, by, bz;
  float4 A, B, C;   // the face record: g = A.xyz, q0 = (A.w, B.x, B.y), q1 = (B.z, B.w, C.x), N = C.yzw
  __device__ __forceinline__ void value(float Jr, float Ji) {
    jr += Jr;
    ji += Ji;
  }
  __device__ __forceinline__ void edge(float, float, float, float, float, float Xbx, float Xby, float Xbz) {
    bx = fmaf(Xby, C.w, fmaf(-Xbz, C.z, bx));
    by = fmaf(Xbz, C.y, fmaf(-Xbx, C.w, by));
    bz = fmaf(Xbx, C.z, fmaf(-Xby, C.y, bz));
  }
  __device__ __forceinline__ void common(float mub, float a0b, float a1b, float sb) {
    bx = fmaf(mub, A.x, fmaf(a0b, A.w, fmaf(a1b, B.z, fmaf(sb, C.y, bx))));
    by = fmaf(mub, A.y, fmaf(a0b, B.x, fmaf(a1b, B.w, fmaf(sb, C.z, by))));
    bz = fmaf(mub, A.z, fmaf(a0b, B.y, fmaf(a1b, C.x, fmaf(sb, C.w, bz))));
  }
};

// ---------------------------------------------------------------------------
// Kernels.
// ---------------------------------------------------------------------------

// Q records: Q rounded to FP32 (as the forward uses it) and gt; Q = 0 and small
// |Q| go to the FP64 list with a zero weight here.
template <int D>
__global__ void k_bq(const double* __restrict__ q, const double* __restrict__ g, int64_t n_q, WsHeader* h,
                     double scale, QRec* rec, int32_t* small, const int32_t* __restrict__ perm = nullptr) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // record slot
  if (s >= n_q) return;
  const int64_t i = perm ? (int64_t)perm[s] : s;                      // its Q point (caller's index)
  // the record holds Q rounded to float (the pair kernels' Q); the weight's phase and 1/|Q|^2 take
  // the caller's Q, as the forward's finish does
  float qf[3] = {0.f, 0.f, 0.f};
  double Q[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < D; ++d) {
    Q[d] = q[D * i + d];
    qf[d] = (float)Q[d];
  }
  const double q2 = Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2];
  QRec r{qf[0], qf[1], qf[2], 0.f, 0.f, 0.f, 0.f, 0.f};
  const double rmax = (double)__uint_as_float(h->rmax_bits);
  if (q2 == 0.0 || sqrt(q2) * rmax < kTauSmallQ) {
    small[atomicAdd(&h->small_q_count, 1u)] = (int32_t)i;
  } else {
    double sp, cp;
    sincos(-(Q[0] * h->center[0] + Q[1] * h->center[1] + Q[2] * h->center[2]), &sp, &cp);
    const double gr = g[2 * i], gi = g[2 * i + 1], k = scale / q2;
    r.gr = (float)(k * (gr * cp - gi * sp));
    r.gi = (float)(k * (gr * sp + gi * cp));
  }
  rec[s] = r;
}

// Thread <-> item (segment or face); Q chunk blockIdx.y; FP64 partial per (chunk, item, field).
// ---------------------------------------------------------------------------
// Q-gradient (3D): dL/dQ = Re(conj(g) dF/dQ) per Q.  With F = e^{iQ.c} S / |Q|^2,
// S = sum over faces of J,
//   dF/dQ = F (i c - 2 Q/|Q|^2) + e^{iQ.c}/|Q|^2 dS/dQ,
// and the second part is sum over faces of Re(conj(gt) dJ/dQ) with the same
// weight gt = g e^{-iQ.c}/|Q|^2 as the vertex adjoint (k_bq).  k_qgrad: thread
// <-> Q (one per thread), face records streamed through the bulk-copy ring, the
// reverse pass of each pair into Q (QAdj), S accumulated alongside; FP64
// partials per face chunk (blockIdx.y).
// ---------------------------------------------------------------------------
constexpr int kFTile = 64;          // face records per shared-memory tile of k_qgrad
constexpr int kQG = 5;              // partial fields per (chunk, Q): S.re, S.im, Qbar.xyz

__global__ void __launch_bounds__(kBwdNT) k_qgrad(const Face32* __restrict__ faces, int64_t n_faces,
                                                  int64_t per_split, const QRec* __restrict__ rec, int64_t n_q,
                                                  Thr th, double* __restrict__ partial, uint32_t* status,
                                                  const int32_t* __restrict__ perm) {
  __shared__ __align__(128) Face32 slots[kStages * kFTile];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ int done[kStages];
  __shared__ int issued;
  const int64_t i = blockIdx.x * (int64_t)kBwdNT + threadIdx.x;
  QRec Q{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // lanes past the end: Q = 0, weight 0
  if (i < n_q) Q = rec[i];
  const int64_t f0 = (int64_t)blockIdx.y * per_split;
  const int64_t nf = max((int64_t)0, min(per_split, n_faces - f0));
  Ring<Face32, kFTile, kBwdNT> ring{slots, full, done, &issued, faces + f0, nf, (int)((nf + kFTile - 1) / kFTile)};
  ring.start();
  CAcc acc[kQG];
#pragma unroll
  for (int f = 0; f < kQG; ++f) acc[f].init();
  bool ok = true;
  for (int t = 0; t < ring.ntiles; ++t) {
    if (!ring.wait(t)) { ok = false; break; }
    const Face32* tf = ring.tile(t);
    const int cnt = ring.count(t);
    QAdj o{0.f, 0.f, 0.f, 0.f, 0.f, make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f),
           make_float4(0.f, 0.f, 0.f, 0.f)};
#pragma unroll 1
    for (int j = 0; j < cnt; ++j) {
      const float4* p = reinterpret_cast<const float4*>(tf + j);
      o.A = p[0];
      o.B = p[1];
      o.C = p[2];
      face_adj_t(Q, o.A, o.B, o.C, th, o);
    }
    acc[0].add(o.jr);
    acc[1].add(o.ji);
    acc[2].add(o.bx);
    acc[3].add(o.by);
    acc[4].add(o.bz);
    ring.release(t);
  }
  if (!ok) set_status(status, ST_TIMEOUT);
  ring.finish();
  if (!ok || i >= n_q) return;
  double* dst = partial + ((int64_t)blockIdx.y * n_q + (perm ? (int64_t)perm[i] : i)) * kQG;   // caller's index
#pragma unroll
  for (int f = 0; f < kQG; ++f) dst[f] = (double)acc[f].hi + (double)acc[f].lo;
}

// Per Q (not in the small-|Q| list): fixed-order FP64 sum of the chunk partials, F, and
// dL/dQ = Re(conj(g) F (i c - 2Q/|Q|^2)) + Qbar.
__global__ void k_qfinal(const double* __restrict__ q, const double* __restrict__ g, int64_t n_q,
                         const double* __restrict__ partial, int ks, const WsHeader* h, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_q) return;
  double Q[3];
  for (int d = 0; d < 3; ++d) Q[d] = q[3 * i + d];   // the caller's Q (factors and phase in FP64)
  const double q2 = Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2];
  const double rmax = (double)__uint_as_float(h->rmax_bits);
  if (q2 == 0.0 || sqrt(q2) * rmax < kTauSmallQ) return;   // k_qsmall's (same test as k_bq)
  double v[kQG] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < ks; ++k)
    for (int f = 0; f < kQG; ++f) v[f] += partial[((int64_t)k * n_q + i) * kQG + f];
  const double c[3] = {h->center[0], h->center[1], h->center[2]};
  double sp, cp;
  sincos(Q[0] * c[0] + Q[1] * c[1] + Q[2] * c[2], &sp, &cp);
  const double Fr = (v[0] * cp - v[1] * sp) / q2, Fi = (v[0] * sp + v[1] * cp) / q2;
  const double gr = g[2 * i], gi = g[2 * i + 1];
  // Re(conj(g) F w) for w = i c_d - 2 Q_d/|Q|^2:  Re(conj(g) F) (-2Q_d/q2) - Im(conj(g) F) c_d
  const double re = gr * Fr + gi * Fi, im = gr * Fi - gi * Fr;
  for (int d = 0; d < 3; ++d) out[3 * i + d] = re * (-2.0 * Q[d] / q2) - im * c[d] + v[2 + d];
}

// Sum over a block of kAux threads (fixed order); every thread gets the total.
__device__ __forceinline__ double block_sum_aux(double x, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < kAux / 32; ++w) r += sh[w];
  __syncthreads();
  return r;
}

// Q = 0 and small |Q| in FP64: S0 = sum over the signed tetrahedra (c, p0, p1, p2) of
// det * series3(x), x_k = Q.(p_k - c); dS0/dQ = sum det * sum_k i series4(x, x_k) (p_k - c),
// since d h_n(x)/d x_k = h_{n-1}(x, x_k) for the complete homogeneous polynomials; then
// dF/dQ = e^{iQ.c} (i c S0 + dS0/dQ).  The faces of each listed Q are cut into chunks so that
// all blocks share the work even for a single listed Q (usually Q = 0 alone): k_qsmall_part
// writes one partial per (listed Q, chunk) into at most kQsUnits slots, k_qsmall_fin adds the
// chunks of each listed Q in order.  There are max(kQsUnits, n_q) slots, so every listed Q
// has at least one.
constexpr int kQsUnits = 8192;      // (listed Q, face chunk) partial slots at least
constexpr int kQsF = 8;             // FP64 fields per slot: S0 (re, im), dS0/dQ (re, im) x 3

__device__ __forceinline__ int64_t qsmall_chunks(uint32_t count, int64_t nf, int64_t slots) {
  const int64_t most = max((int64_t)1, (nf + kAux - 1) / kAux);   // at least kAux faces per chunk
  return max((int64_t)1, min(most, slots / max((int64_t)count, (int64_t)1)));
}

__global__ void __launch_bounds__(kAux) k_qsmall_part(const float* __restrict__ v, int64_t nv,
                                                      const int32_t* __restrict__ f, int64_t nf,
                                                      const double* __restrict__ q, const WsHeader* h,
                                                      const int32_t* list, int64_t slots,
                                                      double* __restrict__ part) {
  __shared__ double sh[kAux / 32];
  const uint32_t count = h->small_q_count;   // <= n_q <= slots
  const int64_t nch = qsmall_chunks(count, nf, slots);
  const int64_t per = (nf + nch - 1) / nch;
  const double c[3] = {h->center[0], h->center[1], h->center[2]};
  for (int64_t u = blockIdx.x; u < (int64_t)count * nch; u += gridDim.x) {
    const int64_t e = u / nch, ch = u % nch;
    const int64_t i = list[e];
    double Q[3];
    for (int d = 0; d < 3; ++d) Q[d] = q[3 * i + d];
    double acc[kQsF] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t m1 = min(nf, (ch + 1) * per);
    for (int64_t m = ch * per + threadIdx.x; m < m1; m += kAux) {
      const int32_t id[3] = {f[3 * m], f[3 * m + 1], f[3 * m + 2]};
      if (id[0] < 0 || id[1] < 0 || id[2] < 0 || id[0] >= nv || id[1] >= nv || id[2] >= nv) continue;
      double P[3][3], x[4];
      for (int k = 0; k < 3; ++k) {
        for (int d = 0; d < 3; ++d) P[k][d] = (double)v[3 * (int64_t)id[k] + d] - c[d];
        x[k] = Q[0] * P[k][0] + Q[1] * P[k][1] + Q[2] * P[k][2];
      }
      const double det = P[0][0] * (P[1][1] * P[2][2] - P[1][2] * P[2][1]) +
                         P[0][1] * (P[1][2] * P[2][0] - P[1][0] * P[2][2]) +
                         P[0][2] * (P[1][0] * P[2][1] - P[1][1] * P[2][0]);
      double sr, si;
      simplex_series<3, 3, 16>(x, sr, si);
      acc[0] += det * sr;
      acc[1] += det * si;
      for (int k = 0; k < 3; ++k) {
        x[3] = x[k];
        double tr, ti;
        simplex_series<4, 4, 16>(x, tr, ti);
        for (int d = 0; d < 3; ++d) {   // i (tr + i ti) P_kd = (-ti + i tr) P_kd
          acc[2 + 2 * d] += -det * ti * P[k][d];
          acc[3 + 2 * d] += det * tr * P[k][d];
        }
      }
    }
    for (int k = 0; k < kQsF; ++k) {
      const double t = block_sum_aux(acc[k], sh);
      if (threadIdx.x == 0) part[u * kQsF + k] = t;
    }
  }
}

__global__ void k_qsmall_fin(int64_t nf, const double* __restrict__ q, const double* __restrict__ g,
                             const WsHeader* h, const int32_t* list, int64_t slots, const double* __restrict__ part,
                             double* __restrict__ out) {
  const uint32_t count = h->small_q_count;
  const int64_t nch = qsmall_chunks(count, nf, slots);
  const double c[3] = {h->center[0], h->center[1], h->center[2]};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = list[e];
    double acc[kQsF] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t ch = 0; ch < nch; ++ch)
      for (int k = 0; k < kQsF; ++k) acc[k] += part[(e * nch + ch) * kQsF + k];
    double Q[3];
    for (int d = 0; d < 3; ++d) Q[d] = q[3 * i + d];
    double sp, cp;
    sincos(Q[0] * c[0] + Q[1] * c[1] + Q[2] * c[2], &sp, &cp);
    const double gr = g[2 * i], gi = g[2 * i + 1];
    for (int d = 0; d < 3; ++d) {
      // D = i c_d S0 + dS0_d, dF = e^{iQ.c} D, out = Re(conj(g) dF)
      const double Dr = -c[d] * acc[1] + acc[2 + 2 * d], Di = c[d] * acc[0] + acc[3 + 2 * d];
      const double dr = Dr * cp - Di * sp, di = Dr * sp + Di * cp;
      out[3 * i + d] = gr * dr + gi * di;
    }
  }
}

// ---------------------------------------------------------------------------
// Q-gradient (2D): the same structure in the plane.  F = e^{iQ.c} (2/|Q|^2) S with
// S = sum over segments of T = -i w sinc(u) e^{i phi}, phi = Q.m, u = Q.h,
// w = Qx hy - Qy hx (m the midpoint, h half the edge vector; Sec. 2, Eq. 6), so
//   dF/dQ = F (i c - 2 Q/|Q|^2) + e^{iQ.c} (2/|Q|^2) dS/dQ,
// the second part being sum over segments of Re(conj(gt) dT/dQ) with gt from k_bq<2>
// (scale 2).  phi, u and w are bilinear in Q and the record, so the reverse pass of
// a pair gives Qbar = phib m + ub h + wb (hy, -hx).  k_qgrad2d: thread <-> Q, segment
// records streamed through the bulk-copy ring, FP64 partials per segment chunk.
// ---------------------------------------------------------------------------
constexpr int kSTile = 128;         // segment records per shared-memory tile of k_qgrad2d
constexpr int kQG2 = 4;             // partial fields per (chunk, Q): S.re, S.im, Qbar.xy

__device__ __forceinline__ void seg_qadj(const QRec& Q, const float4 s, float& jr, float& ji, float& bx, float& by) {
  const float ph = fmaf(Q.qx, s.x, Q.qy * s.y);
  const float u = fmaf(Q.qx, s.z, Q.qy * s.w);
  const float w = fmaf(Q.qx, s.w, -Q.qy * s.z);
  float sn, cs;
  __sincosf(ph, &sn, &cs);
  float S, dS;
  sinc_d(u, S, dS);
  const float ws = w * S;
  jr = fmaf(ws, sn, jr);                        // T = w S (sin - i cos), as the forward's segment term
  ji = fmaf(-ws, cs, ji);
  const float A = fmaf(Q.gr, sn, -Q.gi * cs);   // Re(conj(gt)(sin - i cos))
  const float B = fmaf(Q.gr, cs, Q.gi * sn);    // dA/dph
  const float wb = S * A, ub = w * A * dS, phb = ws * B;
  bx = fmaf(phb, s.x, fmaf(ub, s.z, fmaf(wb, s.w, bx)));
  by = fmaf(phb, s.y, fmaf(ub, s.w, fmaf(-wb, s.z, by)));
}

__global__ void __launch_bounds__(kBwdNT) k_qgrad2d(const Seg32* __restrict__ segs, int64_t n_segs,
                                                    int64_t per_split, const QRec* __restrict__ rec, int64_t n_q,
                                                    double* __restrict__ partial, uint32_t* status,
                                                    const int32_t* __restrict__ perm) {
  __shared__ __align__(128) Seg32 slots[kStages * kSTile];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ int done[kStages];
  __shared__ int issued;
  const int64_t i = blockIdx.x * (int64_t)kBwdNT + threadIdx.x;
  QRec Q{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // lanes past the end: Q = 0, weight 0
  if (i < n_q) Q = rec[i];
  const int64_t s0 = (int64_t)blockIdx.y * per_split;
  const int64_t ns = max((int64_t)0, min(per_split, n_segs - s0));
  Ring<Seg32, kSTile, kBwdNT> ring{slots, full, done, &issued, segs + s0, ns, (int)((ns + kSTile - 1) / kSTile)};
  ring.start();
  CAcc acc[kQG2];
#pragma unroll
  for (int f = 0; f < kQG2; ++f) acc[f].init();
  bool ok = true;
  for (int t = 0; t < ring.ntiles; ++t) {
    if (!ring.wait(t)) { ok = false; break; }
    const float4* ts = reinterpret_cast<const float4*>(ring.tile(t));
    const int cnt = ring.count(t);
    float jr = 0.f, ji = 0.f, bx = 0.f, by = 0.f;
#pragma unroll 2
    for (int j = 0; j < cnt; ++j) seg_qadj(Q, ts[j], jr, ji, bx, by);
    acc[0].add(jr);
    acc[1].add(ji);
    acc[2].add(bx);
    acc[3].add(by);
    ring.release(t);
  }
  if (!ok) set_status(status, ST_TIMEOUT);
  ring.finish();
  if (!ok || i >= n_q) return;
  double* dst = partial + ((int64_t)blockIdx.y * n_q + (perm ? (int64_t)perm[i] : i)) * kQG2;   // caller's index
#pragma unroll
  for (int f = 0; f < kQG2; ++f) dst[f] = (double)acc[f].hi + (double)acc[f].lo;
}

// Per Q (not in the small-|Q| list): fixed-order FP64 sum of the chunk partials,
// F = e^{iQ.c} 2 S/|Q|^2 and dL/dQ = Re(conj(g) F (i c - 2Q/|Q|^2)) + Qbar.
__global__ void k_qfinal2d(const double* __restrict__ q, const double* __restrict__ g, int64_t n_q,
                           const double* __restrict__ partial, int ks, const WsHeader* h, double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_q) return;
  const double Q[2] = {q[2 * i], q[2 * i + 1]};   // the caller's Q (factors and phase in FP64)
  const double q2 = Q[0] * Q[0] + Q[1] * Q[1];
  const double rmax = (double)__uint_as_float(h->rmax_bits);
  if (q2 == 0.0 || sqrt(q2) * rmax < kTauSmallQ) return;   // k_qsmall2d's (same test as k_bq)
  double v[kQG2] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < ks; ++k)
    for (int f = 0; f < kQG2; ++f) v[f] += partial[((int64_t)k * n_q + i) * kQG2 + f];
  const double c[2] = {h->center[0], h->center[1]};
  double sp, cp;
  sincos(Q[0] * c[0] + Q[1] * c[1], &sp, &cp);
  const double Fr = 2.0 * (v[0] * cp - v[1] * sp) / q2, Fi = 2.0 * (v[0] * sp + v[1] * cp) / q2;
  const double gr = g[2 * i], gi = g[2 * i + 1];
  const double re = gr * Fr + gi * Fi, im = gr * Fi - gi * Fr;   // Re and Im of conj(g) F
  for (int d = 0; d < 2; ++d) out[2 * i + d] = re * (-2.0 * Q[d] / q2) - im * c[d] + v[2 + d];
}

// Q = 0 and small |Q| in 2D, FP64: the fan of signed triangles (c, p_j, p_{j+1}) of every
// loop, S0 = sum det * series2(x) with x_k = Q.(p_k - c) (the apex node is 0), and
// dS0/dQ = sum det * sum_k i series3(x, x_k) (p_k - c) (a node repeated: the derivative of
// the complete homogeneous polynomials); dF/dQ = e^{iQ.c} (i c S0 + dS0/dQ).  Chunked over
// the segments and spread over all blocks as k_qsmall_part.
constexpr int kQsF2 = 6;            // FP64 fields per slot: S0 (re, im), dS0/dQ (re, im) x 2

__global__ void __launch_bounds__(kAux) k_qsmall2d_part(const float* __restrict__ v, int64_t nv,
                                                        const int64_t* __restrict__ off, int64_t nl,
                                                        const double* __restrict__ q, const WsHeader* h,
                                                        const int32_t* list, int64_t slots,
                                                        double* __restrict__ part) {
  __shared__ double sh[kAux / 32];
  const uint32_t count = h->small_q_count;   // <= n_q <= slots
  const int64_t nch = qsmall_chunks(count, nv, slots);
  const int64_t per = (nv + nch - 1) / nch;
  const double c[2] = {h->center[0], h->center[1]};
  for (int64_t u = blockIdx.x; u < (int64_t)count * nch; u += gridDim.x) {
    const int64_t e = u / nch, ch = u % nch;
    const int64_t i = list[e];
    const double Q[2] = {q[2 * i], q[2 * i + 1]};
    double acc[kQsF2] = {0, 0, 0, 0, 0, 0};
    const int64_t j1 = min(nv, (ch + 1) * per);
    for (int64_t j = ch * per + threadIdx.x; j < j1; j += kAux) {
      int64_t lo = 0, hi = nl;   // loop of vertex j
      while (lo + 1 < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= j) lo = mid; else hi = mid;
      }
      const int64_t k = (j + 1 < off[lo + 1]) ? j + 1 : off[lo];
      if (k < 0 || k >= nv) continue;
      const double P[2][2] = {{(double)v[2 * j] - c[0], (double)v[2 * j + 1] - c[1]},
                              {(double)v[2 * k] - c[0], (double)v[2 * k + 1] - c[1]}};
      double x[3] = {Q[0] * P[0][0] + Q[1] * P[0][1], Q[0] * P[1][0] + Q[1] * P[1][1], 0.0};
      const double det = P[0][0] * P[1][1] - P[1][0] * P[0][1];
      double sr, si;
      simplex_series<2, 2, 16>(x, sr, si);
      acc[0] += det * sr;
      acc[1] += det * si;
      for (int n = 0; n < 2; ++n) {
        x[2] = x[n];
        double tr, ti;
        simplex_series<3, 3, 16>(x, tr, ti);
        for (int d = 0; d < 2; ++d) {   // i (tr + i ti) P_nd = (-ti + i tr) P_nd
          acc[2 + 2 * d] += -det * ti * P[n][d];
          acc[3 + 2 * d] += det * tr * P[n][d];
        }
      }
    }
    for (int k = 0; k < kQsF2; ++k) {
      const double t = block_sum_aux(acc[k], sh);
      if (threadIdx.x == 0) part[u * kQsF2 + k] = t;
    }
  }
}

__global__ void k_qsmall2d_fin(int64_t nv, const double* __restrict__ q, const double* __restrict__ g,
                               const WsHeader* h, const int32_t* list, int64_t slots,
                               const double* __restrict__ part, double* __restrict__ out) {
  const uint32_t count = h->small_q_count;
  const int64_t nch = qsmall_chunks(count, nv, slots);
  const double c[2] = {h->center[0], h->center[1]};
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = list[e];
    double acc[kQsF2] = {0, 0, 0, 0, 0, 0};
    for (int64_t ch = 0; ch < nch; ++ch)
      for (int k = 0; k < kQsF2; ++k) acc[k] += part[(e * nch + ch) * kQsF2 + k];
    const double Q[2] = {q[2 * i], q[2 * i + 1]};
    double sp, cp;
    sincos(Q[0] * c[0] + Q[1] * c[1], &sp, &cp);
    const double gr = g[2 * i], gi = g[2 * i + 1];
    for (int d = 0; d < 2; ++d) {
      const double Dr = -c[d] * acc[1] + acc[2 + 2 * d], Di = c[d] * acc[0] + acc[3 + 2 * d];
      const double dr = Dr * cp - Di * sp, di = Dr * sp + Di * cp;
      out[2 * i + d] = gr * dr + gi * di;
    }
  }
}

template <int D, int NF>
__global__ void __launch_bounds__(kBwdNT) k_bwd(const void* __restrict__ items, int64_t n_items,
                                                const QRec* __restrict__ rec, int64_t n_q, int64_t per_split,
                                                Thr th, double* __restrict__ partial, uint32_t* status) {
  __shared__ __align__(128) QRec slots[kStages * kQTile];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ int done[kStages];
  __shared__ int issued;
  const int64_t m = blockIdx.x * (int64_t)kBwdNT + threadIdx.x;
  float4 F[3] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
  if (m < n_items) {
    if constexpr (D == 2) F[0] = reinterpret_cast<const float4*>(items)[m];
    else for (int k = 0; k < 3; ++k) F[k] = reinterpret_cast<const float4*>(items)[3 * m + k];
  }
  const int64_t q0 = (int64_t)blockIdx.y * per_split;
  const int64_t nq = max((int64_t)0, min(per_split, n_q - q0));
  Ring<QRec, kQTile, kBwdNT> ring{slots, full, done, &issued, rec + q0, nq, (int)((nq + kQTile - 1) / kQTile)};
  ring.start();
  CAcc acc[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) acc[f].init();
  bool ok = true;
  for (int t = 0; t < ring.ntiles; ++t) {
    if (!ring.wait(t)) { ok = false; break; }
    const QRec* tq = ring.tile(t);
    const int cnt = ring.count(t);
    float a[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) a[f] = 0.f;
#pragma unroll 1
    for (int j = 0; j < cnt; ++j) {
      const QRec Q = tq[j];
      if constexpr (D == 2) seg_adj(Q, *reinterpret_cast<const float(*)[4]>(&F[0]), *reinterpret_cast<float(*)[4]>(a));
      else face_adj(Q, F[0], F[1], F[2], th, *reinterpret_cast<float(*)[12]>(a));
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) acc[f].add(a[f]);
    ring.release(t);
  }
  if (!ok) set_status(status, ST_TIMEOUT);
  ring.finish();
  if (!ok || m >= n_items) return;
  double* dst = partial + ((int64_t)blockIdx.y * n_items + m) * NF;
#pragma unroll
  for (int f = 0; f < NF; ++f) dst[f] = (double)acc[f].hi + (double)acc[f].lo;
}

// 2D vertex gradients: record adjoints of segment j (start) and of the segment
// ending at j, summed over Q chunks in order, plus FP64 small-|Q| terms.
// Small |Q|: dF/dp0 = nu e^{i a0} (J0 - J1), dF/dp1 = nu e^{i a0} J1 with
// nu = (dy, -dx), J0 = int_0^1 e^{itd}, J1 = int_0^1 t e^{itd} (series, |d| small).
// Both ends lie within r_max of the centre and |Q| r_max < 1/4, so |d| < 1/2: the terms
// fall faster than 2^-n/n!, the series stops once one is below 1e-18 (J0 is near 1), and
// 20 terms bound it (remainder below 0.5^20/20! ~ 4e-25).  Q = 0 takes one term.
__constant__ double kInvN[22] = {1.0,        1.0 / 1,  1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,
                                 1.0 / 6,    1.0 / 7,  1.0 / 8,  1.0 / 9,  1.0 / 10, 1.0 / 11,
                                 1.0 / 12,   1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17,
                                 1.0 / 18,   1.0 / 19, 1.0 / 20, 1.0 / 21};   // kInvN[k] = 1/k
__device__ __forceinline__ void seg_small(const double* p0, const double* p1, double qx, double qy, double gr,
                                          double gi, double ph_c, double* g0, double* g1) {
  const double a0 = qx * p0[0] + qy * p0[1], d = qx * (p1[0] - p0[0]) + qy * (p1[1] - p0[1]);
  double j0r = 0, j0i = 0, j1r = 0, j1i = 0, tr = 1, ti = 0;   // term (i d)^n / n!
  for (int n = 0; n < 20; ++n) {
    const double r1 = kInvN[n + 1], r2 = kInvN[n + 2];
    j0r = fma(tr, r1, j0r); j0i = fma(ti, r1, j0i);
    j1r = fma(tr, r2, j1r); j1i = fma(ti, r2, j1i);
    const double dn = d * r1;
    const double nr = -ti * dn, ni = tr * dn;
    tr = nr; ti = ni;
    if (fabs(tr) + fabs(ti) < 1e-18) break;
  }
  double se, ce;
  sincos(a0 + ph_c, &se, &ce);   // exp(i(Q.c + Q.(p0 - c)))
  // conj(g) * e * J  -> real part
  const double er0 = ce * (j0r - j1r) - se * (j0i - j1i), ei0 = ce * (j0i - j1i) + se * (j0r - j1r);
  const double er1 = ce * j1r - se * j1i, ei1 = ce * j1i + se * j1r;
  const double c0 = gr * er0 + gi * ei0, c1 = gr * er1 + gi * ei1;
  const double nu[2] = {p1[1] - p0[1], -(p1[0] - p0[0])};
  g0[0] += c0 * nu[0]; g0[1] += c0 * nu[1];
  g1[0] += c1 * nu[0]; g1[1] += c1 * nu[1];
}

__global__ void k_bvert2d(const float* __restrict__ v, int64_t nv, const int64_t* __restrict__ off, int64_t nl,
                          const double* __restrict__ partial, int ks, const WsHeader* h,
                          const int32_t* __restrict__ small, const double* __restrict__ q,
                          const double* __restrict__ g, float* __restrict__ grad) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nv) return;
  int64_t lo = 0, hi = nl;
  while (lo + 1 < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (off[mid] <= j) lo = mid; else hi = mid;
  }
  const int64_t s0 = off[lo], s1 = off[lo + 1];
  int64_t jp = (j > s0) ? j - 1 : s1 - 1;   // segment ending at j
  int64_t jn = (j + 1 < s1) ? j + 1 : s0;    // end of segment j
  if (jp < 0 || jp >= nv) jp = j;
  if (jn < 0 || jn >= nv) jn = j;
  double mS[2] = {0, 0}, hS[2] = {0, 0}, mP[2] = {0, 0}, hP[2] = {0, 0};
  for (int s = 0; s < ks; ++s) {
    const double* a = partial + ((int64_t)s * nv + j) * 4;
    const double* b = partial + ((int64_t)s * nv + jp) * 4;
    mS[0] += a[0]; mS[1] += a[1]; hS[0] += a[2]; hS[1] += a[3];
    mP[0] += b[0]; mP[1] += b[1]; hP[0] += b[2]; hP[1] += b[3];
  }
  // m = (p0+p1)/2, h = (p1-p0)/2: start of segment j gets mbar/2 - hbar/2, end of segment jp gets mbar/2 + hbar/2
  double gx = 0.5 * (mS[0] - hS[0]) + 0.5 * (mP[0] + hP[0]);
  double gy = 0.5 * (mS[1] - hS[1]) + 0.5 * (mP[1] + hP[1]);
  const uint32_t ns = h->small_q_count;
  if (ns) {
    const double c[2] = {h->center[0], h->center[1]};
    const double pj[2] = {(double)v[2 * j] - c[0], (double)v[2 * j + 1] - c[1]};
    const double pn[2] = {(double)v[2 * jn] - c[0], (double)v[2 * jn + 1] - c[1]};
    const double pp[2] = {(double)v[2 * jp] - c[0], (double)v[2 * jp + 1] - c[1]};
    for (uint32_t e = 0; e < ns; ++e) {   // fixed order is not needed for a plain sum of a few terms, but kept
      const int64_t iq = small[e];
      const double qx = q[2 * iq], qy = q[2 * iq + 1];
      const double phc = qx * c[0] + qy * c[1];
      double d0[2] = {0, 0}, d1[2] = {0, 0}, e0[2] = {0, 0}, e1[2] = {0, 0};
      seg_small(pj, pn, qx, qy, g[2 * iq], g[2 * iq + 1], phc, d0, d1);   // j is the start
      seg_small(pp, pj, qx, qy, g[2 * iq], g[2 * iq + 1], phc, e0, e1);   // j is the end
      gx += d0[0] + e1[0];
      gy += d0[1] + e1[1];
    }
  }
  grad[2 * j] = (float)gx;
  grad[2 * j + 1] = (float)gy;
}

// ---------------------------------------------------------------------------
// Batched 2D adjoint: many polygons, each with its own weights g_i(Q) on a shared Q set.
// Each polygon is centred on its own bounding box (as the batched forward does); Q records
// carry gt_i(Q) = 2 g_i(Q) e^{-iQ.c_i}/|Q|^2 per (polygon, Q) row; pair blocks never straddle
// polygons; the vertex gather adds each polygon's own small-|Q| rows in FP64.
// ---------------------------------------------------------------------------
// Per shape of a batch (polygon or mesh): bounding-box centre (cz = 0 in 2D) and max radius.
struct PolyC {
  double cx, cy, cz;
  float rmax;
  int32_t pad;
};

__device__ __forceinline__ float block_minmax_f(float x, bool is_max, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float y = __shfl_xor_sync(0xffffffffu, x, o);
    x = is_max ? fmaxf(x, y) : fminf(x, y);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  float r = sh[0];
  for (int w = 1; w < kAux / 32; ++w) r = is_max ? fmaxf(r, sh[w]) : fminf(r, sh[w]);
  __syncthreads();
  return r;
}

// One block per polygon: offset checks, bounding-box centre, segment records relative to it,
// max radius, and the number of pair blocks (kBbSegs segments each) the polygon needs.
__global__ void __launch_bounds__(kAux) k_bbprep(const float* __restrict__ v, int64_t nv,
                                                 const int64_t* __restrict__ off, int64_t np, Seg32* segs,
                                                 PolyC* pc, int32_t* nblk, WsHeader* h) {
  __shared__ float sh[kAux / 32];
  const int64_t i = blockIdx.x;
  const int64_t s0 = off[i], s1 = off[i + 1];
  if (threadIdx.x == 0 && (s1 < s0 || s0 < 0 || s1 > nv || (i == 0 && s0 != 0) || (i == np - 1 && s1 != nv)))
    set_status(&h->status, ST_OFFSETS);
  const int64_t b0 = max((int64_t)0, min(s0, nv)), n = max((int64_t)0, min(s1, nv) - b0);
  float mn[2] = {3.4e38f, 3.4e38f}, mx[2] = {-3.4e38f, -3.4e38f};
  bool bad = false;
  for (int64_t j = threadIdx.x; j < n; j += kAux)
    for (int d = 0; d < 2; ++d) {
      const float x = v[2 * (b0 + j) + d];
      if (!isfinite(x)) { bad = true; continue; }
      mn[d] = fminf(mn[d], x);
      mx[d] = fmaxf(mx[d], x);
    }
  if (bad) set_status(&h->status, ST_NONFINITE);
  double c[2];
  for (int d = 0; d < 2; ++d) {
    const float lo = block_minmax_f(mn[d], false, sh), hi = block_minmax_f(mx[d], true, sh);
    c[d] = (n > 0 && lo <= hi) ? 0.5 * ((double)lo + (double)hi) : 0.0;
  }
  float rm = 0.f;
  for (int64_t j = threadIdx.x; j < n; j += kAux) {
    const int64_t a = b0 + j, b = b0 + (j + 1 < n ? j + 1 : 0);
    const double x0 = (double)v[2 * a] - c[0], y0 = (double)v[2 * a + 1] - c[1];
    const double x1 = (double)v[2 * b] - c[0], y1 = (double)v[2 * b + 1] - c[1];
    segs[a] = Seg32{(float)(0.5 * (x0 + x1)), (float)(0.5 * (y0 + y1)), (float)(0.5 * (x1 - x0)),
                    (float)(0.5 * (y1 - y0))};
    rm = fmaxf(rm, __double2float_ru(sqrt(x0 * x0 + y0 * y0)));
  }
  rm = block_minmax_f(rm, true, sh);
  if (threadIdx.x == 0) {
    pc[i] = PolyC{c[0], c[1], 0.0, rm, 0};
    nblk[i] = (int32_t)((n + kBbSegs - 1) / kBbSegs);
  }
}

// One block per polygon: its Q records (weight 0 on small rows) and its small rows, listed in
// Q order (a block-wide ordered compaction, so the gather below is deterministic).
// Rows of polygon i: with q_off (per-polygon Q lists) rows q_off[i] .. q_off[i+1]-1 of q and g;
// without, all n_q points of the shared q and rows i n_q .. (i+1) n_q - 1 of g.  Malformed
// offsets set ST_OFFSETS and are clamped to [0, n_q].
__device__ __forceinline__ void bb_rows(const int64_t* q_off, int64_t i, int64_t n_q, int64_t& qb, int64_t& gb,
                                        int64_t& nqi) {
  if (q_off == nullptr) {
    qb = 0;
    gb = i * n_q;
    nqi = n_q;
  } else {
    const int64_t a = max((int64_t)0, min(q_off[i], n_q)), b = max(a, min(q_off[i + 1], n_q));
    qb = gb = a;
    nqi = b - a;
  }
}

// D = 2: weight 2 g e^{-iQ.c}/|Q|^2 (records hold half segment vectors); D = 3: g e^{-iQ.c}/|Q|^2.
template <int D>
__global__ void __launch_bounds__(kAux) k_bbq(const double* __restrict__ q, const int64_t* __restrict__ q_off,
                                              const double* __restrict__ g, int64_t n_q, int64_t np,
                                              const PolyC* __restrict__ pc, QRec* rec, int32_t* small,
                                              int32_t* small_cnt, WsHeader* h) {
  __shared__ int wcount[kAux / 32];
  __shared__ int base;
  const int64_t i = blockIdx.x;
  const PolyC P = pc[i];
  if (q_off != nullptr && threadIdx.x == 0 &&
      (q_off[i + 1] < q_off[i] || q_off[i] < 0 || q_off[i + 1] > n_q || (i == 0 && q_off[0] != 0) ||
       (i == np - 1 && q_off[np] != n_q)))
    set_status(&h->status, ST_OFFSETS);
  int64_t qb, gb, nqi;
  bb_rows(q_off, i, n_q, qb, gb, nqi);
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int64_t l0 = 0; l0 < nqi; l0 += kAux) {
    const int64_t l = l0 + threadIdx.x;
    bool is_small = false;
    if (l < nqi) {
      // the record holds Q rounded to float; the weight's phase and factor take the caller's Q
      const double Qx = q[D * (qb + l)], Qy = q[D * (qb + l) + 1], Qz = D == 3 ? q[D * (qb + l) + D - 1] : 0.0;
      const float qx = (float)Qx, qy = (float)Qy, qz = (float)Qz;
      const double q2 = Qx * Qx + Qy * Qy + Qz * Qz;
      QRec r{qx, qy, qz, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (q2 == 0.0 || q2 * ((double)P.rmax * (double)P.rmax) < kTauSmallQ * kTauSmallQ) {
        is_small = true;
      } else {
        // e^{-iQ.c}: the phase in FP64, less its nearest multiple of 2 pi (FP64), then an FP32
        // sincos on [-pi, pi]; the record holds FP32 weights, so this loses nothing further
        const double ph = -(Qx * P.cx + Qy * P.cy + Qz * P.cz);
        const float pr = (float)fma(-rint(ph * kInvTwoPiD), kTwoPiD, ph);
        float sp, cp;
        sincosf(pr, &sp, &cp);
        const float gr = (float)g[2 * (gb + l)], gi = (float)g[2 * (gb + l) + 1];
        const float k = (D == 2 ? 2.0f : 1.0f) / (float)q2;
        r.gr = k * fmaf(gr, cp, -gi * sp);
        r.gi = k * fmaf(gr, sp, gi * cp);
      }
      rec[gb + l] = r;
    }
    const unsigned m = __ballot_sync(0xffffffffu, is_small);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wcount[wid] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < kAux / 32; ++w) {
      if (w < wid) before += wcount[w];
      total += wcount[w];
    }
    if (is_small) small[gb + base + before + __popc(m & ((1u << lane) - 1u))] = (int32_t)l;
    __syncthreads();
    if (threadIdx.x == 0) base += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) small_cnt[i] = base;
}

// Pair blocks: block b is pair block b - bstart[i] of polygon i (bisection over the exclusive
// scan bstart of the blocks per polygon); thread t <-> its segments t and t + kBwdNT (one Q record
// load feeds two pairs); the polygon's Q records stream through the ring (Q chunk blockIdx.y).
// Warps with no segment only wait for and release the tiles (polygons end mid-block: the sizes
// vary).  Blocks past the last polygon leave at once.
__global__ void __launch_bounds__(kBwdNT) k_bbwd(const Seg32* __restrict__ segs, int64_t nv,
                                                 const int64_t* __restrict__ off, int64_t np,
                                                 const int64_t* __restrict__ bstart, const int32_t* __restrict__ nblk,
                                                 const QRec* __restrict__ rec, const int64_t* __restrict__ q_off,
                                                 int64_t n_q, int64_t per_split, Thr th,
                                                 double* __restrict__ partial, uint32_t* status) {
  __shared__ __align__(128) QRec slots[kStages * kQTile];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ int done[kStages];
  __shared__ int issued;
  const int64_t b = blockIdx.x;
  if (b >= bstart[np - 1] + nblk[np - 1]) return;   // uniform over the block
  int64_t lo = 0, hi = np - 1;                      // the last polygon whose blocks start at or before b
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (bstart[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const int64_t s0 = max((int64_t)0, min(off[lo], nv)), s1 = max(s0, min(off[lo + 1], nv));
  const int64_t m = s0 + (b - bstart[lo]) * kBbSegs + threadIdx.x, m2 = m + kBwdNT;
  const bool mine = m < s1, mine2 = m2 < s1;
  float4 F = make_float4(0.f, 0.f, 0.f, 0.f), F2 = F;
  if (mine) F = reinterpret_cast<const float4*>(segs)[m];
  if (mine2) F2 = reinterpret_cast<const float4*>(segs)[m2];
  const bool live = __any_sync(0xffffffffu, mine), live2 = __any_sync(0xffffffffu, mine2);
  int64_t qb, gb, nqi;
  bb_rows(q_off, lo, n_q, qb, gb, nqi);
  const int64_t q0 = (int64_t)blockIdx.y * per_split;
  const int64_t nq = max((int64_t)0, min(per_split, nqi - q0));
  Ring<QRec, kQTile, kBwdNT> ring{slots, full, done, &issued, rec + gb + q0, nq,
                                  (int)((nq + kQTile - 1) / kQTile)};
  ring.start();
  CAcc acc[4], acc2[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) { acc[f].init(); acc2[f].init(); }
  bool ok = true;
  for (int t = 0; t < ring.ntiles; ++t) {
    if (!ring.wait(t)) { ok = false; break; }
    const QRec* tq = ring.tile(t);
    const int cnt = ring.count(t);
    float a[4] = {0.f, 0.f, 0.f, 0.f}, a2[4] = {0.f, 0.f, 0.f, 0.f};
    if (live2) {   // both segments in paired registers: .x the first, .y the second
      const float2 sv[4] = {make_float2(F.x, F2.x), make_float2(F.y, F2.y), make_float2(F.z, F2.z),
                            make_float2(F.w, F2.w)};
      float2 ap[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll 1
      for (int j = 0; j < cnt; ++j) seg_adj(tq[j], sv, ap);
#pragma unroll
      for (int f = 0; f < 4; ++f) { a[f] = ap[f].x; a2[f] = ap[f].y; }
    } else if (live) {
      const float sv[4] = {F.x, F.y, F.z, F.w};
#pragma unroll 1
      for (int j = 0; j < cnt; ++j) seg_adj(tq[j], sv, a);
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) { acc[f].add(a[f]); acc2[f].add(a2[f]); }
    ring.release(t);
  }
  if (!ok) set_status(status, ST_TIMEOUT);
  ring.finish();
  if (!ok) return;
  if (mine) {
    double* dst = partial + ((int64_t)blockIdx.y * nv + m) * 4;
#pragma unroll
    for (int f = 0; f < 4; ++f) dst[f] = (double)acc[f].hi + (double)acc[f].lo;
  }
  if (mine2) {
    double* dst = partial + ((int64_t)blockIdx.y * nv + m2) * 4;
#pragma unroll
    for (int f = 0; f < 4; ++f) dst[f] = (double)acc2[f].hi + (double)acc2[f].lo;
  }
}

// Per vertex: record adjoints of the segment it starts and of the one it ends (Q chunks in
// order), and the FP64 small-|Q| boundary-flux terms of its polygon's small rows.
__global__ void k_bbvert(const float* __restrict__ v, int64_t nv, const int64_t* __restrict__ off, int64_t np,
                         const double* __restrict__ partial, int ks, const PolyC* __restrict__ pc,
                         const int32_t* __restrict__ small, const int32_t* __restrict__ small_cnt,
                         const double* __restrict__ q, const int64_t* __restrict__ q_off, int64_t n_q,
                         const double* __restrict__ g, float* __restrict__ grad) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nv) return;
  int64_t lo = 0, hi = np;
  while (lo + 1 < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (off[mid] <= j) lo = mid; else hi = mid;
  }
  const int64_t s0 = off[lo], s1 = off[lo + 1];
  int64_t jp = (j > s0) ? j - 1 : s1 - 1;   // segment ending at j
  int64_t jn = (j + 1 < s1) ? j + 1 : s0;    // end of segment j
  if (jp < 0 || jp >= nv) jp = j;
  if (jn < 0 || jn >= nv) jn = j;
  double mS[2] = {0, 0}, hS[2] = {0, 0}, mP[2] = {0, 0}, hP[2] = {0, 0};
  for (int s = 0; s < ks; ++s) {
    const double* a = partial + ((int64_t)s * nv + j) * 4;
    const double* b = partial + ((int64_t)s * nv + jp) * 4;
    mS[0] += a[0]; mS[1] += a[1]; hS[0] += a[2]; hS[1] += a[3];
    mP[0] += b[0]; mP[1] += b[1]; hP[0] += b[2]; hP[1] += b[3];
  }
  double gx = 0.5 * (mS[0] - hS[0]) + 0.5 * (mP[0] + hP[0]);
  double gy = 0.5 * (mS[1] - hS[1]) + 0.5 * (mP[1] + hP[1]);
  const PolyC P = pc[lo];
  const int32_t ns = small_cnt[lo];
  if (ns > 0) {
    int64_t qb, gb, nqi;
    bb_rows(q_off, lo, n_q, qb, gb, nqi);
    const double c[2] = {P.cx, P.cy};
    const double pj[2] = {(double)v[2 * j] - c[0], (double)v[2 * j + 1] - c[1]};
    const double pn[2] = {(double)v[2 * jn] - c[0], (double)v[2 * jn + 1] - c[1]};
    const double pp[2] = {(double)v[2 * jp] - c[0], (double)v[2 * jp + 1] - c[1]};
    for (int32_t e = 0; e < ns; ++e) {
      const int64_t l = small[gb + e];
      const double qx = q[2 * (qb + l)], qy = q[2 * (qb + l) + 1];
      const double phc = qx * c[0] + qy * c[1];
      const double gr = g[2 * (gb + l)], gi = g[2 * (gb + l) + 1];
      double d0[2] = {0, 0}, d1[2] = {0, 0}, e0[2] = {0, 0}, e1[2] = {0, 0};
      seg_small(pj, pn, qx, qy, gr, gi, phc, d0, d1);   // j is the start
      seg_small(pp, pj, qx, qy, gr, gi, phc, e0, e1);   // j is the end
      gx += d0[0] + e1[0];
      gy += d0[1] + e1[1];
    }
  }
  grad[2 * j] = (float)gx;
  grad[2 * j + 1] = (float)gy;
}

// ---------------------------------------------------------------------------
// Batched 3D adjoint: many closed meshes (CSR mesh_off over the faces, one shared vertex
// array), each centred on the bounding box of its own faces' corners, on a shared Q list or
// per-mesh Q lists.  The structure of the batched 2D adjoint with the 3D pair adjoint:
// k_bbprep3 (one block per mesh: checks, centre, face records, max radius, pair blocks needed),
// the block scan, k_bbq<3> (per (mesh, Q row) records and small-|Q| lists), k_bbwd3 (blocks
// that never straddle meshes, thread <-> face, the mesh's Q records through the bulk-copy ring),
// k_bbcorner3 (corner adjoints with the mesh's small-|Q| rows), and the vertex gather of the
// single-mesh adjoint over all faces.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAux) k_bbprep3(const float* __restrict__ v, int64_t nv,
                                                  const int32_t* __restrict__ f, int64_t nf,
                                                  const int64_t* __restrict__ off, int64_t nm, Face32* recs,
                                                  PolyC* mc, int32_t* nblk, WsHeader* h) {
  __shared__ float sh[kAux / 32];
  const int64_t i = blockIdx.x;
  const int64_t s0 = off[i], s1 = off[i + 1];
  if (threadIdx.x == 0 && (s1 < s0 || s0 < 0 || s1 > nf || (i == 0 && s0 != 0) || (i == nm - 1 && s1 != nf)))
    set_status(&h->status, ST_OFFSETS);
  const int64_t b0 = max((int64_t)0, min(s0, nf)), n = max((int64_t)0, min(s1, nf) - b0);
  auto valid = [&](int64_t m) {
    const int32_t a = f[3 * m], b = f[3 * m + 1], c = f[3 * m + 2];
    return a >= 0 && b >= 0 && c >= 0 && a < nv && b < nv && c < nv;
  };
  float mn[3] = {3.4e38f, 3.4e38f, 3.4e38f}, mx[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
  bool bad_index = false, bad_value = false;
  for (int64_t j = threadIdx.x; j < n; j += kAux) {
    const int64_t m = b0 + j;
    if (!valid(m)) { bad_index = true; continue; }
    for (int k = 0; k < 3; ++k)
      for (int d = 0; d < 3; ++d) {
        const float x = v[3 * (int64_t)f[3 * m + k] + d];
        if (!isfinite(x)) { bad_value = true; continue; }
        mn[d] = fminf(mn[d], x);
        mx[d] = fmaxf(mx[d], x);
      }
  }
  if (bad_index) set_status(&h->status, ST_INDEX);
  if (bad_value) set_status(&h->status, ST_NONFINITE);
  double c[3];
  for (int d = 0; d < 3; ++d) {
    const float lo = block_minmax_f(mn[d], false, sh), hi = block_minmax_f(mx[d], true, sh);
    c[d] = (n > 0 && lo <= hi) ? 0.5 * ((double)lo + (double)hi) : 0.0;
  }
  float rm = 0.f;
  for (int64_t j = threadIdx.x; j < n; j += kAux) {
    const int64_t m = b0 + j;
    Face32 r{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // skipped faces contribute 0
    if (valid(m)) {
      double P[3][3], g[3], q0[3], q1[3];
      for (int k = 0; k < 3; ++k)
        for (int d = 0; d < 3; ++d) P[k][d] = (double)v[3 * (int64_t)f[3 * m + k] + d] - c[d];
      for (int d = 0; d < 3; ++d) {
        g[d] = (P[0][d] + P[1][d] + P[2][d]) / 3.0;
        q0[d] = P[0][d] - g[d];
        q1[d] = P[1][d] - g[d];
      }
      const double e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
      const double e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
      const double N[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                           e1[0] * e2[1] - e1[1] * e2[0]};
      r = Face32{(float)g[0], (float)g[1], (float)g[2], (float)q0[0], (float)q0[1], (float)q0[2],
                 (float)q1[0], (float)q1[1], (float)q1[2], (float)N[0], (float)N[1], (float)N[2]};
      for (int k = 0; k < 3; ++k)
        rm = fmaxf(rm, __double2float_ru(sqrt(P[k][0] * P[k][0] + P[k][1] * P[k][1] + P[k][2] * P[k][2])));
    }
    recs[m] = r;
  }
  rm = block_minmax_f(rm, true, sh);
  if (threadIdx.x == 0) {
    mc[i] = PolyC{c[0], c[1], c[2], rm, 0};
    nblk[i] = (int32_t)((n + kBwdNT - 1) / kBwdNT);
  }
}

// Pair blocks: block b is pair block b - bstart[i] of mesh i; thread t <-> face t of that block;
// the mesh's Q records stream through the ring (Q chunk blockIdx.y).  Warps with no face only wait
// for and release the tiles.  Blocks past the last mesh leave at once.
__global__ void __launch_bounds__(kBwdNT) k_bbwd3(const Face32* __restrict__ recs, int64_t nf,
                                                  const int64_t* __restrict__ off, int64_t nm,
                                                  const int64_t* __restrict__ bstart, const int32_t* __restrict__ nblk,
                                                  const QRec* __restrict__ rec, const int64_t* __restrict__ q_off,
                                                  int64_t n_q, int64_t per_split, Thr th,
                                                  double* __restrict__ partial, uint32_t* status) {
  __shared__ __align__(128) QRec slots[kStages * kQTile];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ int done[kStages];
  __shared__ int issued;
  const int64_t b = blockIdx.x;
  if (b >= bstart[nm - 1] + nblk[nm - 1]) return;   // uniform over the block
  int64_t lo = 0, hi = nm - 1;                      // the last mesh whose blocks start at or before b
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (bstart[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const int64_t s0 = max((int64_t)0, min(off[lo], nf)), s1 = max(s0, min(off[lo + 1], nf));
  const int64_t m = s0 + (b - bstart[lo]) * kBwdNT + threadIdx.x;
  const bool mine = m < s1;
  float4 F[3] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
  if (mine)
    for (int k = 0; k < 3; ++k) F[k] = reinterpret_cast<const float4*>(recs)[3 * m + k];
  const bool live = __any_sync(0xffffffffu, mine);
  int64_t qb, gb, nqi;
  bb_rows(q_off, lo, n_q, qb, gb, nqi);
  const int64_t q0 = (int64_t)blockIdx.y * per_split;
  const int64_t nq = max((int64_t)0, min(per_split, nqi - q0));
  Ring<QRec, kQTile, kBwdNT> ring{slots, full, done, &issued, rec + gb + q0, nq, (int)((nq + kQTile - 1) / kQTile)};
  ring.start();
  CAcc acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k].init();
  bool ok = true;
  for (int t = 0; t < ring.ntiles; ++t) {
    if (!ring.wait(t)) { ok = false; break; }
    const QRec* tq = ring.tile(t);
    const int cnt = ring.count(t);
    float a[12] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (live) {
#pragma unroll 1
      for (int j = 0; j < cnt; ++j) face_adj(tq[j], F[0], F[1], F[2], th, a);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k].add(a[k]);
    ring.release(t);
  }
  if (!ok) set_status(status, ST_TIMEOUT);
  ring.finish();
  if (!ok || !mine) return;
  double* dst = partial + ((int64_t)blockIdx.y * nf + m) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) dst[k] = (double)acc[k].hi + (double)acc[k].lo;
}

__device__ void corner_adj(int64_t m, const float* __restrict__ v, int64_t nv, const int32_t* __restrict__ f,
                           int64_t nf, const double* __restrict__ partial, int ks, const double* c,
                           const int32_t* __restrict__ small, uint32_t ns, int64_t q_base, int64_t g_base,
                           const double* __restrict__ q, const double* __restrict__ g, double* __restrict__ out);

// Per face: its mesh (bisection over the offsets), then the corner adjoints with that mesh's
// centre and small-|Q| rows.
__global__ void k_bbcorner3(const float* __restrict__ v, int64_t nv, const int32_t* __restrict__ f, int64_t nf,
                            const int64_t* __restrict__ off, int64_t nm, const double* __restrict__ partial, int ks,
                            const PolyC* __restrict__ mc, const int32_t* __restrict__ small,
                            const int32_t* __restrict__ small_cnt, const double* __restrict__ q,
                            const int64_t* __restrict__ q_off, int64_t n_q, const double* __restrict__ g,
                            double* __restrict__ corner) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= nf) return;
  int64_t lo = 0, hi = nm;   // the last mesh whose faces start at or before m
  while (lo + 1 < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (off[mid] <= m) lo = mid; else hi = mid;
  }
  int64_t qb, gb, nqi;
  bb_rows(q_off, lo, n_q, qb, gb, nqi);
  const PolyC C = mc[lo];
  const double c[3] = {C.cx, C.cy, C.cz};
  const uint32_t ns = (uint32_t)max(0, min(small_cnt[lo], (int32_t)nqi));
  corner_adj(m, v, nv, f, nf, partial, ks, c, small + gb, ns, qb, gb, q, g, corner + 9 * m);
}

// 3D: per face, chunk sums of the record adjoints -> corner adjoints (FP64), plus
// small-|Q| corner terms dF/dp_k = exp(iQ.c) N sum_j i^j h_j(a, a_k)/(j+3)!.
// Corner adjoints of face m (FP64): the record adjoints summed over the Q chunks, mapped to the
// three corners, plus the small-|Q| terms of the ns listed Q rows small[0 .. ns-1] (rows of q from
// q_base, of g from g_base) about the centre c.
__device__ void corner_adj(int64_t m, const float* __restrict__ v, int64_t nv, const int32_t* __restrict__ f,
                           int64_t nf, const double* __restrict__ partial, int ks, const double* c,
                           const int32_t* __restrict__ small, uint32_t ns, int64_t q_base, int64_t g_base,
                           const double* __restrict__ q, const double* __restrict__ g, double* __restrict__ out) {
  const int32_t id[3] = {f[3 * m], f[3 * m + 1], f[3 * m + 2]};
  if (id[0] < 0 || id[1] < 0 || id[2] < 0 || id[0] >= nv || id[1] >= nv || id[2] >= nv) {
    for (int k = 0; k < 9; ++k) out[k] = 0.0;
    return;
  }
  double ab[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int s = 0; s < ks; ++s) {
    const double* a = partial + ((int64_t)s * nf + m) * 12;
    for (int k = 0; k < 12; ++k) ab[k] += a[k];
  }
  double P[3][3];
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) P[k][d] = (double)v[3 * (int64_t)id[k] + d] - c[d];
  // records: g = (P0+P1+P2)/3, q0 = P0 - g, q1 = P1 - g, N = (P1-P0) x (P2-P0)
  double pb[3][3];
  for (int d = 0; d < 3; ++d) {
    const double gt = ab[d] - ab[3 + d] - ab[6 + d];
    pb[0][d] = ab[3 + d] + gt / 3.0;
    pb[1][d] = ab[6 + d] + gt / 3.0;
    pb[2][d] = gt / 3.0;
  }
  const double e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
  const double e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
  const double* Nb = ab + 9;
  const double e1b[3] = {e2[1] * Nb[2] - e2[2] * Nb[1], e2[2] * Nb[0] - e2[0] * Nb[2], e2[0] * Nb[1] - e2[1] * Nb[0]};
  const double e2b[3] = {Nb[1] * e1[2] - Nb[2] * e1[1], Nb[2] * e1[0] - Nb[0] * e1[2], Nb[0] * e1[1] - Nb[1] * e1[0]};
  for (int d = 0; d < 3; ++d) {
    pb[1][d] += e1b[d];
    pb[2][d] += e2b[d];
    pb[0][d] -= e1b[d] + e2b[d];
  }
  if (ns) {
    const double N[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    for (uint32_t e = 0; e < ns; ++e) {
      const int64_t iq = q_base + small[e], ig = g_base + small[e];
      const double Q[3] = {q[3 * iq], q[3 * iq + 1], q[3 * iq + 2]};
      const double al[3] = {Q[0] * P[0][0] + Q[1] * P[0][1] + Q[2] * P[0][2],
                            Q[0] * P[1][0] + Q[1] * P[1][1] + Q[2] * P[1][2],
                            Q[0] * P[2][0] + Q[1] * P[2][1] + Q[2] * P[2][2]};
      const double mu = (al[0] + al[1] + al[2]) / 3.0;
      double se, ce;
      sincos(mu + Q[0] * c[0] + Q[1] * c[1] + Q[2] * c[2], &se, &ce);
      for (int k = 0; k < 3; ++k) {
        // sum_j i^j h_j(x) / (j+3)!, x = (a0, a1, a2, a_k) centred at mu, 18 terms
        const double x[4] = {al[0] - mu, al[1] - mu, al[2] - mu, al[k] - mu};
        double hh[19];
        hh[0] = 1.0;
        for (int j = 1; j <= 18; ++j) hh[j] = 0.0;
        for (int t = 0; t < 4; ++t)
          for (int j = 1; j <= 18; ++j) hh[j] = fma(x[t], hh[j - 1], hh[j]);
        double sr = 0.0, si = 0.0, inv = 1.0 / 6.0;
        for (int j = 0; j <= 18; ++j) {
          const double t = hh[j] * inv;
          switch (j & 3) { case 0: sr += t; break; case 1: si += t; break; case 2: sr -= t; break; default: si -= t; }
          inv /= (double)(j + 4);
        }
        const double hr = ce * sr - se * si, hi = ce * si + se * sr;
        const double cf = g[2 * ig] * hr + g[2 * ig + 1] * hi;   // Re(conj(g) * H)
        for (int d = 0; d < 3; ++d) pb[k][d] += cf * N[d];
      }
    }
  }
  for (int k = 0; k < 3; ++k)
    for (int d = 0; d < 3; ++d) out[3 * k + d] = pb[k][d];
}

__global__ void k_bcorner3d(const float* __restrict__ v, int64_t nv, const int32_t* __restrict__ f, int64_t nf,
                            const double* __restrict__ partial, int ks, const WsHeader* h,
                            const int32_t* __restrict__ small, const double* __restrict__ q,
                            const double* __restrict__ g, double* __restrict__ corner) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= nf) return;
  const double c[3] = {h->center[0], h->center[1], h->center[2]};
  corner_adj(m, v, nv, f, nf, partial, ks, c, small, h->small_q_count, 0, 0, q, g, corner + 9 * m);
}

// Vertex -> face-corner CSR: degrees, exclusive scan, fill, per-vertex sort.
__global__ void k_deg(const int32_t* __restrict__ f, int64_t nf, int64_t nv, int32_t* deg) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 3 * nf) return;
  const int32_t vtx = f[i];
  if (vtx >= 0 && vtx < nv) atomicAdd(&deg[vtx], 1);
}

// Exclusive scan in three steps: per-block scan with block totals, scan of the
// totals (one block, sequential over chunks), add back.
__global__ void k_scan_block(const int32_t* __restrict__ in, int64_t n, int64_t* out, int64_t* block_tot) {
  __shared__ int64_t sh[kAux];
  const int64_t i = blockIdx.x * (int64_t)kAux + threadIdx.x;
  int64_t x = (i < n) ? in[i] : 0;
  sh[threadIdx.x] = x;
  __syncthreads();
  for (int o = 1; o < kAux; o <<= 1) {
    const int64_t y = (threadIdx.x >= (unsigned)o) ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += y;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - x;
  if (threadIdx.x == kAux - 1) block_tot[blockIdx.x] = sh[kAux - 1];
}

__global__ void k_scan_totals(int64_t* block_tot, int64_t nb) {
  if (threadIdx.x != 0) return;
  int64_t run = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t t = block_tot[b];
    block_tot[b] = run;
    run += t;
  }
}

__global__ void k_scan_add(int64_t* out, int64_t n, const int64_t* block_tot) {
  const int64_t i = blockIdx.x * (int64_t)kAux + threadIdx.x;
  if (i < n) out[i] += block_tot[blockIdx.x];
}

__global__ void k_fill(const int32_t* __restrict__ f, int64_t nf, int64_t nv, const int64_t* __restrict__ start,
                       int32_t* cursor, int32_t* list) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 3 * nf) return;
  const int32_t vtx = f[i];
  if (vtx < 0 || vtx >= nv) return;
  list[start[vtx] + atomicAdd(&cursor[vtx], 1)] = (int32_t)i;   // corner id 3m + k
}

__global__ void k_gather3d(int64_t nv, const int64_t* __restrict__ start, const int32_t* __restrict__ deg,
                           int32_t* list, const double* __restrict__ corner, float* __restrict__ grad) {
  const int64_t vtx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (vtx >= nv) return;
  int32_t* L = list + start[vtx];
  const int n = deg[vtx];
  for (int a = 1; a < n; ++a) {   // insertion sort: corner ids in increasing order
    const int32_t key = L[a];
    int b = a - 1;
    while (b >= 0 && L[b] > key) { L[b + 1] = L[b]; --b; }
    L[b + 1] = key;
  }
  double s[3] = {0, 0, 0};
  for (int a = 0; a < n; ++a) {
    const int64_t cid = L[a];
    const int64_t mm = cid / 3, k = cid % 3;
    for (int d = 0; d < 3; ++d) s[d] += corner[9 * mm + 3 * k + d];
  }
  for (int d = 0; d < 3; ++d) grad[3 * vtx + d] = (float)s[d];
}

__global__ void k_zero_i32(int32_t* p, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0;
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
thread_local int g_bwd_launches = 0;
inline size_t al(size_t x) { return (x + 255) / 256 * 256; }
template <typename T>
T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }
inline unsigned blocks(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

int sm_count() {
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, sms);
}

// Q chunks so that the grid (item blocks x chunks) is 16 waves of 8 blocks per SM (about 25 waves at
// the pair kernels' 5 resident blocks): blocks do not finish in waves (the resident blocks of an SM
// share it unevenly), and the last ones to start leave SMs partly idle for about a third of a
// block's run.  The 3D adjoint on 81,920 faces x 32,768 Q: 9.29 ms at 4 waves of 8, 9.07 ms at 16.
int q_splits(int64_t n_items, int64_t n_q) {
  const int64_t item_blocks = std::max<int64_t>(1, (n_items + kBwdNT - 1) / kBwdNT);
  const int64_t slots = (int64_t)sm_count() * 8;
  const int64_t q_tiles = std::max<int64_t>(1, (n_q + kQTile - 1) / kQTile);
  int64_t k = std::max<int64_t>(1, (16 * slots + item_blocks - 1) / item_blocks);
  return (int)std::min<int64_t>({k, q_tiles, 256});
}

// Chunks of a Q-gradient launch: k (the fewest that fill whole waves, the last >= 97 % full) raised,
// for a launch of fewer than 40 waves, as far as chunks of at least 16 tiles and 64 chunks allow,
// the last wave still >= 97 % full (the tail of the last blocks, as above).  The 3D Q-gradient on
// 81,920 faces x 32,768 Q: 7 chunks (2 waves) 9.91 ms, 64 chunks 9.22 ms.
int more_chunks(int k, int64_t q_blocks, int64_t slots, int64_t tiles) {
  const int kw_max = (int)std::min<int64_t>(64, tiles / 16);
  if ((double)(q_blocks * k) / (double)slots >= 40.0) return k;
  for (int c = k + 1; c <= kw_max; ++c) {
    const double waves = (double)(q_blocks * c) / (double)slots;
    if (waves / std::ceil(waves) < 0.97) continue;
    k = c;
    if (waves >= 40.0) break;
  }
  return k;
}

struct BwdLayout {
  size_t mparts, items, qrec, small, partial, corner, deg, cursor, start, btot, list, total;
  int nblk, ks;
  int64_t per_split;
};

BwdLayout bwd_layout(int dim, int64_t n_verts, int64_t n_items, int64_t n_prep, int64_t n_q) {
  BwdLayout y{};
  y.ks = q_splits(n_items, n_q);
  const int64_t q_tiles = std::max<int64_t>(1, (n_q + kQTile - 1) / kQTile);
  y.per_split = ((q_tiles + y.ks - 1) / y.ks) * kQTile;
  y.ks = (int)std::max<int64_t>(1, (n_q + y.per_split - 1) / y.per_split);
  y.nblk = std::max(1, prep_blocks(n_prep));
  const int nf = dim == 2 ? 4 : 12;
  size_t o = al(sizeof(WsHeader));
  y.mparts = o;  o = al(o + sizeof(double) * (size_t)y.nblk);
  y.items = o;   o = al(o + (dim == 2 ? sizeof(Seg32) : sizeof(Face32)) * (size_t)std::max<int64_t>(n_items, 1));
  y.qrec = o;    o = al(o + sizeof(QRec) * (size_t)std::max<int64_t>(n_q, 1));
  y.small = o;   o = al(o + sizeof(int32_t) * (size_t)std::max<int64_t>(n_q, 1));
  y.partial = o; o = al(o + sizeof(double) * nf * (size_t)y.ks * (size_t)std::max<int64_t>(n_items, 1));
  if (dim == 3) {
    y.corner = o; o = al(o + sizeof(double) * 9 * (size_t)std::max<int64_t>(n_items, 1));
    y.deg = o;    o = al(o + sizeof(int32_t) * (size_t)std::max<int64_t>(n_verts, 1));
    y.cursor = o; o = al(o + sizeof(int32_t) * (size_t)std::max<int64_t>(n_verts, 1));
    y.start = o;  o = al(o + sizeof(int64_t) * (size_t)std::max<int64_t>(n_verts, 1));
    y.btot = o;   o = al(o + sizeof(int64_t) * (size_t)blocks(n_verts, kAux));
    y.list = o;   o = al(o + sizeof(int32_t) * 3 * (size_t)std::max<int64_t>(n_items, 1));
  }
  y.total = o;
  return y;
}

// Q-gradient workspace: header, volume partials (written by the prep kernel), face
// records, Q records, small-|Q| list, kQG FP64 partials per (face chunk, Q).
struct QgLayout {
  size_t mparts, items, qrec, small, partial, spart, qperm, qscratch, total;
  bool tiled;   // the pair kernel visits the Q points in the library's order (q_order option)
  int nblk, ks;
  int64_t per_split, slots;
};

// The Q-gradient kernels hold one Q point per thread, so a group of 32 threads is 32 consecutive
// slots: with the library's order (q_order option) those are 32 consecutive points of the Z-order.
void qg_order_regions(QgLayout& y, size_t& o, int64_t n_q, int64_t n_items, bool tiled) {
  y.tiled = tiled && qorder_wanted(n_q, n_items, 1, kBwdNT);
  if (!y.tiled) return;
  y.qperm = o;    o = al(o + sizeof(int32_t) * (size_t)n_q);
  y.qscratch = o; o = al(o + qorder_layout(n_q).total);
}

QgLayout qg_layout(int64_t n_faces, int64_t n_q, bool tiled) {
  QgLayout y{};
  const int64_t face_tiles = std::max<int64_t>(1, (n_faces + kFTile - 1) / kFTile);
  const int64_t q_blocks = std::max<int64_t>(1, (n_q + kBwdNT - 1) / kBwdNT);
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_qgrad, kBwdNT, 0) != cudaSuccess || occ < 1) occ = 1;
  const int64_t slots = (int64_t)sm_count() * occ;
  const int kmax = (int)std::max<int64_t>(1, std::min<int64_t>(64, face_tiles / 2));
  int k = 0, best_k = 1;
  double best_eff = -1.0;
  for (int c = 1; c <= kmax; ++c) {   // smallest split that fills whole waves (last one >= 97 %)
    const double waves = (double)(q_blocks * c) / (double)slots;
    const double eff = waves / std::ceil(waves);
    if (q_blocks * c >= slots && eff >= 0.97) { k = c; break; }
    if (eff > best_eff + 1e-9) { best_eff = eff; best_k = c; }
  }
  if (k == 0) k = best_k;
  k = more_chunks(k, q_blocks, slots, face_tiles);
  const int64_t tiles_per = (face_tiles + k - 1) / k;
  y.per_split = tiles_per * kFTile;
  y.ks = (int)((face_tiles + tiles_per - 1) / tiles_per);
  y.nblk = std::max(1, prep_blocks(n_faces));
  size_t o = al(sizeof(WsHeader));
  y.mparts = o;  o = al(o + sizeof(double) * (size_t)y.nblk);
  y.items = o;   o = al(o + sizeof(Face32) * (size_t)std::max<int64_t>(n_faces, 1));
  y.qrec = o;    o = al(o + sizeof(QRec) * (size_t)std::max<int64_t>(n_q, 1));
  y.small = o;   o = al(o + sizeof(int32_t) * (size_t)std::max<int64_t>(n_q, 1));
  y.partial = o; o = al(o + sizeof(double) * kQG * (size_t)y.ks * (size_t)std::max<int64_t>(n_q, 1));
  y.slots = std::max<int64_t>(kQsUnits, n_q);
  y.spart = o;   o = al(o + sizeof(double) * kQsF * (size_t)y.slots);
  qg_order_regions(y, o, n_q, n_faces, tiled);
  y.total = o;
  return y;
}

// 2D Q-gradient workspace: header, area partials, segment records, Q records, small-|Q|
// list, kQG2 FP64 partials per (segment chunk, Q), small-|Q| slots.
QgLayout qg2_layout(int64_t n_segs, int64_t n_prep, int64_t n_q, bool tiled) {
  QgLayout y{};
  const int64_t seg_tiles = std::max<int64_t>(1, (n_segs + kSTile - 1) / kSTile);
  const int64_t q_blocks = std::max<int64_t>(1, (n_q + kBwdNT - 1) / kBwdNT);
  int occ = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_qgrad2d, kBwdNT, 0) != cudaSuccess || occ < 1) occ = 1;
  const int64_t slots = (int64_t)sm_count() * occ;
  const int kmax = (int)std::max<int64_t>(1, std::min<int64_t>(64, seg_tiles / 2));
  int k = 0, best_k = 1;
  double best_eff = -1.0;
  for (int c = 1; c <= kmax; ++c) {   // smallest split that fills whole waves (last one >= 97 %)
    const double waves = (double)(q_blocks * c) / (double)slots;
    const double eff = waves / std::ceil(waves);
    if (q_blocks * c >= slots && eff >= 0.97) { k = c; break; }
    if (eff > best_eff + 1e-9) { best_eff = eff; best_k = c; }
  }
  if (k == 0) k = best_k;
  k = more_chunks(k, q_blocks, slots, seg_tiles);
  const int64_t tiles_per = (seg_tiles + k - 1) / k;
  y.per_split = tiles_per * kSTile;
  y.ks = (int)((seg_tiles + tiles_per - 1) / tiles_per);
  y.nblk = std::max(1, prep_blocks(n_prep));
  size_t o = al(sizeof(WsHeader));
  y.mparts = o;  o = al(o + sizeof(double) * (size_t)y.nblk);
  y.items = o;   o = al(o + sizeof(Seg32) * (size_t)std::max<int64_t>(n_segs, 1));
  y.qrec = o;    o = al(o + sizeof(QRec) * (size_t)std::max<int64_t>(n_q, 1));
  y.small = o;   o = al(o + sizeof(int32_t) * (size_t)std::max<int64_t>(n_q, 1));
  y.partial = o; o = al(o + sizeof(double) * kQG2 * (size_t)y.ks * (size_t)std::max<int64_t>(n_q, 1));
  y.slots = std::max<int64_t>(kQsUnits, n_q);
  y.spart = o;   o = al(o + sizeof(double) * kQsF2 * (size_t)y.slots);
  qg_order_regions(y, o, n_q, n_segs, tiled);
  y.total = o;
  return y;
}

// Batched 2D adjoint workspace.
struct BbLayout {
  size_t segs, pc, nblk, bstart, btot, rec, small, scnt, partial, total;
  int ks;
  int64_t per_split, grid;
};

// per_poly_q: Q lists per polygon (q_off), n_q rows in all; else a shared list, n_polys x n_q
// rows.  Either way every polygon has at most n_q rows, which the Q chunking covers.
BbLayout bb_layout(int64_t nv, int64_t np, int64_t n_q, bool per_poly_q) {
  BbLayout y{};
  y.grid = std::max<int64_t>(1, np + (nv + kBbSegs - 1) / kBbSegs);   // at least the pair blocks needed
  const int64_t slots = (int64_t)sm_count() * 8;
  const int64_t q_tiles = std::max<int64_t>(1, (n_q + kQTile - 1) / kQTile);
  // Q chunks for 16 waves of 8 blocks per SM, as q_splits (the tail of the last blocks to start):
  // 4,096 polygons x 64^2 Q 17.32 -> 17.04 ms, 1,024 meshes x 32^3 Q 218.5 -> 212.6 ms against 4 waves
  const int64_t k = std::min<int64_t>({std::max<int64_t>(1, (16 * slots + y.grid - 1) / y.grid), q_tiles, 256});
  y.per_split = ((q_tiles + k - 1) / k) * kQTile;
  y.ks = (int)std::max<int64_t>(1, (n_q + y.per_split - 1) / y.per_split);
  const int64_t rows = std::max<int64_t>(per_poly_q ? n_q : np * n_q, 1);
  size_t o = al(sizeof(WsHeader));
  y.segs = o;    o = al(o + sizeof(Seg32) * (size_t)std::max<int64_t>(nv, 1));
  y.pc = o;      o = al(o + sizeof(PolyC) * (size_t)std::max<int64_t>(np, 1));
  y.nblk = o;    o = al(o + sizeof(int32_t) * (size_t)std::max<int64_t>(np, 1));
  y.bstart = o;  o = al(o + sizeof(int64_t) * (size_t)std::max<int64_t>(np, 1));
  y.btot = o;    o = al(o + sizeof(int64_t) * (size_t)blocks(np, kAux));
  y.rec = o;     o = al(o + sizeof(QRec) * (size_t)rows);
  y.small = o;   o = al(o + sizeof(int32_t) * (size_t)rows);
  y.scnt = o;    o = al(o + sizeof(int32_t) * (size_t)std::max<int64_t>(np, 1));
  y.partial = o; o = al(o + sizeof(double) * 4 * (size_t)y.ks * (size_t)std::max<int64_t>(nv, 1));
  y.total = o;
  return y;
}

// Batched 3D adjoint workspace: face records, per-mesh centres and block counts, the block scan,
// Q records and small lists per (mesh, Q) row, FP64 partials per (Q chunk, face), corner adjoints
// and the vertex -> face-corner CSR of the vertex gather.
struct Bb3Layout {
  size_t recs, mc, nblk, bstart, btot, rec, small, scnt, partial, corner, deg, cursor, start, vtot, list, total;
  int ks;
  int64_t per_split, grid;
};

Bb3Layout bb3_layout(int64_t nv, int64_t nf, int64_t nm, int64_t n_q, bool per_mesh_q) {
  Bb3Layout y{};
  y.grid = std::max<int64_t>(1, nm + (nf + kBwdNT - 1) / kBwdNT);   // at least the pair blocks needed
  const int64_t slots = (int64_t)sm_count() * 8;
  const int64_t q_tiles = std::max<int64_t>(1, (n_q + kQTile - 1) / kQTile);
  // Q chunks for 16 waves of 8 blocks per SM, as q_splits (the tail of the last blocks to start):
  // 4,096 polygons x 64^2 Q 17.32 -> 17.04 ms, 1,024 meshes x 32^3 Q 218.5 -> 212.6 ms against 4 waves
  const int64_t k = std::min<int64_t>({std::max<int64_t>(1, (16 * slots + y.grid - 1) / y.grid), q_tiles, 256});
  y.per_split = ((q_tiles + k - 1) / k) * kQTile;
  y.ks = (int)std::max<int64_t>(1, (n_q + y.per_split - 1) / y.per_split);
  const int64_t rows = std::max<int64_t>(per_mesh_q ? n_q : nm * n_q, 1);
  const size_t nf1 = (size_t)std::max<int64_t>(nf, 1), nm1 = (size_t)std::max<int64_t>(nm, 1),
               nv1 = (size_t)std::max<int64_t>(nv, 1);
  size_t o = al(sizeof(WsHeader));
  y.recs = o;    o = al(o + sizeof(Face32) * nf1);
  y.mc = o;      o = al(o + sizeof(PolyC) * nm1);
  y.nblk = o;    o = al(o + sizeof(int32_t) * nm1);
  y.bstart = o;  o = al(o + sizeof(int64_t) * nm1);
  y.btot = o;    o = al(o + sizeof(int64_t) * (size_t)blocks(nm, kAux));
  y.rec = o;     o = al(o + sizeof(QRec) * (size_t)rows);
  y.small = o;   o = al(o + sizeof(int32_t) * (size_t)rows);
  y.scnt = o;    o = al(o + sizeof(int32_t) * nm1);
  y.partial = o; o = al(o + sizeof(double) * 12 * (size_t)y.ks * nf1);
  y.corner = o;  o = al(o + sizeof(double) * 9 * nf1);
  y.deg = o;     o = al(o + sizeof(int32_t) * nv1);
  y.cursor = o;  o = al(o + sizeof(int32_t) * nv1);
  y.start = o;   o = al(o + sizeof(int64_t) * nv1);
  y.vtot = o;    o = al(o + sizeof(int64_t) * (size_t)blocks(nv, kAux));
  y.list = o;    o = al(o + sizeof(int32_t) * 3 * nf1);
  y.total = o;
  return y;
}

// Caller events recorded around the main pair kernel of the current call (set by check_opts).
thread_local cudaEvent_t g_ev_start = nullptr, g_ev_stop = nullptr;

int check_opts(const pft_options* o, Thr& th, bool* tiled = nullptr) {
  pft_options z;
  std::memset(&z, 0, sizeof(z));
  const pft_options& p = o ? *o : z;
  if (p.q_order != PFT_Q_TILED && p.q_order != PFT_Q_AS_GIVEN) return PFT_ERR_INVALID_ARG;
  if (tiled) *tiled = p.q_order == PFT_Q_TILED;
  g_ev_start = static_cast<cudaEvent_t>(p.main_start_event);
  g_ev_stop = static_cast<cudaEvent_t>(p.main_stop_event);
  if (p.precision != PFT_FP32_COMPENSATED) return PFT_ERR_UNSUPPORTED;   // the adjoint runs in FP32
  if (p.q_per_thread != 0 || p.block_threads != 0 || p.k_splits != 0 || p.tile_items != 0)
    return PFT_ERR_UNSUPPORTED;
  float tau = p.face_series_tau == 0.f ? 6.0f : p.face_series_tau;
  if (!(tau > 0.f && tau <= 6.f)) return PFT_ERR_INVALID_ARG;
  const float lo = std::min(tau, 0.05f);
  th = Thr{0.25f * tau * tau, 0.25f * lo * lo, tau > 1.f ? 1 : 0, tau > 3.f ? 1 : 0};
  return PFT_OK;
}

#define PFT_MARK(ev)                                                                        \
  do {                                                                                      \
    if ((ev) != nullptr && cudaEventRecord((ev), st) != cudaSuccess) return PFT_ERR_CUDA; \
  } while (0)

#define PFT_BWD_LAUNCH()                                   \
  do {                                                     \
    if (cudaGetLastError() != cudaSuccess) return PFT_ERR_CUDA; \
    ++g_bwd_launches;                                      \
  } while (0)

// The slot -> Q map of a Q-gradient call (NULL: the caller's order), computed on the stream.
int qg_order(int dim, const QgLayout& y, const double* q, int64_t n_q, void* ws, cudaStream_t st,
             const int32_t*& perm) {
  perm = nullptr;
  if (!y.tiled) return PFT_OK;
  int32_t* p = at<int32_t>(ws, y.qperm);
  if (launch_qorder(dim, q, n_q, 1, kBwdNT, at<void>(ws, y.qscratch), p, st, &g_bwd_launches) != cudaSuccess)
    return PFT_ERR_CUDA;
  perm = p;
  return PFT_OK;
}

}  // namespace
}  // namespace pft

using namespace pft;

namespace pft {
namespace {

// The 3D adjoint after argument checks and the header reset: records, Q weights, the pair
// kernel, corner adjoints, the vertex -> corner CSR and the fixed-order gather.
int mesh3d_backward_body(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
                         const double* q, int64_t n_q, const double* grad_out, float* grad_verts, void* ws,
                         const BwdLayout& y, const Thr& th, WsHeader* h, cudaStream_t st) {
  if (launch_bbox(verts, n_verts, 3, h, st) != cudaSuccess) return PFT_ERR_CUDA;
  if (launch_prep3d(verts, n_verts, faces, n_faces, h, at<void>(ws, y.items), false, at<double>(ws, y.mparts),
                    y.nblk, st) != cudaSuccess)
    return PFT_ERR_CUDA;
  g_bwd_launches += 2;
  k_bq<3><<<blocks(n_q, kAux), kAux, 0, st>>>(q, grad_out, n_q, h, 1.0, at<QRec>(ws, y.qrec), at<int32_t>(ws, y.small));
  PFT_BWD_LAUNCH();
  dim3 grid(blocks(n_faces, kBwdNT), (unsigned)y.ks);
  PFT_MARK(g_ev_start);
  k_bwd<3, 12><<<grid, kBwdNT, 0, st>>>(at<void>(ws, y.items), n_faces, at<QRec>(ws, y.qrec), n_q, y.per_split, th,
                                        at<double>(ws, y.partial), &h->status);
  PFT_BWD_LAUNCH();
  PFT_MARK(g_ev_stop);
  k_bcorner3d<<<blocks(n_faces, kAux), kAux, 0, st>>>(verts, n_verts, faces, n_faces, at<double>(ws, y.partial),
                                                      y.ks, h, at<int32_t>(ws, y.small), q, grad_out,
                                                      at<double>(ws, y.corner));
  PFT_BWD_LAUNCH();
  int32_t* deg = at<int32_t>(ws, y.deg);
  int32_t* cursor = at<int32_t>(ws, y.cursor);
  int64_t* start = at<int64_t>(ws, y.start);
  int64_t* btot = at<int64_t>(ws, y.btot);
  k_zero_i32<<<blocks(n_verts, kAux), kAux, 0, st>>>(deg, n_verts);
  PFT_BWD_LAUNCH();
  k_zero_i32<<<blocks(n_verts, kAux), kAux, 0, st>>>(cursor, n_verts);
  PFT_BWD_LAUNCH();
  k_deg<<<blocks(3 * n_faces, kAux), kAux, 0, st>>>(faces, n_faces, n_verts, deg);
  PFT_BWD_LAUNCH();
  const unsigned nb = blocks(n_verts, kAux);
  k_scan_block<<<nb, kAux, 0, st>>>(deg, n_verts, start, btot);
  PFT_BWD_LAUNCH();
  k_scan_totals<<<1, 32, 0, st>>>(btot, nb);
  PFT_BWD_LAUNCH();
  k_scan_add<<<nb, kAux, 0, st>>>(start, n_verts, btot);
  PFT_BWD_LAUNCH();
  k_fill<<<blocks(3 * n_faces, kAux), kAux, 0, st>>>(faces, n_faces, n_verts, start, cursor, at<int32_t>(ws, y.list));
  PFT_BWD_LAUNCH();
  k_gather3d<<<blocks(n_verts, kAux), kAux, 0, st>>>(n_verts, start, deg, at<int32_t>(ws, y.list),
                                                     at<double>(ws, y.corner), grad_verts);
  PFT_BWD_LAUNCH();
  return PFT_OK;
}

}  // namespace
}  // namespace pft

extern "C" {

size_t pft2d_backward_workspace_size(int64_t n_verts, int64_t n_loops, int64_t n_q, const pft_options* opts) {
  Thr th;
  if (n_verts < 0 || n_loops < 0 || n_q < 0 || check_opts(opts, th) != PFT_OK) return 0;
  return bwd_layout(2, n_verts, n_verts, std::max<int64_t>(n_verts, n_loops + 1), n_q).total;
}

size_t pft3d_backward_workspace_size(int64_t n_verts, int64_t n_faces, int64_t n_q, const pft_options* opts) {
  Thr th;
  if (n_verts < 0 || n_faces < 0 || n_q < 0 || check_opts(opts, th) != PFT_OK) return 0;
  return bwd_layout(3, n_verts, n_faces, n_faces, n_q).total;
}

int pft2d_polygons_backward(const float* verts, int64_t n_verts, const int64_t* loop_off, int64_t n_loops,
                            const double* q, int64_t n_q, const double* grad_out, float* grad_verts, void* ws,
                            size_t ws_bytes, const pft_options* opts, void* stream) {
  g_bwd_launches = 0;
  Thr th;
  if (int e = check_opts(opts, th)) return e;
  if (n_verts < 0 || n_loops < 0 || n_q < 0) return PFT_ERR_INVALID_ARG;
  if (n_verts > 0 && (verts == nullptr || loop_off == nullptr || grad_verts == nullptr || n_loops == 0))
    return PFT_ERR_INVALID_ARG;
  if (n_q > 0 && (q == nullptr || grad_out == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_q > INT32_MAX) return PFT_ERR_UNSUPPORTED;
  const BwdLayout y = bwd_layout(2, n_verts, n_verts, std::max<int64_t>(n_verts, n_loops + 1), n_q);
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < y.total) return PFT_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* h = at<WsHeader>(ws, 0);
  if (launch_init_header(h, st) != cudaSuccess) return PFT_ERR_CUDA;
  ++g_bwd_launches;
  if (n_verts == 0) return PFT_OK;
  if (n_q == 0) {
    return cudaMemsetAsync(grad_verts, 0, sizeof(float) * 2 * (size_t)n_verts, st) == cudaSuccess ? PFT_OK
                                                                                                  : PFT_ERR_CUDA;
  }
  if (launch_bbox(verts, n_verts, 2, h, st) != cudaSuccess) return PFT_ERR_CUDA;
  if (launch_prep2d(verts, n_verts, loop_off, n_loops, h, at<void>(ws, y.items), false, at<double>(ws, y.mparts),
                    y.nblk, st) != cudaSuccess)
    return PFT_ERR_CUDA;
  g_bwd_launches += 2;
  k_bq<2><<<blocks(n_q, kAux), kAux, 0, st>>>(q, grad_out, n_q, h, 2.0, at<QRec>(ws, y.qrec), at<int32_t>(ws, y.small));
  PFT_BWD_LAUNCH();
  dim3 grid(blocks(n_verts, kBwdNT), (unsigned)y.ks);
  PFT_MARK(g_ev_start);
  k_bwd<2, 4><<<grid, kBwdNT, 0, st>>>(at<void>(ws, y.items), n_verts, at<QRec>(ws, y.qrec), n_q, y.per_split, th,
                                       at<double>(ws, y.partial), &h->status);
  PFT_BWD_LAUNCH();
  PFT_MARK(g_ev_stop);
  k_bvert2d<<<blocks(n_verts, kAux), kAux, 0, st>>>(verts, n_verts, loop_off, n_loops, at<double>(ws, y.partial),
                                                    y.ks, h, at<int32_t>(ws, y.small), q, grad_out, grad_verts);
  PFT_BWD_LAUNCH();
  return PFT_OK;
}

int pft3d_mesh_backward(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces, const double* q,
                        int64_t n_q, const double* grad_out, float* grad_verts, void* ws, size_t ws_bytes,
                        const pft_options* opts, void* stream) {
  g_bwd_launches = 0;
  Thr th;
  if (int e = check_opts(opts, th)) return e;
  if (n_verts < 0 || n_faces < 0 || n_q < 0) return PFT_ERR_INVALID_ARG;
  if (n_verts > 0 && (verts == nullptr || grad_verts == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_faces > 0 && faces == nullptr) return PFT_ERR_INVALID_ARG;
  if (n_q > 0 && (q == nullptr || grad_out == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_q > INT32_MAX || n_verts > INT32_MAX || 3 * n_faces > INT32_MAX) return PFT_ERR_UNSUPPORTED;
  const BwdLayout y = bwd_layout(3, n_verts, n_faces, n_faces, n_q);
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < y.total) return PFT_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* h = at<WsHeader>(ws, 0);
  if (launch_init_header(h, st) != cudaSuccess) return PFT_ERR_CUDA;
  ++g_bwd_launches;
  if (n_verts == 0) return PFT_OK;
  if (n_faces == 0 || n_q == 0) {
    return cudaMemsetAsync(grad_verts, 0, sizeof(float) * 3 * (size_t)n_verts, st) == cudaSuccess ? PFT_OK
                                                                                                  : PFT_ERR_CUDA;
  }
  return mesh3d_backward_body(verts, n_verts, faces, n_faces, q, n_q, grad_out, grad_verts, ws, y, th, h, st);
}

size_t pft3d_polymesh_backward_workspace_size(int64_t n_verts, int64_t n_idx, int64_t n_faces, int64_t n_q,
                                              const pft_options* opts) {
  Thr th;
  if (n_verts < 0 || n_idx < 0 || n_faces < 0 || n_q < 0 || n_idx < 3 * n_faces || check_opts(opts, th) != PFT_OK)
    return 0;
  const int64_t nt = n_idx - 2 * n_faces;
  const size_t tri_bytes = (sizeof(int32_t) * 3 * (size_t)std::max<int64_t>(nt, 1) + 255) / 256 * 256;
  return bwd_layout(3, n_verts, nt, nt, n_q).total + tri_bytes;
}

int pft3d_polymesh_backward(const float* verts, int64_t n_verts, const int32_t* face_idx, int64_t n_idx,
                            const int64_t* face_off, int64_t n_faces, const double* q, int64_t n_q,
                            const double* grad_out, float* grad_verts, void* ws, size_t ws_bytes,
                            const pft_options* opts, void* stream) {
  g_bwd_launches = 0;
  Thr th;
  if (int e = check_opts(opts, th)) return e;
  if (n_verts < 0 || n_idx < 0 || n_faces < 0 || n_q < 0 || n_idx < 3 * n_faces) return PFT_ERR_INVALID_ARG;
  if (n_verts > 0 && (verts == nullptr || grad_verts == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_faces > 0 && (face_idx == nullptr || face_off == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_q > 0 && (q == nullptr || grad_out == nullptr)) return PFT_ERR_INVALID_ARG;
  const int64_t n_tris = n_idx - 2 * n_faces;
  if (n_q > INT32_MAX || n_verts > INT32_MAX || 3 * n_tris > INT32_MAX) return PFT_ERR_UNSUPPORTED;
  const BwdLayout y = bwd_layout(3, n_verts, n_tris, n_tris, n_q);
  const size_t need = pft3d_polymesh_backward_workspace_size(n_verts, n_idx, n_faces, n_q, opts);
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < need) return PFT_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* h = at<WsHeader>(ws, 0);
  if (launch_init_header(h, st) != cudaSuccess) return PFT_ERR_CUDA;
  ++g_bwd_launches;
  if (n_verts == 0) return PFT_OK;
  if (n_faces == 0 || n_q == 0) {
    return cudaMemsetAsync(grad_verts, 0, sizeof(float) * 3 * (size_t)n_verts, st) == cudaSuccess ? PFT_OK
                                                                                                  : PFT_ERR_CUDA;
  }
  int32_t* tris = at<int32_t>(ws, y.total);
  if (launch_fan3d(face_idx, n_idx, face_off, n_faces, tris, n_tris, h, st) != cudaSuccess) return PFT_ERR_CUDA;
  ++g_bwd_launches;
  return mesh3d_backward_body(verts, n_verts, tris, n_tris, q, n_q, grad_out, grad_verts, ws, y, th, h, st);
}

size_t pft3d_qgrad_workspace_size(int64_t n_verts, int64_t n_faces, int64_t n_q, const pft_options* opts) {
  Thr th;
  bool tiled;
  if (n_verts < 0 || n_faces < 0 || n_q < 0 || check_opts(opts, th, &tiled) != PFT_OK) return 0;
  return qg_layout(n_faces, n_q, tiled).total;
}

int pft3d_mesh_qgrad(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces, const double* q,
                     int64_t n_q, const double* grad_out, double* grad_q, void* ws, size_t ws_bytes,
                     const pft_options* opts, void* stream) {
  g_bwd_launches = 0;
  Thr th;
  bool tiled;
  if (int e = check_opts(opts, th, &tiled)) return e;
  if (n_verts < 0 || n_faces < 0 || n_q < 0) return PFT_ERR_INVALID_ARG;
  if (n_faces > 0 && (faces == nullptr || verts == nullptr || n_verts == 0)) return PFT_ERR_INVALID_ARG;
  if (n_q > 0 && (q == nullptr || grad_out == nullptr || grad_q == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_q > INT32_MAX || n_verts > INT32_MAX) return PFT_ERR_UNSUPPORTED;
  const QgLayout y = qg_layout(n_faces, n_q, tiled);
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < y.total) return PFT_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* h = at<WsHeader>(ws, 0);
  if (launch_init_header(h, st) != cudaSuccess) return PFT_ERR_CUDA;
  ++g_bwd_launches;
  if (n_q == 0) return PFT_OK;
  if (n_faces == 0)
    return cudaMemsetAsync(grad_q, 0, sizeof(double) * 3 * (size_t)n_q, st) == cudaSuccess ? PFT_OK : PFT_ERR_CUDA;
  if (launch_bbox(verts, n_verts, 3, h, st) != cudaSuccess) return PFT_ERR_CUDA;
  if (launch_prep3d(verts, n_verts, faces, n_faces, h, at<void>(ws, y.items), false, at<double>(ws, y.mparts),
                    y.nblk, st) != cudaSuccess)
    return PFT_ERR_CUDA;
  g_bwd_launches += 2;
  const int32_t* perm = nullptr;
  if (int e = qg_order(3, y, q, n_q, ws, st, perm)) return e;
  k_bq<3><<<blocks(n_q, kAux), kAux, 0, st>>>(q, grad_out, n_q, h, 1.0, at<QRec>(ws, y.qrec), at<int32_t>(ws, y.small),
                                              perm);
  PFT_BWD_LAUNCH();
  dim3 grid(blocks(n_q, kBwdNT), (unsigned)y.ks);
  PFT_MARK(g_ev_start);
  k_qgrad<<<grid, kBwdNT, 0, st>>>(at<Face32>(ws, y.items), n_faces, y.per_split, at<QRec>(ws, y.qrec), n_q, th,
                                   at<double>(ws, y.partial), &h->status, perm);
  PFT_BWD_LAUNCH();
  PFT_MARK(g_ev_stop);
  k_qfinal<<<blocks(n_q, kAux), kAux, 0, st>>>(q, grad_out, n_q, at<double>(ws, y.partial), y.ks, h, grad_q);
  PFT_BWD_LAUNCH();
  k_qsmall_part<<<(unsigned)(4 * sm_count()), kAux, 0, st>>>(verts, n_verts, faces, n_faces, q, h,
                                                             at<int32_t>(ws, y.small), y.slots,
                                                             at<double>(ws, y.spart));
  PFT_BWD_LAUNCH();
  k_qsmall_fin<<<blocks(n_q, kAux), kAux, 0, st>>>(n_faces, q, grad_out, h, at<int32_t>(ws, y.small), y.slots,
                                                   at<double>(ws, y.spart), grad_q);
  PFT_BWD_LAUNCH();
  return PFT_OK;
}

size_t pft2d_qgrad_workspace_size(int64_t n_verts, int64_t n_loops, int64_t n_q, const pft_options* opts) {
  Thr th;
  bool tiled;
  if (n_verts < 0 || n_loops < 0 || n_q < 0 || check_opts(opts, th, &tiled) != PFT_OK) return 0;
  return qg2_layout(n_verts, std::max<int64_t>(n_verts, n_loops + 1), n_q, tiled).total;
}

int pft2d_polygons_qgrad(const float* verts, int64_t n_verts, const int64_t* loop_off, int64_t n_loops,
                         const double* q, int64_t n_q, const double* grad_out, double* grad_q, void* ws,
                         size_t ws_bytes, const pft_options* opts, void* stream) {
  g_bwd_launches = 0;
  Thr th;
  bool tiled;
  if (int e = check_opts(opts, th, &tiled)) return e;
  if (n_verts < 0 || n_loops < 0 || n_q < 0) return PFT_ERR_INVALID_ARG;
  if (n_verts > 0 && (verts == nullptr || loop_off == nullptr || n_loops == 0)) return PFT_ERR_INVALID_ARG;
  if (n_q > 0 && (q == nullptr || grad_out == nullptr || grad_q == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_q > INT32_MAX) return PFT_ERR_UNSUPPORTED;
  const QgLayout y = qg2_layout(n_verts, std::max<int64_t>(n_verts, n_loops + 1), n_q, tiled);
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < y.total) return PFT_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* h = at<WsHeader>(ws, 0);
  if (launch_init_header(h, st) != cudaSuccess) return PFT_ERR_CUDA;
  ++g_bwd_launches;
  if (n_q == 0) return PFT_OK;
  if (n_verts == 0)
    return cudaMemsetAsync(grad_q, 0, sizeof(double) * 2 * (size_t)n_q, st) == cudaSuccess ? PFT_OK : PFT_ERR_CUDA;
  if (launch_bbox(verts, n_verts, 2, h, st) != cudaSuccess) return PFT_ERR_CUDA;
  if (launch_prep2d(verts, n_verts, loop_off, n_loops, h, at<void>(ws, y.items), false, at<double>(ws, y.mparts),
                    y.nblk, st) != cudaSuccess)
    return PFT_ERR_CUDA;
  g_bwd_launches += 2;
  const int32_t* perm = nullptr;
  if (int e = qg_order(2, y, q, n_q, ws, st, perm)) return e;
  k_bq<2><<<blocks(n_q, kAux), kAux, 0, st>>>(q, grad_out, n_q, h, 2.0, at<QRec>(ws, y.qrec), at<int32_t>(ws, y.small),
                                              perm);
  PFT_BWD_LAUNCH();
  dim3 grid(blocks(n_q, kBwdNT), (unsigned)y.ks);
  PFT_MARK(g_ev_start);
  k_qgrad2d<<<grid, kBwdNT, 0, st>>>(at<Seg32>(ws, y.items), n_verts, y.per_split, at<QRec>(ws, y.qrec), n_q,
                                     at<double>(ws, y.partial), &h->status, perm);
  PFT_BWD_LAUNCH();
  PFT_MARK(g_ev_stop);
  k_qfinal2d<<<blocks(n_q, kAux), kAux, 0, st>>>(q, grad_out, n_q, at<double>(ws, y.partial), y.ks, h, grad_q);
  PFT_BWD_LAUNCH();
  k_qsmall2d_part<<<(unsigned)(4 * sm_count()), kAux, 0, st>>>(verts, n_verts, loop_off, n_loops, q, h,
                                                               at<int32_t>(ws, y.small), y.slots,
                                                               at<double>(ws, y.spart));
  PFT_BWD_LAUNCH();
  k_qsmall2d_fin<<<blocks(n_q, kAux), kAux, 0, st>>>(n_verts, q, grad_out, h, at<int32_t>(ws, y.small), y.slots,
                                                     at<double>(ws, y.spart), grad_q);
  PFT_BWD_LAUNCH();
  return PFT_OK;
}

size_t pft2d_batched_backward_workspace_size(int64_t n_verts, int64_t n_polys, int64_t n_q, int per_polygon_q,
                                             const pft_options* opts) {
  Thr th;
  if (n_verts < 0 || n_polys < 0 || n_q < 0 || check_opts(opts, th) != PFT_OK) return 0;
  return bb_layout(n_verts, n_polys, n_q, per_polygon_q != 0).total;
}

int pft2d_polygons_batched_backward(const float* verts, int64_t n_verts, const int64_t* poly_off, int64_t n_polys,
                                    const double* q, const int64_t* q_off, int64_t n_q, const double* grad_out,
                                    float* grad_verts, void* ws, size_t ws_bytes, const pft_options* opts,
                                    void* stream) {
  g_bwd_launches = 0;
  Thr th;
  if (int e = check_opts(opts, th)) return e;
  if (n_verts < 0 || n_polys < 0 || n_q < 0) return PFT_ERR_INVALID_ARG;
  if (n_verts > 0 && (verts == nullptr || poly_off == nullptr || grad_verts == nullptr || n_polys == 0))
    return PFT_ERR_INVALID_ARG;
  if (n_q > 0 && (q == nullptr || grad_out == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_q > INT32_MAX || n_polys > INT32_MAX || n_polys * n_q > (int64_t)1 << 40) return PFT_ERR_UNSUPPORTED;
  if (q_off != nullptr && n_polys == 0) return PFT_ERR_INVALID_ARG;
  const BbLayout y = bb_layout(n_verts, n_polys, n_q, q_off != nullptr);
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < y.total) return PFT_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* h = at<WsHeader>(ws, 0);
  if (launch_init_header(h, st) != cudaSuccess) return PFT_ERR_CUDA;
  ++g_bwd_launches;
  if (n_verts == 0) return PFT_OK;
  if (n_q == 0)
    return cudaMemsetAsync(grad_verts, 0, sizeof(float) * 2 * (size_t)n_verts, st) == cudaSuccess ? PFT_OK
                                                                                                 : PFT_ERR_CUDA;
  Seg32* segs = at<Seg32>(ws, y.segs);
  PolyC* pc = at<PolyC>(ws, y.pc);
  int32_t* nblk = at<int32_t>(ws, y.nblk);
  int64_t* bstart = at<int64_t>(ws, y.bstart);
  int64_t* btot = at<int64_t>(ws, y.btot);
  k_bbprep<<<(unsigned)n_polys, kAux, 0, st>>>(verts, n_verts, poly_off, n_polys, segs, pc, nblk, h);
  PFT_BWD_LAUNCH();
  const unsigned nb = blocks(n_polys, kAux);
  k_scan_block<<<nb, kAux, 0, st>>>(nblk, n_polys, bstart, btot);
  PFT_BWD_LAUNCH();
  k_scan_totals<<<1, 32, 0, st>>>(btot, nb);
  PFT_BWD_LAUNCH();
  k_scan_add<<<nb, kAux, 0, st>>>(bstart, n_polys, btot);
  PFT_BWD_LAUNCH();
  k_bbq<2><<<(unsigned)n_polys, kAux, 0, st>>>(q, q_off, grad_out, n_q, n_polys, pc, at<QRec>(ws, y.rec),
                                            at<int32_t>(ws, y.small), at<int32_t>(ws, y.scnt), h);
  PFT_BWD_LAUNCH();
  if (y.grid > INT32_MAX) return PFT_ERR_UNSUPPORTED;
  dim3 grid((unsigned)y.grid, (unsigned)y.ks);
  PFT_MARK(g_ev_start);
  k_bbwd<<<grid, kBwdNT, 0, st>>>(segs, n_verts, poly_off, n_polys, bstart, nblk, at<QRec>(ws, y.rec), q_off, n_q,
                                  y.per_split, th, at<double>(ws, y.partial), &h->status);
  PFT_BWD_LAUNCH();
  PFT_MARK(g_ev_stop);
  k_bbvert<<<blocks(n_verts, kAux), kAux, 0, st>>>(verts, n_verts, poly_off, n_polys, at<double>(ws, y.partial), y.ks,
                                                   pc, at<int32_t>(ws, y.small), at<int32_t>(ws, y.scnt), q, q_off,
                                                   n_q, grad_out, grad_verts);
  PFT_BWD_LAUNCH();
  return PFT_OK;
}

size_t pft3d_batched_backward_workspace_size(int64_t n_verts, int64_t n_faces, int64_t n_meshes, int64_t n_q,
                                             int per_mesh_q, const pft_options* opts) {
  Thr th;
  if (n_verts < 0 || n_faces < 0 || n_meshes < 0 || n_q < 0 || check_opts(opts, th) != PFT_OK) return 0;
  return bb3_layout(n_verts, n_faces, n_meshes, n_q, per_mesh_q != 0).total;
}

int pft3d_meshes_batched_backward(const float* verts, int64_t n_verts, const int32_t* faces, int64_t n_faces,
                                  const int64_t* mesh_off, int64_t n_meshes, const double* q, const int64_t* q_off,
                                  int64_t n_q, const double* grad_out, float* grad_verts, void* ws, size_t ws_bytes,
                                  const pft_options* opts, void* stream) {
  g_bwd_launches = 0;
  Thr th;
  if (int e = check_opts(opts, th)) return e;
  if (n_verts < 0 || n_faces < 0 || n_meshes < 0 || n_q < 0) return PFT_ERR_INVALID_ARG;
  if (n_verts > 0 && (verts == nullptr || grad_verts == nullptr)) return PFT_ERR_INVALID_ARG;
  if (n_faces > 0 && (faces == nullptr || mesh_off == nullptr || n_meshes == 0 || n_verts == 0))
    return PFT_ERR_INVALID_ARG;
  if (n_q > 0 && (q == nullptr || grad_out == nullptr)) return PFT_ERR_INVALID_ARG;
  if (q_off != nullptr && n_meshes == 0) return PFT_ERR_INVALID_ARG;
  if (n_q > INT32_MAX || n_verts > INT32_MAX || 3 * n_faces > INT32_MAX || n_meshes > INT32_MAX ||
      n_meshes * n_q > (int64_t)1 << 40)
    return PFT_ERR_UNSUPPORTED;
  const Bb3Layout y = bb3_layout(n_verts, n_faces, n_meshes, n_q, q_off != nullptr);
  if (ws == nullptr || reinterpret_cast<uintptr_t>(ws) % 256 != 0 || ws_bytes < y.total) return PFT_ERR_WORKSPACE;
  if (y.grid > INT32_MAX) return PFT_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader* h = at<WsHeader>(ws, 0);
  if (launch_init_header(h, st) != cudaSuccess) return PFT_ERR_CUDA;
  ++g_bwd_launches;
  if (n_verts == 0) return PFT_OK;
  if (n_q == 0 || n_faces == 0)
    return cudaMemsetAsync(grad_verts, 0, sizeof(float) * 3 * (size_t)n_verts, st) == cudaSuccess ? PFT_OK
                                                                                                 : PFT_ERR_CUDA;
  Face32* recs = at<Face32>(ws, y.recs);
  PolyC* mc = at<PolyC>(ws, y.mc);
  int32_t* nblk = at<int32_t>(ws, y.nblk);
  int64_t* bstart = at<int64_t>(ws, y.bstart);
  int64_t* btot = at<int64_t>(ws, y.btot);
  k_bbprep3<<<(unsigned)n_meshes, kAux, 0, st>>>(verts, n_verts, faces, n_faces, mesh_off, n_meshes, recs, mc, nblk,
                                                 h);
  PFT_BWD_LAUNCH();
  const unsigned nb = blocks(n_meshes, kAux);
  k_scan_block<<<nb, kAux, 0, st>>>(nblk, n_meshes, bstart, btot);
  PFT_BWD_LAUNCH();
  k_scan_totals<<<1, 32, 0, st>>>(btot, nb);
  PFT_BWD_LAUNCH();
  k_scan_add<<<nb, kAux, 0, st>>>(bstart, n_meshes, btot);
  PFT_BWD_LAUNCH();
  k_bbq<3><<<(unsigned)n_meshes, kAux, 0, st>>>(q, q_off, grad_out, n_q, n_meshes, mc, at<QRec>(ws, y.rec),
                                                at<int32_t>(ws, y.small), at<int32_t>(ws, y.scnt), h);
  PFT_BWD_LAUNCH();
  dim3 grid((unsigned)y.grid, (unsigned)y.ks);
  PFT_MARK(g_ev_start);
  k_bbwd3<<<grid, kBwdNT, 0, st>>>(recs, n_faces, mesh_off, n_meshes, bstart, nblk, at<QRec>(ws, y.rec), q_off, n_q,
                                   y.per_split, th, at<double>(ws, y.partial), &h->status);
  PFT_BWD_LAUNCH();
  PFT_MARK(g_ev_stop);
  k_bbcorner3<<<blocks(n_faces, kAux), kAux, 0, st>>>(verts, n_verts, faces, n_faces, mesh_off, n_meshes,
                                                      at<double>(ws, y.partial), y.ks, mc, at<int32_t>(ws, y.small),
                                                      at<int32_t>(ws, y.scnt), q, q_off, n_q, grad_out,
                                                      at<double>(ws, y.corner));
  PFT_BWD_LAUNCH();
  int32_t* deg = at<int32_t>(ws, y.deg);
  int32_t* cursor = at<int32_t>(ws, y.cursor);
  int64_t* start = at<int64_t>(ws, y.start);
  int64_t* vtot = at<int64_t>(ws, y.vtot);
  k_zero_i32<<<blocks(n_verts, kAux), kAux, 0, st>>>(deg, n_verts);
  PFT_BWD_LAUNCH();
  k_zero_i32<<<blocks(n_verts, kAux), kAux, 0, st>>>(cursor, n_verts);
  PFT_BWD_LAUNCH();
  k_deg<<<blocks(3 * n_faces, kAux), kAux, 0, st>>>(faces, n_faces, n_verts, deg);
  PFT_BWD_LAUNCH();
  const unsigned nbv = blocks(n_verts, kAux);
  k_scan_block<<<nbv, kAux, 0, st>>>(deg, n_verts, start, vtot);
  PFT_BWD_LAUNCH();
  k_scan_totals<<<1, 32, 0, st>>>(vtot, nbv);
  PFT_BWD_LAUNCH();
  k_scan_add<<<nbv, kAux, 0, st>>>(start, n_verts, vtot);
  PFT_BWD_LAUNCH();
  k_fill<<<blocks(3 * n_faces, kAux), kAux, 0, st>>>(faces, n_faces, n_verts, start, cursor, at<int32_t>(ws, y.list));
  PFT_BWD_LAUNCH();
  k_gather3d<<<blocks(n_verts, kAux), kAux, 0, st>>>(n_verts, start, deg, at<int32_t>(ws, y.list),
                                                     at<double>(ws, y.corner), grad_verts);
  PFT_BWD_LAUNCH();
  return PFT_OK;
}

int pft_backward_last_launch_count(void) { return g_bwd_launches; }

}  // extern "C"
