// pft_pairs.cuh -- per-pair arithmetic of the divergence-theorem sums and the
// per-tile policies (record type, Q registers, accumulators) shared by the
// forward kernels (single shape and batched).
#pragma once

#include <type_traits>

#include "pft_kernels.cuh"

namespace pft {

constexpr int kStages = 4;

// Thresholds on P (see the 3D face term below): p_hi = tau^2/4, p_lo = tau_lo^2/4.
struct Thr {
  float hi, lo;
  int longs;    // tau > 1: warps whose faces are not all below kPShort take a longer series (adjoint)
  int xlongs;   // tau > 3: warps whose faces are not all below kPLong take the extra-long series (adjoint)
  int64_t pair_end;   // faces [0, pair_end) come in pairs sharing their first edge (forward, 3D FP32)
};
constexpr float kTauLo = 0.05f;
constexpr float kPShort = 0.25f;   // P below which the short series (k <= 7) suffices (tau = 1)
constexpr float kP9 = 1.0f;        // P below which the k <= 9 series suffices (tau = 2)
constexpr float kPLong = 2.25f;    // P below which the long series (k <= 11) suffices (tau = 3)
constexpr float kP13 = 4.0f;       // P below which the k <= 13 series suffices (tau = 4)

// Resident blocks per SM the register budget is sized for: 16-24 warps of
// 256 threads, fewer registers per thread for fewer Q points per thread.  The
// 3D default (R = 4, 128 threads) is held to 102 registers for 5 blocks (20
// warps), which it fits without spilling and which ran 9 % faster than 4 blocks.
// (FP64 paths: one block, so that the double-precision temporaries never spill.)
template <class Pol, int R, int NT>
constexpr int kMinBlocks = sizeof(typename Pol::QT) == 8 ? 1
                           : (Pol::kDim == 3 && R == 4 && NT == 128) ? 5
                           : (NT == 256 ? 1 : 2) * (R >= 8 ? 1 : (R == 4 ? 2 : 3));

// ---------------------------------------------------------------------------
// Per-pair arithmetic.
// ---------------------------------------------------------------------------

// 2D, Eq. 6 (Sec. 2): the segment p0 -> p1 contributes
//   -i (Qx Dy - Qy Dx) sinc(Q.D/2) exp(iQ.m)           (times 1/|Q|^2, applied later)
// Records hold m and D/2, so w below is half the cross product; the factor 2
// and 1/|Q|^2 are applied in FP64 by the finalize kernel.  The term itself is
// evaluated in Pol2F32::tile (the sinc of |Q.D/2| > pi is a warp-uniform branch).

__device__ __forceinline__ double sinc_f64(double u) {
  const double u2 = u * u;
  if (u2 < 1e-2) {   // Taylor through u^10: truncation < 1e-18 at |u| = 0.1
    double p = fma(u2, -1.0 / 39916800.0, 1.0 / 362880.0);
    p = fma(u2, p, -1.0 / 5040.0);
    p = fma(u2, p, 1.0 / 120.0);
    p = fma(u2, p, -1.0 / 6.0);
    return fma(u2, p, 1.0);
  }
  return sin(u) / u;
}

__device__ __forceinline__ void seg_pair_f64(double qx, double qy, const Seg64& s, double& re, double& im) {
  const double ph = fma(qx, s.mx, qy * s.my);
  const double u = fma(qx, s.hx, qy * s.hy);
  const double w = fma(qx, s.hy, -qy * s.hx);
  double sn, cs;
  sincos(ph, &sn, &cs);
  const double ws = w * sinc_f64(u);
  re = ws * sn;
  im = -ws * cs;
}

// 3D, Eq. 14 with the sign fixed (Sec. 3).  With X = N x Q, s = Q.N and the
// corner phases a_k = Q.(p_k - centroid) (a_0 + a_1 + a_2 = 0), a face gives
//   |Q|^2 I_m = -s exp(i mu) Z,     mu = Q.centroid,
//   Z = (1/|X|^2) sum_l w_l sinc(u_l) exp(i psi_l)         (edge sum)
// with w_l = Q.(d_l x N) = b_{l+1} - b_l, b_k = (p_k - centroid).X,
// u_l = (a_{l+1} - a_l)/2 and psi_l = (a_l + a_{l+1})/2 = -a_{l+2}/2.
// The edge sum cancels to O(spread) of its terms when the phase spread of the
// face is small (it is 0/0 for Q parallel to N); there the same face integral
// (Eq. 13) is taken from its series, Z = i G,
//   G = sum_k i^k h_k(a) / (k+2)!,   h_k = P h_{k-2} + T h_{k-3},
// P = a0^2 + a0 a1 + a1^2 (= h_2), T = a0 a1 a2 (= h_3); P < tau^2/4 implies
// max_l |Q.d_l| < tau.  The series is kept through k = 7 for P < 1/4, k = 9 for
// P < 1, k = 11 for P < 9/4, k = 13 for P < 4 and k = 17 for P < 9; the omitted
// terms stay below 4e-9 in each (|G| <= 1/2).
//
// Branch choice, per face and warp: the series is taken for all of a thread's
// Q points when every Q point of every lane of the warp has P < p_hi = tau^2/4,
// in the shortest of the five forms whose bound every one of them meets;
// otherwise the edge sum, except for Q points with P < p_lo = tau_lo^2/4
// (tau_lo = min(tau, 0.05): below it the edge sum would lose more than ~4 bits
// to cancellation), which are redone with the short series.  All three evaluate
// the same face integral, so the choice only moves rounding; the R Q points of
// a thread share the branch, so their arithmetic interleaves.

// Projections shared by both branches.  A = g.xyz, q0.x  B = q0.yz, q1.xy  C = q1.z, N.xyz
__device__ __forceinline__ void face_common(float qx, float qy, float qz, const float4 A, const float4 B,
                                            const float4 C, float& mu, float& a0, float& a1, float& s, float& P) {
  mu = fmaf(qx, A.x, fmaf(qy, A.y, qz * A.z));
  a0 = fmaf(qx, A.w, fmaf(qy, B.x, qz * B.y));
  a1 = fmaf(qx, B.z, fmaf(qy, B.w, qz * C.x));
  s = fmaf(qx, C.y, fmaf(qy, C.z, qz * C.w));
  P = fmaf(a0, a0 + a1, a1 * a1);
}

// As face_common, with T = a0 a1 a2 as well: s1 = a0 + a1 and p1 = a0 a1 give
// P = s1^2 - p1 and T = -p1 s1.
template <class V>
__device__ __forceinline__ void face_common_pt(V qx, V qy, V qz, const float4 A, const float4 B,
                                               const float4 C, V& mu, V& a0, V& a1, V& s, V& P,
                                               V& T) {
  mu = vfma(qx, vs<V>(A.x), vfma(qy, vs<V>(A.y), vmul(qz, vs<V>(A.z))));
  a0 = vfma(qx, vs<V>(A.w), vfma(qy, vs<V>(B.x), vmul(qz, vs<V>(B.y))));
  a1 = vfma(qx, vs<V>(B.z), vfma(qy, vs<V>(B.w), vmul(qz, vs<V>(C.x))));
  s = vfma(qx, vs<V>(C.y), vfma(qy, vs<V>(C.z), vmul(qz, vs<V>(C.w))));
  const V s1 = vadd(a0, a1), p1 = vmul(a0, a1);
  P = vfma(s1, s1, vneg(p1));
  T = vmul(vneg(p1), s1);
}

// Z = i G from the face-integral series.
// Short form (P < 1/4, i.e. tau <= 1): h_k through k = 7,
//   G_re = 1/2! - P/4! + P^2/6! - (P^3 + T^2)/8!,  G_im = T (-1/5! + 2P/7! - 3P^2/9!);
// the omitted terms (k >= 8) are below 2e-9 (|G| <= 1/2).
template <class V>
__device__ __forceinline__ void face_series(V T, V P, V& zr, V& zi) {
  V gre = vfma(P, vs<V>(-2.48015873e-5f), vs<V>(1.38888889e-3f));   // -1/8!, 1/6!
  gre = vfma(P, gre, vs<V>(-4.16666667e-2f));                     // -1/4!
  gre = vfma(P, gre, vs<V>(0.5f));                                // 1/2!
  gre = vfma(vmul(T, T), vs<V>(-2.48015873e-5f), gre);                 // -T^2/8!
  const V gim = vmul(T, vfma(P, vfma(P, vs<V>(-8.26719577e-6f), vs<V>(3.96825397e-4f)), vs<V>(-8.33333333e-3f)));  // -3/9!, 2/7!, -1/5!
  zr = vneg(gim);
  zi = gre;
}

// Long form (P < 9/4, i.e. tau <= 3): h_k through k = 11, with
//   h8 = P^4 + 3P T^2, h9 = 4P^3 T + T^3, h10 = P^5 + 6P^2 T^2, h11 = 5P^4 T + 4P T^3;
// G_re = A(P) + T^2 B(P),  G_im = T (D(P) + T^2 E(P)); the omitted terms (k >= 12)
// are below 4e-9 (|G| <= 1/2).
template <class V>
__device__ __forceinline__ void face_series_long(V T, V P, V& zr, V& zi) {
  const V T2 = vmul(T, T);
  V A = vfma(P, vs<V>(-2.087675588e-9f), vs<V>(2.75573192e-7f));    // -1/12!, 1/10!
  A = vfma(P, A, vs<V>(-2.48015873e-5f));                         // -1/8!
  A = vfma(P, A, vs<V>(1.38888889e-3f));                          // 1/6!
  A = vfma(P, A, vs<V>(-4.16666667e-2f));                         // -1/4!
  A = vfma(P, A, vs<V>(0.5f));                                    // 1/2!
  V B = vfma(P, vs<V>(-1.252605397e-8f), vs<V>(8.26719577e-7f));    // -6/12!, 3/10!
  B = vfma(P, B, vs<V>(-2.48015873e-5f));                         // -1/8!
  const V gre = vfma(T2, B, A);
  V D = vfma(P, vs<V>(-8.029522047e-10f), vs<V>(1.002084318e-7f));   // -5/13!, 4/11!
  D = vfma(P, D, vs<V>(-8.26719577e-6f));                         // -3/9!
  D = vfma(P, D, vs<V>(3.96825397e-4f));                          // 2/7!
  D = vfma(P, D, vs<V>(-8.33333333e-3f));                         // -1/5!
  const V E = vfma(P, vs<V>(-6.423617749e-10f), vs<V>(2.505210794e-8f));   // -4/13!, 1/11!
  const V gim = vmul(T, vfma(T2, E, D));
  zr = vneg(gim);
  zi = gre;
}

// Intermediate forms.  With h_k = sum over 2i + 3j = k of C(i + j, i) P^i T^j, the
// coefficient of P^i T^j is +-C(i + j, i)/(2i + 3j + 2)! (the sign that of i^k), and
//   G_re = A0(P) + T^2 (A2(P) + T^2 A4(P)),  G_im = T (D1(P) + T^2 (D3(P) + T^2 D5(P)))
// keep the terms with k <= K.  Omitted terms: k <= 9 on P < 1 below 4e-9, k <= 13 on
// P < 4 below 3e-9 (|G| <= 1/2).  (A k <= 15 form for 4 <= P < 25/4 would save a
// further 6 operations per pair there, but the larger loop body ran slower.)
template <class V>
__device__ __forceinline__ void face_series_k9(V T, V P, V& zr, V& zi) {
  const V T2 = vmul(T, T);
  V A0 = vfma(P, vs<V>(2.755731922e-07f), vs<V>(-2.480158730e-05f));   // 1/10!, -1/8!
  A0 = vfma(P, A0, vs<V>(1.388888889e-03f));                         // 1/6!
  A0 = vfma(P, A0, vs<V>(-4.166666667e-02f));                        // -1/4!
  A0 = vfma(P, A0, vs<V>(0.5f));                                     // 1/2!
  const V A2 = vfma(P, vs<V>(8.267195767e-07f), vs<V>(-2.480158730e-05f));   // 3/10!, -1/8!
  V D1 = vfma(P, vs<V>(1.002084335e-07f), vs<V>(-8.267195767e-06f));   // 4/11!, -3/9!
  D1 = vfma(P, D1, vs<V>(3.968253968e-04f));                         // 2/7!
  D1 = vfma(P, D1, vs<V>(-8.333333333e-03f));                        // -1/5!
  const V gre = vfma(T2, A2, A0);
  const V gim = vmul(T, vfma(T2, vs<V>(2.505210839e-08f), D1));      // 1/11!
  zr = vneg(gim);
  zi = gre;
}

template <class V>
__device__ __forceinline__ void face_series_k13(V T, V P, V& zr, V& zi) {
  const V T2 = vmul(T, T);
  V A0 = vfma(P, vs<V>(1.147074560e-11f), vs<V>(-2.087675699e-09f));   // 1/14!, -1/12!
  A0 = vfma(P, A0, vs<V>(2.755731922e-07f));                         // 1/10!
  A0 = vfma(P, A0, vs<V>(-2.480158730e-05f));                        // -1/8!
  A0 = vfma(P, A0, vs<V>(1.388888889e-03f));                         // 1/6!
  A0 = vfma(P, A0, vs<V>(-4.166666667e-02f));                        // -1/4!
  A0 = vfma(P, A0, vs<V>(0.5f));                                     // 1/2!
  V A2 = vfma(P, vs<V>(1.147074560e-10f), vs<V>(-1.252605419e-08f));   // 10/14!, -6/12!
  A2 = vfma(P, A2, vs<V>(8.267195767e-07f));                         // 3/10!
  A2 = vfma(P, A2, vs<V>(-2.480158730e-05f));                        // -1/8!
  V D1 = vfma(P, vs<V>(4.588298239e-12f), vs<V>(-8.029521918e-10f));   // 6/15!, -5/13!
  D1 = vfma(P, D1, vs<V>(1.002084335e-07f));                         // 4/11!
  D1 = vfma(P, D1, vs<V>(-8.267195767e-06f));                        // -3/9!
  D1 = vfma(P, D1, vs<V>(3.968253968e-04f));                         // 2/7!
  D1 = vfma(P, D1, vs<V>(-8.333333333e-03f));                        // -1/5!
  V D3 = vfma(P, vs<V>(7.647163732e-12f), vs<V>(-6.423617535e-10f));   // 10/15!, -4/13!
  D3 = vfma(P, D3, vs<V>(2.505210839e-08f));                         // 1/11!
  const V gre = vfma(T2, vfma(T2, vs<V>(1.147074560e-11f), A2), A0);   // 1/14!
  const V gim = vmul(T, vfma(T2, D3, D1));
  zr = vneg(gim);
  zi = gre;
}

// Extra-long form (P < 9, i.e. tau <= 6): h_k through k = 17.  With
// h_k = sum over 2i + 3j = k of C(i + j, i) P^i T^j,
//   G_re = A0(P) + T^2 (A2(P) + T^2 A4(P)),  G_im = T (D1(P) + T^2 (D3(P) + T^2 D5(P))),
// the coefficient of P^i in A_j / D_j being +-C(i + j, i)/(2i + 3j + 2)!;
// the omitted terms (k >= 18) are below 1e-9 (|G| <= 1/2).
template <class V>
__device__ __forceinline__ void face_series_xlong(V T, V P, V& zr, V& zi) {
  const V T2 = vmul(T, T);
  V A0 = vfma(P, vs<V>(1.561920697e-16f), vs<V>(-4.779477332e-14f));   // 1/18!, -1/16!
  A0 = vfma(P, A0, vs<V>(1.147074560e-11f));                         // 1/14!
  A0 = vfma(P, A0, vs<V>(-2.087675699e-09f));                        // -1/12!
  A0 = vfma(P, A0, vs<V>(2.755731922e-07f));                         // 1/10!
  A0 = vfma(P, A0, vs<V>(-2.480158730e-05f));                        // -1/8!
  A0 = vfma(P, A0, vs<V>(1.388888889e-03f));                         // 1/6!
  A0 = vfma(P, A0, vs<V>(-4.166666667e-02f));                        // -1/4!
  A0 = vfma(P, A0, vs<V>(0.5f));                                     // 1/2!
  V A2 = vfma(P, vs<V>(3.280033463e-15f), vs<V>(-7.169215999e-13f));   // 21/18!, -15/16!
  A2 = vfma(P, A2, vs<V>(1.147074560e-10f));                         // 10/14!
  A2 = vfma(P, A2, vs<V>(-1.252605419e-08f));                        // -6/12!
  A2 = vfma(P, A2, vs<V>(8.267195767e-07f));                         // 3/10!
  A2 = vfma(P, A2, vs<V>(-2.480158730e-05f));                        // -1/8!
  V A4 = vfma(P, vs<V>(2.342881045e-15f), vs<V>(-2.389738666e-13f));   // 15/18!, -5/16!
  A4 = vfma(P, A4, vs<V>(1.147074560e-11f));                         // 1/14!
  V D1 = vfma(P, vs<V>(6.576508197e-17f), vs<V>(-1.968020078e-14f));   // 8/19!, -7/17!
  D1 = vfma(P, D1, vs<V>(4.588298239e-12f));                         // 6/15!
  D1 = vfma(P, D1, vs<V>(-8.029521918e-10f));                        // -5/13!
  D1 = vfma(P, D1, vs<V>(1.002084335e-07f));                         // 4/11!
  D1 = vfma(P, D1, vs<V>(-8.267195767e-06f));                        // -3/9!
  D1 = vfma(P, D1, vs<V>(3.968253968e-04f));                         // 2/7!
  D1 = vfma(P, D1, vs<V>(-8.333333333e-03f));                        // -1/5!
  V D3 = vfma(P, vs<V>(2.877222336e-16f), vs<V>(-5.622914509e-14f));   // 35/19!, -20/17!
  D3 = vfma(P, D3, vs<V>(7.647163732e-12f));                         // 10/15!
  D3 = vfma(P, D3, vs<V>(-6.423617535e-10f));                        // -4/13!
  D3 = vfma(P, D3, vs<V>(2.505210839e-08f));                         // 1/11!
  const V D5 = vfma(P, vs<V>(4.932381148e-17f), vs<V>(-2.811457254e-15f));   // 6/19!, -1/17!
  const V gre = vfma(T2, vfma(T2, A4, A2), A0);
  const V gim = vmul(T, vfma(T2, vfma(T2, D5, D3), D1));
  zr = vneg(gim);
  zi = gre;
}

// Z from the edge sum of Eq. 14.  The first edge's sinc(u_0) comes in through S0 when kShared
// (the other face of a pair evaluated it: the same edge run the other way, and sinc is even) and
// goes out through it otherwise.  V = float2 carries two Q points through the same arithmetic.
__device__ __forceinline__ void sincos_v(float x, float& sn, float& cs) { __sincosf(x, &sn, &cs); }
__device__ __forceinline__ void sincos_v(float2 x, float2& sn, float2& cs) {
  __sincosf(x.x, &sn.x, &cs.x);
  __sincosf(x.y, &sn.y, &cs.y);
}
// 1/x2, and 0 for x2 = 0 (Q parallel to N: the series is taken there)
__device__ __forceinline__ float rcp_or0(float x2) { return x2 > 0.f ? rcp_approx(x2) : 0.f; }
__device__ __forceinline__ float2 rcp_or0(float2 x2) { return make_float2(rcp_or0(x2.x), rcp_or0(x2.y)); }

template <bool kShared, class V>
__device__ __forceinline__ void face_edge(V qx, V qy, V qz, const float4 A, const float4 B, const float4 C,
                                          V a0, V a1, V& zr, V& zi, V& S0) {
  const float nx = C.y, ny = C.z, nz = C.w;
  const V Xx = vfma(vs<V>(ny), qz, vmul(vs<V>(-nz), qy));
  const V Xy = vfma(vs<V>(nz), qx, vmul(vs<V>(-nx), qz));
  const V Xz = vfma(vs<V>(nx), qy, vmul(vs<V>(-ny), qx));
  const V x2 = vfma(Xx, Xx, vfma(Xy, Xy, vmul(Xz, Xz)));
  const V b0 = vfma(vs<V>(A.w), Xx, vfma(vs<V>(B.x), Xy, vmul(vs<V>(B.y), Xz)));
  const V b1 = vfma(vs<V>(B.z), Xx, vfma(vs<V>(B.w), Xy, vmul(vs<V>(C.x), Xz)));
  const V b2 = vneg(vadd(b0, b1));
  const V w[3] = {vadd(b1, vneg(b0)), vadd(b2, vneg(b1)), vadd(b0, vneg(b2))};
  const V h0 = vmul(vs<V>(0.5f), a0), h1 = vmul(vs<V>(0.5f), a1);
  const V u[3] = {vadd(h1, vneg(h0)), vfma(vs<V>(-2.0f), h1, vneg(h0)), vfma(vs<V>(2.0f), h0, h1)};   // (a_{l+1} - a_l)/2
  // exp(i psi_l), psi_l = -a_{l+2}/2: psi_1 = -h0 and psi_2 = -h1 on the SFU,
  // psi_0 = h0 + h1 as the conjugate of their product.
  V sp[3], cp[3];
  sincos_v(vneg(h0), sp[1], cp[1]);
  sincos_v(vneg(h1), sp[2], cp[2]);
  cp[0] = vfma(cp[1], cp[2], vneg(vmul(sp[1], sp[2])));
  sp[0] = vneg(vfma(sp[1], cp[2], vmul(cp[1], sp[2])));
  V u2[3], S[3];
#pragma unroll
  for (int l = kShared ? 1 : 0; l < 3; ++l) {
    u2[l] = vmul(u[l], u[l]);
    S[l] = sinc_poly_v(u2[l]);
  }
  // rare: an edge with |Q.d_l| > 2 pi somewhere in the warp (face_edge runs warp-converged)
  constexpr int kE = sizeof(V) / sizeof(float);
  bool big = false;
#pragma unroll
  for (int l = kShared ? 1 : 0; l < 3; ++l)
#pragma unroll
    for (int e = 0; e < kE; ++e) big = big || (el(&u2[l], e) > kPi2);
  if (__any_sync(0xffffffffu, big)) {
#pragma unroll
    for (int l = kShared ? 1 : 0; l < 3; ++l)
#pragma unroll
      for (int e = 0; e < kE; ++e)
        if (el(&u2[l], e) > kPi2) el(&S[l], e) = sinc_large(el(&u[l], e));
  }
  if (kShared) S[0] = S0;
  else S0 = S[0];
  V sr = vs<V>(0.f), si = vs<V>(0.f);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const V ws = vmul(w[l], S[l]);
    sr = vfma(ws, cp[l], sr);
    si = vfma(ws, sp[l], si);
  }
  const V inv = rcp_or0(x2);
  zr = vmul(sr, inv);
  zi = vmul(si, inv);
}

// |Q|^2 I_m = -s exp(i mu) Z, added into the tile sums (tre, tim).

template <class V>
__device__ __forceinline__ void face_finish(V mu, V s, V zr, V zi, V& tre, V& tim) {
  V sm, cm;
  sincos_v(mu, sm, cm);
  const V c = vmul(vneg(s), cm), d = vmul(vneg(s), sm);   // -s exp(i mu) = c + i d
  tre = vfma(c, zr, vfma(vneg(d), zi, tre));
  tim = vfma(c, zi, vfma(d, zr, tim));
}

// Same face term in FP64 (comparison path): library sincos, series through k = 16.
__device__ __forceinline__ void face_pair_f64(double qx, double qy, double qz, const Face64& f, double p_hi, double p_lo,
                                              double& re, double& im) {
  const double mu = fma(qx, f.gx, fma(qy, f.gy, qz * f.gz));
  const double a0 = fma(qx, f.q0x, fma(qy, f.q0y, qz * f.q0z));
  const double a1 = fma(qx, f.q1x, fma(qy, f.q1y, qz * f.q1z));
  const double s = fma(qx, f.nx, fma(qy, f.ny, qz * f.nz));
  const double a2 = -(a0 + a1);
  const double P = fma(a0, a0 + a1, a1 * a1);
  double zr, zi;
  const bool series = __all_sync(0xffffffffu, P < p_hi) || (P < p_lo);
  if (series) {
    const double T = a0 * a1 * a2;
    constexpr int K = 16;
    double h[K + 1];
    h[0] = 1.0; h[1] = 0.0; h[2] = P;
#pragma unroll
    for (int k = 3; k <= K; ++k) h[k] = fma(P, h[k - 2], T * h[k - 3]);
    double gre = 0.0, gim = 0.0, inv = 0.5;   // 1/(k+2)!
#pragma unroll
    for (int k = 0; k <= K; ++k) {
      const double t = h[k] * inv;
      switch (k & 3) { case 0: gre += t; break; case 1: gim += t; break; case 2: gre -= t; break; default: gim -= t; }
      inv /= (double)(k + 3);
    }
    zr = -gim;
    zi = gre;
  } else {
    const double Xx = fma(f.ny, qz, -f.nz * qy), Xy = fma(f.nz, qx, -f.nx * qz), Xz = fma(f.nx, qy, -f.ny * qx);
    const double x2 = fma(Xx, Xx, fma(Xy, Xy, Xz * Xz));
    const double b0 = fma(f.q0x, Xx, fma(f.q0y, Xy, f.q0z * Xz));
    const double b1 = fma(f.q1x, Xx, fma(f.q1y, Xy, f.q1z * Xz));
    const double b2 = -(b0 + b1);
    const double w[3] = {b1 - b0, b2 - b1, b0 - b2};
    const double psi[3] = {-0.5 * a2, -0.5 * a0, -0.5 * a1};
    const double u[3] = {0.5 * (a1 - a0), 0.5 * (a2 - a1), 0.5 * (a0 - a2)};
    double sr = 0.0, si = 0.0;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      double sp, cp;
      sincos(psi[l], &sp, &cp);
      const double ws = w[l] * sinc_f64(u[l]);
      sr = fma(ws, cp, sr);
      si = fma(ws, sp, si);
    }
    const double inv = (x2 > 0.0) ? 1.0 / x2 : 0.0;
    zr = sr * inv;
    zi = si * inv;
  }
  double sm, cm;
  sincos(mu, &sm, &cm);
  re = -s * fma(cm, zr, -sm * zi);
  im = -s * fma(cm, zi, sm * zr);
}

// ---------------------------------------------------------------------------
// Policies: record type, Q registers, accumulators and the per-tile loop.
// ---------------------------------------------------------------------------

template <int R>
struct Acc32 {
  CAcc re[R], im[R];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int r = 0; r < R; ++r) { re[r].init(); im[r].init(); }
  }
  __device__ __forceinline__ double2 get(int r) const {
    return make_double2((double)re[r].hi + (double)re[r].lo, (double)im[r].hi + (double)im[r].lo);
  }
};

template <int R>
struct Acc64 {
  double re[R], im[R];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int r = 0; r < R; ++r) { re[r] = 0.0; im[r] = 0.0; }
  }
  __device__ __forceinline__ double2 get(int r) const { return make_double2(re[r], im[r]); }
};

// Per-Q values of a thread: R floats, or R/2 float2 pairs when R is even, so that the per-pair
// arithmetic runs as paired FP32 instructions (two Q points per issue slot).
template <int R>
struct QPack {
  static constexpr bool kPacked = (R % 2) == 0;
  static constexpr int N = kPacked ? R / 2 : R;
  using V = typename std::conditional<kPacked, float2, float>::type;
  template <int D>
  __device__ static __forceinline__ void pack(const float (&q)[R][3], V (&qv)[N][3]) {
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if constexpr (kPacked) qv[j][d] = make_float2(q[2 * j][d], q[2 * j + 1][d]);
        else qv[j][d] = q[j][d];
      }
  }
};

struct Pol2F32 {
  using Item = Seg32;
  static constexpr int kDim = 2, kTile = 128;
  static constexpr bool kPaired = false;
  template <int R> using Acc = Acc32<R>;
  using QT = float;
  template <int R>
  __device__ static __forceinline__ void tile(const Item* t, int cnt, const QT (&q)[R][3], Acc<R>& acc, Thr,
                                              int64_t) {
    using V = typename QPack<R>::V;
    constexpr int N = QPack<R>::N;
    V qv[N][3], tre[N], tim[N];
    QPack<R>::template pack<2>(q, qv);
#pragma unroll
    for (int j = 0; j < N; ++j) { tre[j] = vs<V>(0.f); tim[j] = vs<V>(0.f); }
#pragma unroll 1
    for (int i = 0; i < cnt; ++i) {
      const float4 s = reinterpret_cast<const float4*>(t)[i];   // m.x, m.y, D.x/2, D.y/2
      V ph[N], u[N], u2[N], w[N], S[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const V qx = qv[j][0], qy = qv[j][1];
        ph[j] = vfma(qx, vs<V>(s.x), vmul(qy, vs<V>(s.y)));          // Q.m
        u[j] = vfma(qx, vs<V>(s.z), vmul(qy, vs<V>(s.w)));           // Q.D / 2
        w[j] = vfma(qx, vs<V>(s.w), vmul(vneg(qy), vs<V>(s.z)));     // (Qx Dy - Qy Dx) / 2
        u2[j] = vmul(u[j], u[j]);
        S[j] = sinc_poly_v(u2[j]);
      }
      bool big = false;
#pragma unroll
      for (int r = 0; r < R; ++r) big = big || (el(u2, r) > kPi2);
      // segments long against 1/|Q|: the SFU sinc, only in warps where some lane needs it
      if (__any_sync(0xffffffffu, big)) {
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (el(u2, r) > kPi2) el(S, r) = sinc_large(el(u, r));
      }
#pragma unroll
      for (int j = 0; j < N; ++j) {
        V sn, cs;
        sincos_v(ph[j], sn, cs);
        const V ws = vmul(w[j], S[j]);
        tre[j] = vfma(ws, sn, tre[j]);     // -i ws (cos + i sin) = ws sin - i ws cos
        tim[j] = vfma(vneg(ws), cs, tim[j]);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) { acc.re[r].add(el(tre, r)); acc.im[r].add(el(tim, r)); }
  }
};

struct Pol2F64 {
  using Item = Seg64;
  static constexpr int kDim = 2, kTile = 64;
  static constexpr bool kPaired = false;
  template <int R> using Acc = Acc64<R>;
  using QT = double;
  template <int R>
  __device__ static __forceinline__ void tile(const Item* t, int cnt, const QT (&q)[R][3], Acc<R>& acc, Thr,
                                              int64_t) {
    for (int i = 0; i < cnt; ++i) {
      const Seg64 s = t[i];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        double re, im;
        seg_pair_f64(q[r][0], q[r][1], s, re, im);
        acc.re[r] += re;
        acc.im[r] += im;
      }
    }
  }
};

// One face of the 3D FP32 policy for a thread's R Q points: the projections, their branch
// quantities and the warp's largest P (the branch tests need only it and the thread's smallest P).
template <int R>
struct FaceQ {
  using V = typename QPack<R>::V;
  static constexpr int N = QPack<R>::N;
  V mu[N], a0[N], a1[N], s[N], P[N], T[N];
  float pmin, wmax;
  __device__ __forceinline__ void load(const V (&qv)[N][3], const float4 A, const float4 B, const float4 C) {
#pragma unroll
    for (int j = 0; j < N; ++j)
      face_common_pt(qv[j][0], qv[j][1], qv[j][2], A, B, C, mu[j], a0[j], a1[j], s[j], P[j], T[j]);
    float pmax = el(P, 0);
    pmin = el(P, 0);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      pmax = fmaxf(pmax, el(P, r));
      pmin = fminf(pmin, el(P, r));
    }
    // P >= +0 (it is s1^2 - a0 a1 = a0^2 + a0 a1 + a1^2) or NaN, so its bits order as unsigned
    // integers, and one reduction replaces a vote per rung of the ladder
    wmax = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(pmax)));
  }
  // the shortest series whose bound holds for the whole warp (wmax and th.hi are uniform)
  __device__ __forceinline__ void series(const Thr& th, V (&zr)[N], V (&zi)[N]) const {
    if (th.hi <= kPShort || wmax < kPShort) {
#pragma unroll
      for (int j = 0; j < N; ++j) face_series(T[j], P[j], zr[j], zi[j]);
    } else if (th.hi <= kP9 || wmax < kP9) {
#pragma unroll
      for (int j = 0; j < N; ++j) face_series_k9(T[j], P[j], zr[j], zi[j]);
    } else if (th.hi <= kPLong || wmax < kPLong) {
#pragma unroll
      for (int j = 0; j < N; ++j) face_series_long(T[j], P[j], zr[j], zi[j]);
    } else if (th.hi <= kP13 || wmax < kP13) {
#pragma unroll
      for (int j = 0; j < N; ++j) face_series_k13(T[j], P[j], zr[j], zi[j]);
    } else {
#pragma unroll
      for (int j = 0; j < N; ++j) face_series_xlong(T[j], P[j], zr[j], zi[j]);
    }
  }
  // the edge sum (per Q point), with the few Q points below tau_lo^2/4 redone by the short series
  template <bool kShared>
  __device__ __forceinline__ void edge(const Thr& th, const V (&qv)[N][3], const float4 A, const float4 B,
                                       const float4 C, V (&zr)[N], V (&zi)[N], V (&S0)[N]) const {
#pragma unroll
    for (int j = 0; j < N; ++j)
      face_edge<kShared>(qv[j][0], qv[j][1], qv[j][2], A, B, C, a0[j], a1[j], zr[j], zi[j], S0[j]);
    if (pmin < th.lo) {
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (el(P, r) < th.lo) face_series(el(T, r), el(P, r), el(zr, r), el(zi, r));   // P < tau_lo^2/4 <= 1/4
    }
  }
  __device__ __forceinline__ void finish(const V (&zr)[N], const V (&zi)[N], V (&tre)[N], V (&tim)[N]) const {
#pragma unroll
    for (int j = 0; j < N; ++j) face_finish(mu[j], s[j], zr[j], zi[j], tre[j], tim[j]);
  }
};

// kPairs: faces [0, th.pair_end) come in pairs that share their first edge (face_pairs option): when
// both faces of a pair take the edge sum in a warp, the second takes the shared edge's sinc from the
// first (carried in registers from one face to the next).  A separate instantiation, so that the
// single-face kernel is unchanged.
template <bool kPairs>
struct Pol3F32T {
  using Item = Face32;
  // 128 faces (6 KB) per tile: on the 1.31M-face mesh x 128^3 Q, 3262 against 3283 ms at 64
  static constexpr int kDim = 3, kTile = 128;
  static constexpr bool kPaired = kPairs;
  template <int R> using Acc = Acc32<R>;
  using QT = float;
  // `first`: index of the tile's first face among all faces (pairs start at even indices, and tiles
  // start at multiples of kTile, so a pair never straddles two tiles).
  template <int R>
  __device__ static __forceinline__ void tile(const Item* t, int cnt, const QT (&q)[R][3], Acc<R>& acc,
                                              Thr th, int64_t first) {
    using V = typename QPack<R>::V;
    constexpr int N = QPack<R>::N;
    V qv[N][3], tre[N], tim[N];
    QPack<R>::template pack<3>(q, qv);
#pragma unroll
    for (int j = 0; j < N; ++j) { tre[j] = vs<V>(0.f); tim[j] = vs<V>(0.f); }
    // S0 carries the first edge's sinc from the first face of a pair to the second; `held` says
    // that it does (warp-uniform: it follows the warp-uniform branch decisions)
    V S0[N];
    bool held = false;
#pragma unroll 1
    for (int i = 0; i < cnt; ++i) {
      const float4* p = reinterpret_cast<const float4*>(t + i);
      const float4 A = p[0], B = p[1], C = p[2];
      FaceQ<R> f;
      f.load(qv, A, B, C);
      V zr[N], zi[N];
      if (f.wmax < th.hi) {
        f.series(th, zr, zi);
        held = false;
      } else if (kPairs && held && first + i < th.pair_end) {
        // the second face of a pair whose first face took the edge sum in this warp: the shared
        // edge's sinc comes from it
        f.template edge<true>(th, qv, A, B, C, zr, zi, S0);
        held = false;
      } else {
        f.template edge<false>(th, qv, A, B, C, zr, zi, S0);
        held = kPairs && ((first + i) & 1) == 0 && first + i < th.pair_end;   // the first face of a pair
      }
      f.finish(zr, zi, tre, tim);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) { acc.re[r].add(el(tre, r)); acc.im[r].add(el(tim, r)); }
  }
};
using Pol3F32 = Pol3F32T<false>;
using Pol3F32Pair = Pol3F32T<true>;

struct Pol3F64 {
  using Item = Face64;
  static constexpr int kDim = 3, kTile = 32;
  static constexpr bool kPaired = false;
  template <int R> using Acc = Acc64<R>;
  using QT = double;
  template <int R>
  __device__ static __forceinline__ void tile(const Item* t, int cnt, const QT (&q)[R][3], Acc<R>& acc,
                                              Thr th, int64_t) {
    for (int i = 0; i < cnt; ++i) {
      const Face64 f = t[i];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        double re, im;
        face_pair_f64(q[r][0], q[r][1], q[r][2], f, (double)th.hi, (double)th.lo, re, im);
        acc.re[r] += re;
        acc.im[r] += im;
      }
    }
  }
};

}  // namespace pft
