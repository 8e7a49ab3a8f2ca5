"""Host-side checks of the constants the FP32 kernels hard-code (no GPU needed).

The coefficients are read out of the CUDA header/source text and evaluated
here in float32 the way the kernels evaluate them (Horner with FMA-free
float32 steps, which bounds the FMA form from above).
"""
import math
import os
import re
from fractions import Fraction

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2104_08309_gb300", "csrc")


def _body(path, name):
    text = open(os.path.join(CSRC, path)).read()
    i = text.index(name)
    return text[i:text.index("\n}\n", i)]


def _floats(body):
    return [float(x) for x in re.findall(r"[-+]?\d\.\d+e[-+]\d+", body)]


def test_sinc_polynomial_accuracy():
    """sinc(u) on |u| <= pi from the degree-6 polynomial in u^2."""
    c = _floats(_body("pft_common.cuh", "V sinc_poly_v("))
    assert len(c) == 6
    # Horner order in the source: c6, c5, then c4..c1, constant 1
    coef = np.array([1.0] + c[::-1], dtype=np.float32)     # c0..c6
    u = np.linspace(0.0, math.pi, 200001)
    v = (u * u).astype(np.float32)
    acc = np.full_like(v, coef[-1])
    for ck in coef[-2::-1]:
        acc = (acc * v + ck).astype(np.float32)
    ref = np.sinc(u / math.pi)
    assert np.max(np.abs(acc - ref)) < 3e-7


def test_face_series_coefficients_are_inverse_factorials():
    """G = sum_k i^k h_k/(k+2)!: the constants are +-1/(k+2)! and their combinations."""
    c = _floats(_body("pft_pairs.cuh", "void face_series("))
    f = math.factorial
    expected = [-1 / f(8), 1 / f(6), -1 / f(4),                      # Horner in P for the real part (+ 1/2)
                -1 / f(8),                                             # T^2 term of h6
                -1 / 120960, 1 / 2520, -1 / f(5)]                      # imaginary part: -T/5! + PT/2520 - P^2T/120960
    assert len(c) == len(expected)
    for got, want in zip(c, expected):
        assert abs(got - want) <= 1e-6 * abs(want)
    # 2520 = 7!/2 (coefficient 2/7! of P T) and 120960 = 9!/3 (coefficient 3/9! of P^2 T)
    assert f(7) // 2 == 2520 and f(9) // 3 == 120960


def test_long_face_series_coefficients():
    """Long form: A(P) = sum (-1)^j P^j/(2j+2)!, B, D, E from h_8..h_11 (see the kernel comment)."""
    c = _floats(_body("pft_pairs.cuh", "void face_series_long("))
    f = math.factorial
    expected = [-1 / f(12), 1 / f(10), -1 / f(8), 1 / f(6), -1 / f(4),    # A
                -6 / f(12), 3 / f(10), -1 / f(8),                          # B (T^2 terms of h6, h8, h10)
                -5 / f(13), 4 / f(11), -3 / f(9), 2 / f(7), -1 / f(5),     # D
                -4 / f(13), 1 / f(11)]                                     # E
    assert len(c) == len(expected)
    for got, want in zip(c, expected):
        assert abs(got - want) <= 1e-6 * abs(want)


def _exact_G(a0, a1, K=40):
    """G = sum_k i^k h_k/(k+2)! with h_k = P h_{k-2} + T h_{k-3}, summed far past convergence."""
    P = a0 * a0 + a0 * a1 + a1 * a1
    T = -(a0 * a1) * (a0 + a1)
    h = [np.ones_like(P), np.zeros_like(P), P]
    for k in range(3, K + 1):
        h.append(P * h[k - 2] + T * h[k - 3])
    g = np.zeros_like(P, dtype=complex)
    for k in range(K + 1):
        g += (1j ** k) * h[k] / math.factorial(k + 2)
    return P, T, g


def _horner(coef, x):
    acc = np.zeros_like(x)
    for c in coef:
        acc = acc * x + c
    return acc


def _phases(pmax, n=200000, seed=3):
    # a0 = x - y/sqrt3, a1 = 2y/sqrt3 maps the disc x^2 + y^2 < pmax onto P < pmax
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * np.pi, n)
    rad = np.sqrt(pmax) * np.sqrt(rng.uniform(0, 1, n))
    x, y = rad * np.cos(ang), rad * np.sin(ang)
    return x - y / np.sqrt(3), 2 * y / np.sqrt(3)


def test_face_series_truncation_bounds():
    """The kernel's short form (k <= 7) on P < 1/4 and long form (k <= 11) on P < 9/4, with
    the constants read from the source, against the converged series: within 2e-9 and 4e-9."""
    cs = _floats(_body("pft_pairs.cuh", "void face_series("))
    P, T, g = _exact_G(*_phases(0.25))
    gre = _horner(cs[0:3] + [0.5], P) + T * T * cs[3]
    gim = T * _horner(cs[4:7], P)
    assert np.max(np.abs(gre + 1j * gim - g)) < 2e-9
    cl = _floats(_body("pft_pairs.cuh", "void face_series_long("))
    P, T, g = _exact_G(*_phases(2.25))
    A = _horner(cl[0:5] + [0.5], P)
    B = _horner(cl[5:8], P)
    D = _horner(cl[8:13], P)
    E = _horner(cl[13:15], P)
    gre = A + T * T * B
    gim = T * (D + T * T * E)
    assert np.max(np.abs(gre + 1j * gim - g)) < 4e-9
    # the converged series itself is the second divided difference of e^z at the points i a_k,
    # G = sum_k e^{i a_k} / prod_{j != k} (i a_k - i a_j): checked where the corners are well separated
    a0, a1 = _phases(2.25, n=2000, seed=4)
    a2 = -(a0 + a1)
    ok = np.minimum.reduce([abs(a0 - a1), abs(a1 - a2), abs(a2 - a0)]) > 0.3
    a0, a1, a2 = a0[ok], a1[ok], a2[ok]
    dd = sum(np.exp(1j * x) / ((1j * x - 1j * y) * (1j * x - 1j * z)) for x, y, z in
             ((a0, a1, a2), (a1, a2, a0), (a2, a0, a1)))
    _, _, g = _exact_G(a0, a1)
    assert np.max(np.abs(g - dd)) < 1e-12


def _xlong_expected():
    """Coefficients of face_series_xlong in source order: A0, A2, A4, D1, D3, D5, each from its
    highest power of P down (A0's constant 1/2 is written as 0.5f and not listed)."""
    from math import comb
    f = math.factorial

    def c(i, j):
        k = 2 * i + 3 * j
        sign = (1 if k % 4 == 0 else -1) if k % 2 == 0 else (1 if k % 4 == 1 else -1)
        return sign * comb(i + j, i) / f(k + 2)

    out = []
    for j, imax in ((0, 8), (2, 5), (4, 2), (1, 7), (3, 4), (5, 1)):
        out += [c(i, j) for i in range(imax, -1, -1) if not (j == 0 and i == 0)]
    return out


def test_xlong_face_series_coefficients():
    """Extra-long form: the coefficient of P^i T^j is +-C(i + j, i)/(2i + 3j + 2)! (h_k through k = 17)."""
    c = _floats(_body("pft_pairs.cuh", "void face_series_xlong("))
    expected = _xlong_expected()
    assert len(c) == len(expected)
    for got, want in zip(c, expected):
        assert abs(got - want) <= 1e-6 * abs(want)


def test_xlong_face_series_truncation_bound():
    """The extra-long form with the source's constants, on P < 9, against the converged series."""
    c = _floats(_body("pft_pairs.cuh", "void face_series_xlong("))
    P, T, g = _exact_G(*_phases(9.0))
    A0 = _horner(c[0:8] + [0.5], P)
    A2 = _horner(c[8:14], P)
    A4 = _horner(c[14:17], P)
    D1 = _horner(c[17:25], P)
    D3 = _horner(c[25:30], P)
    D5 = _horner(c[30:32], P)
    T2 = T * T
    gre = A0 + T2 * (A2 + T2 * A4)
    gim = T * (D1 + T2 * (D3 + T2 * D5))
    assert np.max(np.abs(gre + 1j * gim - g)) < 1e-9
    # and in float32 (the kernel's precision) within a few units of rounding of |G| <= 1/2
    f32 = np.float32
    P32, T32 = P.astype(f32), T.astype(f32)
    T232 = (T32 * T32).astype(f32)
    h = lambda cs: _horner32([f32(x) for x in cs], P32)
    g32 = (h(c[0:8] + [0.5]) + T232 * (h(c[8:14]) + T232 * h(c[14:17]))) + 1j * (
        T32 * (h(c[17:25]) + T232 * (h(c[25:30]) + T232 * h(c[30:32]))))
    assert np.max(np.abs(g32 - g)) < 2e-7


def _horner32(coef, x):
    acc = np.zeros_like(x)
    for c in coef:
        acc = (acc * x + c).astype(np.float32)
    return acc


# Intermediate forms: (j, highest i .. lowest i) of each polynomial, in the order the constants
# appear in the source (the 1/2 of A0 is written as 0.5f and not listed).
_MID_LAYOUT = {
    "void face_series_k9(": (9, 1.0, [(0, 4, 1), (2, 1, 0), (1, 3, 0), (3, 0, 0)]),
    "void face_series_k13(": (13, 4.0, [(0, 6, 1), (2, 3, 0), (1, 5, 0), (3, 2, 0), (4, 0, 0)]),
}


def _coef(i, j):
    from math import comb
    k = 2 * i + 3 * j
    sign = (1 if k % 4 == 0 else -1) if k % 2 == 0 else (1 if k % 4 == 1 else -1)
    return sign * comb(i + j, i) / math.factorial(k + 2)


def _mid_coefficients(name):
    K, bound, layout = _MID_LAYOUT[name]
    c = _floats(_body("pft_pairs.cuh", name))
    keys = [(i, j) for j, hi, lo in layout for i in range(hi, lo - 1, -1)]
    assert len(c) == len(keys), name
    got = dict(zip(keys, c))
    got[(0, 0)] = 0.5
    return K, bound, got


def test_intermediate_face_series_coefficients():
    """k <= 9 and k <= 13 forms: the coefficient of P^i T^j is +-C(i + j, i)/(2i + 3j + 2)!, every term
    with 2i + 3j <= K present exactly once."""
    for name in _MID_LAYOUT:
        K, _, got = _mid_coefficients(name)
        assert set(got) == {(i, j) for j in range(K // 3 + 1) for i in range((K - 3 * j) // 2 + 1)}, name
        for (i, j), v in got.items():
            assert abs(v - _coef(i, j)) <= 1e-6 * abs(_coef(i, j)), (name, i, j)


def test_intermediate_face_series_truncation_bounds():
    """With the source's constants, on P below each form's bound, against the converged series:
    within 4e-9 in FP64 and within a few float32 roundings of |G| <= 1/2 in float32."""
    for name in _MID_LAYOUT:
        K, bound, got = _mid_coefficients(name)
        P, T, g = _exact_G(*_phases(bound))
        gre = sum(v * P ** i * T ** j for (i, j), v in got.items() if j % 2 == 0)
        gim = sum(v * P ** i * T ** j for (i, j), v in got.items() if j % 2 == 1)
        assert np.max(np.abs(gre + 1j * gim - g)) < 4e-9, name
        f32 = np.float32
        P32, T32 = P.astype(f32), T.astype(f32)
        T232 = (T32 * T32).astype(f32)
        polys = {}
        for j in sorted({j for _, j in got}):
            polys[j] = _horner32([f32(got[(i, j)]) for i in range(max(i for i, jj in got if jj == j), -1, -1)], P32)
        re = np.zeros_like(P32)
        for j in sorted((j for j in polys if j % 2 == 0), reverse=True):
            re = (re * T232 + polys[j]).astype(f32)
        im = np.zeros_like(P32)
        for j in sorted((j for j in polys if j % 2 == 1), reverse=True):
            im = (im * T232 + polys[j]).astype(f32)
        assert np.max(np.abs(re + 1j * (T32 * im) - g)) < 2e-7, name


def test_p_bits_order_as_unsigned():
    """The 3D branch ladders take the warp's largest P as the unsigned maximum of float32 bits.
    Forward: P = fmaf(s1, s1, -p1) with s1 = a0 + a1, p1 = a0 a1 is never negative nor -0, so its
    bits are used as they are.  Adjoint: P = fmaf(a0, a0 + a1, a1 a1) can be -0 or a negative
    subnormal (a1 a1 underflows before the fused add), so the kernel clears the sign bit; those
    values are far below every threshold, so ordering by |P| takes the same branch.  Emulated in
    float32 (the product inside the FMA is exact in float64; the sum is rounded to float64 and then
    to float32, which can move the value but not its sign), with signed zeros, subnormals and huge
    values."""
    rng = np.random.default_rng(11)
    f32 = np.float32
    vals = np.concatenate([rng.normal(size=200000) * 10.0 ** rng.uniform(-40, 18, 200000),
                           [0.0, -0.0, 1e-45, -1e-45, 1e-38, -1e-38, 3e38, -3e38]]).astype(f32)
    a0 = rng.choice(vals, 400000)
    a1 = np.where(rng.uniform(size=400000) < 0.2, -a0 / f32(2), rng.choice(vals, 400000)).astype(f32)
    with np.errstate(over="ignore", invalid="ignore"):
        s1 = (a0 + a1).astype(f32)
        p1 = (a0 * a1).astype(f32)
        P_fwd = (s1.astype(np.float64) * s1.astype(np.float64) - p1.astype(np.float64)).astype(f32)
        P_adj = (a0.astype(np.float64) * (a0 + a1).astype(f32).astype(np.float64)
                 + (a1 * a1).astype(f32).astype(np.float64)).astype(f32)
    fin = np.isfinite(P_fwd)
    assert np.all(P_fwd[fin] >= 0) and not np.any(np.signbit(P_fwd[fin]))
    neg = np.isfinite(P_adj) & np.signbit(P_adj)
    assert np.any(neg)                                   # the case the kernel guards against occurs
    assert np.all(np.abs(P_adj[neg]) < 1e-37)            # and only far below kPShort = 1/4
    # unsigned order of the bits of non-negative floats (and +inf, NaN above them) follows the values
    x = np.sort(np.abs(vals[np.isfinite(vals)]))
    bits = x.view(np.uint32)
    assert np.all(np.diff(bits.astype(np.int64)) >= 0)
    assert np.uint32(0x7F800000) > bits.max() and np.float32(np.nan).view(np.uint32) > np.uint32(0x7F800000)


def _fmaf(a, b, c):
    """fmaf for float32 inputs: the product is exact in float64; the sum is rounded to float64 and then
    to float32, which differs from the fused single rounding only in rare ties (immaterial to the
    bound below; the one exactness claim is checked with rationals)."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _two_sum(a, b):
    s = np.float32(a + b)
    bb = np.float32(s - a)
    return s, np.float32(np.float32(a - np.float32(s - bb)) + np.float32(b - bb))


def test_fp32_finish_phase_reduction():
    """The batched FP32 finish reduces the translation phase Q.c without FP64 arithmetic: Q.c as
    s + t (products with the centre's float high part split exactly by FMA, the low parts of Q and
    c in t), k = rint(s / 2 pi), ph = fma(-k, 2pi_hi, s) + fma(-k, 2pi_lo, t).  The constants are
    the float32 rounding of 2 pi and its residual; s - k 2pi_hi is exact in float32; and the phase
    matches Q.c mod 2 pi (50-digit reference) within 3e-7 rad for |Q.c| below 2^20."""
    mpmath = __import__("pytest").importorskip("mpmath")
    text = open(os.path.join(CSRC, "pft_batched.cu")).read()
    hi = np.float32(float(re.search(r"kTwoPiHi = ([-+0-9.e]+)f", text).group(1)))
    lo = np.float32(float(re.search(r"kTwoPiLo = ([-+0-9.e]+)f", text).group(1)))
    inv = np.float32(float(re.search(r"kInvTwoPi = ([-+0-9.e]+)f", open(os.path.join(CSRC, "pft_common.cuh")).read()).group(1)))
    assert hi == np.float32(2 * math.pi) and lo == np.float32(2 * math.pi - float(hi))
    mpmath.mp.dps = 50
    two_pi = 2 * mpmath.pi
    rng = np.random.default_rng(7)
    worst, n_checked = 0.0, 0
    for _ in range(400):
        q = rng.uniform(-60, 60, 3)                                     # the caller's FP64 Q
        c = rng.uniform(-1e4, 1e4, 3) * rng.choice([1e-4, 1e-2, 1.0])   # the FP64 centre
        qh = q.astype(np.float32)
        ql = (q - qh.astype(np.float64)).astype(np.float32)
        ch = c.astype(np.float32)
        cl = (c - ch.astype(np.float64)).astype(np.float32)
        s = np.float32(qh[0] * ch[0])
        t = _fmaf(qh[0], ch[0], -s)
        for d in (1, 2):
            p = np.float32(qh[d] * ch[d])
            e = _fmaf(qh[d], ch[d], -p)
            s, e2 = _two_sum(s, p)
            t = np.float32(t + np.float32(e2 + e))
        for d in range(3):
            t = _fmaf(ql[d], ch[d], _fmaf(qh[d], cl[d], t))
        if not abs(s) < 2.0 ** 20:       # the kernel takes its FP64 finish there
            continue
        n_checked += 1
        k = np.float32(np.rint(np.float32(s * inv)))
        exact = Fraction(float(s)) - Fraction(float(k)) * Fraction(float(hi))
        r = np.float32(float(exact))
        assert Fraction(float(r)) == exact                                       # s - k 2pi_hi fits a float32
        ph = np.float32(r + _fmaf(-k, lo, t))
        ref = mpmath.fsum(mpmath.mpf(float(qd)) * mpmath.mpf(float(cd)) for qd, cd in zip(q, c))
        ref = ref - two_pi * mpmath.nint(ref / two_pi)
        err = abs(float(ph) - float(ref))
        worst = max(worst, min(err, abs(err - 2 * math.pi)))
    assert n_checked > 300 and worst < 3e-7, (n_checked, worst)
