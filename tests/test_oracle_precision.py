"""Rounding accuracy of the FP64 oracle, pinned by 40-digit arithmetic on tiny cases.

The oracle's segment sum (Eq. 6) and face sum (sign-corrected Eq. 14), with their
series branches, are checked here against a form that shares none of their
arithmetic: the region cut into signed simplices from an interior point, each
simplex integral written as a divided difference of e^{ix} at the projected
corners (Hermite-Genocchi: the integral of g(t0 x0 + ... + tn xn) over the unit
n-simplex is G[x0..xn] with G^(n) = g).  A triangle of signed area A gives
-2A E[a, b, c] and a tetrahedron of signed volume V gives 6V i E[a, b, c, d], with
E the divided difference of e^{ix}.  Evaluated with mpmath at 40 significant
digits, the cancellation of the divided differences costs nothing, so the
difference measures the oracle's own FP64 rounding (and its series truncation).
"""
import numpy as np
import pytest

import oracle
from paper_2104_08309_gb300 import synth

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp


def _dd_exp(x):
    """Divided difference E[x0..xn] of e^{ix} by the recursive definition (distinct nodes)."""
    vals = [mpmath.expj(t) for t in x]
    n = len(x)
    for level in range(1, n):
        vals = [(vals[k + 1] - vals[k]) / (x[k + level] - x[k]) for k in range(n - level)]
    return vals[0]


def _ft2d_simplices(v, q, o):
    """Sum over the triangles (o, p_j, p_j+1) of -2 A_j E[Q.o, Q.p_j, Q.p_j+1]."""
    P = [(mp.mpf(float(a)), mp.mpf(float(b))) for a, b in v]
    ox, oy = (mp.mpf(float(t)) for t in o)
    out = []
    for qx, qy in q:
        Qx, Qy = mp.mpf(float(qx)), mp.mpf(float(qy))
        s = mp.mpc(0)
        for j in range(len(P)):
            (x0, y0), (x1, y1) = P[j], P[(j + 1) % len(P)]
            A = ((x0 - ox) * (y1 - oy) - (x1 - ox) * (y0 - oy)) / 2
            s += -2 * A * _dd_exp([Qx * ox + Qy * oy, Qx * x0 + Qy * y0, Qx * x1 + Qy * y1])
        out.append(complex(s))
    return np.array(out)


def _ft3d_simplices(v, f, q, o):
    """Sum over the tetrahedra (o, p0, p1, p2) of 6 V i E[Q.o, Q.p0, Q.p1, Q.p2]."""
    P = [tuple(mp.mpf(float(t)) for t in p) for p in v]
    O = tuple(mp.mpf(float(t)) for t in o)
    out = []
    for qv in q:
        Q = tuple(mp.mpf(float(t)) for t in qv)
        dot = lambda p: Q[0] * p[0] + Q[1] * p[1] + Q[2] * p[2]
        s = mp.mpc(0)
        for a, b, c in f:
            A, B, C = ([P[k][d] - O[d] for d in range(3)] for k in (a, b, c))
            V6 = (A[0] * (B[1] * C[2] - B[2] * C[1]) - A[1] * (B[0] * C[2] - B[2] * C[0])
                  + A[2] * (B[0] * C[1] - B[1] * C[0]))
            s += V6 * 1j * _dd_exp([dot(O), dot(P[a]), dot(P[b]), dot(P[c])])
        out.append(complex(s))
    return np.array(out)


@pytest.fixture(autouse=True)
def _digits():
    with mp.workdps(40):
        yield


def test_2d_star_polygon_rounding(rng):
    """C1-style star polygon (64 vertices): generic, large and small |Q| (series branches)."""
    v = synth.star_polygon(64, seed=1).astype(np.float64)
    q = np.concatenate([rng.uniform(-40, 40, (10, 2)), [[39.375, -38.75], [0.3, -0.2]],
                        rng.uniform(-1e-3, 1e-3, (3, 2)), [[2.5e-4, 0.0], [0.0, -7.5e-6]]])
    o = (0.01234, -0.00567)   # interior, on no vertex
    ref = _ft2d_simplices(v, q, o)
    F = oracle.ft2d(v, q)
    area = abs(oracle.ft2d(v, np.zeros((1, 2)))[0])
    err = np.max(np.abs(F - ref)) / area
    assert err < 1e-14, err


def test_3d_icosphere_rounding(rng):
    """Level-1 icosphere (80 faces): generic Q, |Q| near the face-series threshold and small |Q|."""
    v, f = synth.icosphere(1)
    v = v.astype(np.float64)
    d = rng.normal(size=(4, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    q = np.concatenate([rng.uniform(-30, 30, (5, 3)), d * 0.0095, d[:2] * 2e-4, [[0.5, -0.25, 0.125]]])
    o = (0.0123, -0.0211, 0.0307)
    ref = _ft3d_simplices(v, f, q, o)
    F = oracle.ft3d(v, f, q)
    vol = abs(oracle.ft3d(v, f, np.zeros((1, 3)))[0])
    err = np.max(np.abs(F - ref)) / vol
    assert err < 1e-14, err


def test_simplex_form_against_direct_integral():
    """The divided-difference form on its own: the unit right triangle at Q = (a, b) against the
    definition integrated directly, int_0^1 e^{iax} int_0^{1-x} e^{iby} dy dx with the inner
    integral (e^{ib(1-x)} - 1)/(ib)."""
    a, b = mp.mpf("1.7"), mp.mpf("0.4")
    got = _ft2d_simplices(np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), np.array([[1.7, 0.4]]), (0.2, 0.3))[0]
    ref = complex(mpmath.quad(lambda x: mpmath.expj(a * x) * (mpmath.expj(b * (1 - x)) - 1) / (1j * b), [0, 1]))
    assert abs(got - ref) < 1e-15
