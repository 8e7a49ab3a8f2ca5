"""The oracle's 2D Q-gradient (Richardson-extrapolated differences of ft2d) against what fixes it
independently: the derivative of the rectangle closed form (Sec. 4.1), the first-moment integral
dF/dQ = i * integral of r e^{iQ.r} by brute-force quadrature, the translation identity
dF_{P+t}/dQ = e^{iQ.t} (i t F_P + dF_P/dQ), Hermitian symmetry, and its value at Q = 0 (i times
the area's first moment)."""
import numpy as np

import oracle
from paper_2104_08309_gb300 import synth
from tests import quadrature as quad


def _seg(q, L):
    x = 0.5 * q * L
    return L * np.sinc(x / np.pi) * np.exp(1j * x)


def _dseg(q, L):
    """d/dq of (e^{iqL} - 1)/(iq) = i int_0^L x e^{iqx} dx, closed form away from q = 0."""
    if q == 0:
        return 0.5j * L * L
    e = np.exp(1j * q * L)
    return 1j * (L * e / (1j * q) - (e - 1) / (1j * q) ** 2)


def _dF(verts, q, loop_off=None):
    """Complex dF/dQ [n_q, 2] from two real-weighted calls: g = 1 gives Re dF, g = i gives Im dF."""
    one = np.ones(len(q))
    return oracle.qgrad2d(verts, q, one, loop_off) + 1j * oracle.qgrad2d(verts, q, 1j * one, loop_off)


def test_rectangle_closed_form_gradient(rng):
    a, b = 1.25, 0.75
    v = np.array([[0.0, 0.0], [a, 0.0], [a, b], [0.0, b]])
    q = np.concatenate([[[0.0, 0.0], [2.0, 0.0], [0.0, -3.0]], rng.uniform(-12, 12, (40, 2))])
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    got = oracle.qgrad2d(v, q, g)
    ref = np.array([[np.real(np.conj(gi) * _dseg(Q[0], a) * _seg(Q[1], b)),
                     np.real(np.conj(gi) * _seg(Q[0], a) * _dseg(Q[1], b))] for Q, gi in zip(q, g)])
    scale = np.max(np.abs(g)) * a * b * np.hypot(a, b)
    assert np.max(np.abs(got - ref)) < 1e-9 * scale


def test_first_moment_by_quadrature(rng):
    """A 40-vertex star off the origin: dF/dQ against i * integral of r e^{iQ.r} over signed fan
    triangles (Gauss-Legendre, independent of the segment formula)."""
    v = synth.star_polygon(40, seed=8).astype(np.float64) + np.array([0.3, -0.2])
    q = np.concatenate([[[0.0, 0.0], [1e-3, 0.0]], rng.uniform(-9, 9, (30, 2))])
    got = _dF(v, q)
    ref = quad.moment2d_fan(v, q, n=40)
    area = abs(oracle.ft2d(v, [[0.0, 0.0]])[0])
    rmax = float(np.max(np.linalg.norm(v, axis=1)))
    assert np.max(np.abs(got - ref)) < 1e-9 * area * rmax


def test_translation_hermitian_and_zero(rng):
    v = synth.star_polygon(32, seed=9).astype(np.float64)
    t = np.array([0.25, -0.5])
    q = rng.uniform(-10, 10, (50, 2))
    F = oracle.ft2d(v, q)
    lhs = _dF(v + t, q)
    rhs = np.exp(1j * (q @ t))[:, None] * (1j * t[None, :] * F[:, None] + _dF(v, q))
    area = abs(oracle.ft2d(v, [[0.0, 0.0]])[0])
    assert np.max(np.abs(lhs - rhs)) < 1e-9 * area * 2.0
    # F(-Q) = conj F(Q)  =>  dF/dQ(-Q) = -conj(dF/dQ(Q))
    assert np.max(np.abs(_dF(v, -q) + np.conj(_dF(v, q)))) < 1e-9 * area
    # at Q = 0: i times the first moment of the area, from the shoelace-type centroid formula
    p0, p1 = v, np.roll(v, -1, axis=0)
    c = p0[:, 0] * p1[:, 1] - p1[:, 0] * p0[:, 1]
    m = np.array([np.sum((p0[:, 0] + p1[:, 0]) * c), np.sum((p0[:, 1] + p1[:, 1]) * c)]) / 6.0
    assert np.max(np.abs(_dF(v, [[0.0, 0.0]])[0] - 1j * m)) < 1e-9 * area


def test_loops_with_a_hole(rng):
    """An outer CCW loop and an inner CW loop: the gradient is the difference of the two shapes'."""
    outer = synth.regular_polygon(24, 1.0).astype(np.float64)
    inner = (0.4 * synth.regular_polygon(12, 1.0).astype(np.float64) + np.array([0.1, 0.05]))[::-1]
    v = np.concatenate([outer, inner])
    off = np.array([0, outer.shape[0], v.shape[0]], np.int64)
    q = rng.uniform(-8, 8, (30, 2))
    got = _dF(v, q, off)
    ref = _dF(outer, q) - _dF(inner[::-1].copy(), q)
    assert np.max(np.abs(got - ref)) < 1e-9 * np.pi
