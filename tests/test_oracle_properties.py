"""Property tests of the FP64 oracle over generated shapes and Q points (hypothesis).

Each property holds for the exact transform of any shape, so a plausible slip in the oracle (a
dropped term, a wrong sign, a transposed operand, a branch that disagrees with its neighbour)
fails one of them for some draw:
  * Hermitian symmetry F(-Q) = conj F(Q);
  * translation F_{P+t}(Q) = e^{iQ.t} F_P(Q);
  * additivity: cutting a polygon along a chord gives two loops whose transforms add up to the
    whole (the chord is traversed once each way);
  * orientation: reversing the loop negates F;
  * |F(Q)| <= F(0) (the area or volume) for any Q;
  * 90-degree rotations (exact in floating point) with Q rotated alike;
  * scaling by 2: F_{2P}(Q) = 4 F_P(2Q) in 2D, 8 F_P(2Q) in 3D.
"""
import numpy as np
import pytest

import oracle
from paper_2104_08309_gb300 import synth

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

SETTINGS = dict(max_examples=150, deadline=None, derandomize=True)
q2d = st.tuples(st.floats(-30, 30), st.floats(-30, 30))
q3d = st.tuples(st.floats(-20, 20), st.floats(-20, 20), st.floats(-20, 20))
small_or_large = st.one_of(st.floats(-1e-3, 1e-3), st.floats(-30, 30))


def _star(n, seed):
    return synth.star_polygon(n, seed=seed).astype(np.float64)


@settings(**SETTINGS)
@given(n=st.integers(3, 60), seed=st.integers(0, 10_000), q=q2d,
       t=st.tuples(st.floats(-2, 2), st.floats(-2, 2)))
def test_2d_hermitian_translation_bound(n, seed, q, t):
    v = _star(n, seed)
    Q = np.array([q, [-q[0], -q[1]]])
    F = oracle.ft2d(v, Q)
    area = oracle.ft2d(v, [[0.0, 0.0]])[0].real
    assert abs(F[1] - np.conj(F[0])) < 1e-12 * area
    assert abs(F[0]) <= area * (1 + 1e-12)
    tt = np.array(t)
    Ft = oracle.ft2d(v + tt, Q[:1])[0]
    assert abs(Ft - np.exp(1j * (Q[0] @ tt)) * F[0]) < 1e-11 * area


@settings(**SETTINGS)
@given(n=st.integers(4, 60), seed=st.integers(0, 10_000), qx=small_or_large, qy=small_or_large)
def test_2d_chord_additivity_and_orientation(n, seed, qx, qy):
    """Cut the star along the chord from vertex 0 to vertex n//2: the two loops traverse the chord
    once in each direction, so their transforms sum to the whole (whether or not they are simple)."""
    v = _star(n, seed)
    k = n // 2
    a = v[:k + 1]
    b = np.concatenate([v[k:], v[:1]])
    Q = np.array([[qx, qy]])
    whole = oracle.ft2d(v, Q)[0]
    area = oracle.ft2d(v, [[0.0, 0.0]])[0].real
    assert abs(oracle.ft2d(a, Q)[0] + oracle.ft2d(b, Q)[0] - whole) < 1e-11 * area
    assert abs(oracle.ft2d(v[::-1].copy(), Q)[0] + whole) < 1e-12 * area


@settings(**SETTINGS)
@given(n=st.integers(3, 40), seed=st.integers(0, 10_000), q=q2d)
def test_2d_rotation_and_scaling(n, seed, q):
    v = _star(n, seed)
    Q = np.array([q])
    F = oracle.ft2d(v, Q)[0]
    area = oracle.ft2d(v, [[0.0, 0.0]])[0].real
    rot = np.stack([-v[:, 1], v[:, 0]], axis=1)                # (x, y) -> (-y, x), exact
    Qr = np.stack([-Q[:, 1], Q[:, 0]], axis=1)
    assert abs(oracle.ft2d(rot, Qr)[0] - F) < 1e-11 * area
    assert abs(oracle.ft2d(2.0 * v, 0.5 * Q)[0] - 4.0 * F) < 4e-11 * area


@settings(max_examples=60, deadline=None, derandomize=True)
@given(level=st.integers(0, 2), seed=st.integers(0, 10_000), q=q3d,
       t=st.tuples(st.floats(-1, 1), st.floats(-1, 1), st.floats(-1, 1)))
def test_3d_hermitian_translation_rotation_scaling(level, seed, q, t):
    v, f = synth.perturbed_icosphere(level, seed=seed, amp=0.2)
    v = v.astype(np.float64)
    Q = np.array([q, [-q[0], -q[1], -q[2]]])
    F = oracle.ft3d(v, f, Q)
    vol = oracle.ft3d(v, f, [[0.0, 0.0, 0.0]])[0].real
    assert abs(F[1] - np.conj(F[0])) < 1e-12 * vol
    assert abs(F[0]) <= vol * (1 + 1e-12)
    tt = np.array(t)
    assert abs(oracle.ft3d(v + tt, f, Q[:1])[0] - np.exp(1j * (Q[0] @ tt)) * F[0]) < 1e-11 * vol
    rot = np.stack([-v[:, 1], v[:, 0], v[:, 2]], axis=1)       # 90 degrees about z, exact
    Qr = np.array([[-q[1], q[0], q[2]]])
    assert abs(oracle.ft3d(rot, f, Qr)[0] - F[0]) < 1e-11 * vol
    assert abs(oracle.ft3d(2.0 * v, f, 0.5 * Q[:1])[0] - 8.0 * F[0]) < 8e-11 * vol
    assert abs(oracle.ft3d(v, f[:, ::-1].copy(), Q[:1])[0] + F[0]) < 1e-12 * vol
