"""The oracle's Q-gradient (Richardson-extrapolated differences of ft3d) against what fixes it
independently: the derivative of the box closed form, the translation identity
dF_{P+t}/dQ = e^{iQ.t} (i t F_P + dF_P/dQ), and Hermitian symmetry."""
import numpy as np

import oracle
from paper_2104_08309_gb300 import synth


def _seg(q, L):
    x = 0.5 * q * L
    return L * np.sinc(x / np.pi) * np.exp(1j * x)


def _dseg(q, L):
    """d/dq of (e^{iqL} - 1)/(iq) = i int_0^L x e^{iqx} dx, closed form away from q = 0."""
    if q == 0:
        return 0.5j * L * L
    e = np.exp(1j * q * L)
    return 1j * (L * e / (1j * q) - (e - 1) / (1j * q) ** 2)


def test_box_closed_form_gradient(rng):
    L = (1.25, 0.75, 1.875)
    v, f = synth.box_mesh(*L)
    q = np.concatenate([[[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]], rng.uniform(-8, 8, (40, 3))])
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    got = oracle.qgrad3d(v, f, q, g)
    ref = np.empty_like(got)
    for i, Q in enumerate(q):
        s = [_seg(Q[c], L[c]) for c in range(3)]
        for j in range(3):
            d = _dseg(Q[j], L[j]) * np.prod([s[c] for c in range(3) if c != j])
            ref[i, j] = np.real(np.conj(g[i]) * d)
    scale = np.max(np.abs(g)) * np.prod(L) * np.linalg.norm(L)
    assert np.max(np.abs(got - ref)) < 1e-9 * scale


def test_translation_identity_and_hermitian_symmetry(rng):
    v, f = synth.perturbed_icosphere(2, seed=3, amp=0.1)
    v = v.astype(np.float64)                    # the oracle works in FP64: P + t is exact enough
    t = np.array([0.25, -0.5, 0.375])
    q = rng.uniform(-10, 10, (60, 3))
    one = np.ones(q.shape[0])
    # complex gradient from two real-weighted calls: g = 1 gives Re dF, g = i gives Im dF
    def dF(verts, qq):
        return oracle.qgrad3d(verts, f, qq, one) + 1j * oracle.qgrad3d(verts, f, qq, 1j * one)
    F = oracle.ft3d(v, f, q)
    lhs = dF(v + t, q)
    rhs = np.exp(1j * (q @ t))[:, None] * (1j * t[None, :] * F[:, None] + dF(v, q))
    vol = abs(oracle.ft3d(v, f, [[0.0, 0.0, 0.0]])[0])
    assert np.max(np.abs(lhs - rhs)) < 1e-9 * vol * 2.0
    # F(-Q) = conj F(Q)  =>  dF/dQ(-Q) = -conj(dF/dQ(Q))
    assert np.max(np.abs(dF(v, -q) + np.conj(dF(v, q)))) < 1e-9 * vol
