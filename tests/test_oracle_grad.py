"""Pins of the oracle's vertex gradients (shape derivative of the transform).

The gradients are checked against central finite differences of the pinned
forward oracle, against the translation identity sum_k dF/dv_k = i Q F, and
against the Q = 0 limits (derivatives of the shoelace area and of the
signed-tetrahedron volume).
"""
import numpy as np

import oracle
from paper_2104_08309_gb300 import synth


def _loss_parts(F, target):
    """L = sum (|F|^2 - I)^2 and g = dL/dRe F + i dL/dIm F = 4 (|F|^2 - I) F."""
    r = np.abs(F) ** 2 - target
    return np.sum(r * r), 4.0 * r * F


def test_grad2d_vs_central_fd(rng):
    v = synth.star_polygon(10, seed=4).astype(np.float64)
    q = rng.uniform(-6, 6, (40, 2))
    target = np.abs(oracle.ft2d(v * 1.03, q)) ** 2
    F = oracle.ft2d(v, q)
    _, g = _loss_parts(F, target)
    G = oracle.grad2d(v, q, g)
    h = 1e-6
    for j in range(v.shape[0]):
        for c in range(2):
            vp, vm = v.copy(), v.copy()
            vp[j, c] += h
            vm[j, c] -= h
            fd = (_loss_parts(oracle.ft2d(vp, q), target)[0] - _loss_parts(oracle.ft2d(vm, q), target)[0]) / (2 * h)
            assert abs(fd - G[j, c]) < 1e-6 * max(1.0, abs(fd)), (j, c, fd, G[j, c])


def test_grad2d_identities(rng):
    v = synth.star_polygon(9, seed=6).astype(np.float64) + np.array([0.2, -0.4])
    # translation: sum_k dF/dv_k = i Q F.  With g = 1: sum_k Re dF/dv_k = Re(i Q F) = -Q Im F
    for Q in rng.uniform(-5, 5, (5, 2)):
        F = oracle.ft2d(v, [Q])[0]
        s1 = oracle.grad2d(v, [Q], np.array([1.0 + 0j])).sum(0)
        si = oracle.grad2d(v, [Q], np.array([1j])).sum(0)      # Re(conj(i) dF) = Im dF
        assert np.allclose(s1, -Q * F.imag, atol=1e-12)
        assert np.allclose(si, Q * F.real, atol=1e-12)
    # Q = 0: dA/dv_k = 1/2 (y_{k+1} - y_{k-1}, x_{k-1} - x_{k+1})
    G = oracle.grad2d(v, [[0.0, 0.0]], np.array([1.0 + 0j]))
    nxt, prv = np.roll(v, -1, 0), np.roll(v, 1, 0)
    ref = 0.5 * np.stack([nxt[:, 1] - prv[:, 1], prv[:, 0] - nxt[:, 0]], 1)
    assert np.max(np.abs(G - ref)) < 1e-14


def test_grad3d_vs_central_fd(rng):
    v, f = synth.perturbed_icosphere(1, seed=2, amp=0.1)
    v = v.astype(np.float64) + np.array([0.1, 0.2, -0.3])
    q = np.concatenate([rng.uniform(-5, 5, (24, 3)), [[0.0, 0.0, 0.0], [0.0, 0.0, 3.0]]])
    target = np.abs(oracle.ft3d(v * 1.02, f, q)) ** 2
    F = oracle.ft3d(v, f, q)
    _, g = _loss_parts(F, target)
    G = oracle.grad3d(v, f, q, g)
    h = 1e-6
    for j in rng.choice(v.shape[0], 12, replace=False):
        for c in range(3):
            vp, vm = v.copy(), v.copy()
            vp[j, c] += h
            vm[j, c] -= h
            fd = (_loss_parts(oracle.ft3d(vp, f, q), target)[0] - _loss_parts(oracle.ft3d(vm, f, q), target)[0]) / (2 * h)
            assert abs(fd - G[j, c]) < 1e-6 * max(1.0, abs(fd)), (j, c, fd, G[j, c])
    # vertex selection returns the same rows
    sel = np.array([5, 0, 17])
    assert np.max(np.abs(oracle.grad3d(v, f, q, g, vsel=sel) - G[sel])) < 1e-14


def test_grad3d_large_spread_subdivision(rng):
    """Spreads above the subdivision threshold (large |Q| on a coarse mesh) still match FD."""
    v, f = synth.perturbed_icosphere(0, seed=9, amp=0.1)
    v = v.astype(np.float64)
    q = rng.uniform(-9, 9, (6, 3))
    g = rng.normal(size=6) + 1j * rng.normal(size=6)
    G = oracle.grad3d(v, f, q, g)
    h = 1e-6
    for j in range(4):
        for c in range(3):
            vp, vm = v.copy(), v.copy()
            vp[j, c] += h
            vm[j, c] -= h
            dF = (oracle.ft3d(vp, f, q) - oracle.ft3d(vm, f, q)) / (2 * h)
            fd = np.sum(np.real(np.conj(g) * dF))
            assert abs(fd - G[j, c]) < 1e-6 * max(1.0, abs(fd))


def test_grad3d_identities(rng):
    v, f = synth.perturbed_icosphere(1, seed=8, amp=0.2)
    v = v.astype(np.float64)
    for Q in rng.uniform(-4, 4, (4, 3)):
        F = oracle.ft3d(v, f, [Q])[0]
        s1 = oracle.grad3d(v, f, [Q], np.array([1.0 + 0j])).sum(0)
        si = oracle.grad3d(v, f, [Q], np.array([1j])).sum(0)
        assert np.allclose(s1, -Q * F.imag, atol=1e-12)
        assert np.allclose(si, Q * F.real, atol=1e-12)
    # Q = 0: dV/dv_k = sum over faces m of (p_{k+1} x p_{k+2}) / 6 (derivative of the tetra volumes)
    G = oracle.grad3d(v, f, [[0.0, 0.0, 0.0]], np.array([1.0 + 0j]))
    ref = np.zeros_like(v)
    for tri in f:
        for k in range(3):
            ref[tri[k]] += np.cross(v[tri[(k + 1) % 3]], v[tri[(k + 2) % 3]]) / 6.0
    assert np.max(np.abs(G - ref)) < 1e-14
