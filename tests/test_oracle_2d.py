"""Pins of the 2D oracle against what the paper and the mathematics fix.

Each test checks oracle.ft2d (Eq. 6 summed over CCW segments, Sec. 2) against
something it does not compute itself: the paper's rectangle worked example
(Sec. 4.1), brute-force quadrature, the disc limit, exact invariances and the
Q -> 0 limit.
"""
import numpy as np
import pytest
from scipy.special import j1

import oracle
from paper_2104_08309_gb300 import synth
from tests import quadrature as quad

A, B = 2.0, 1.5


def rect_closed_form(q, a=A, b=B):
    """Separable integral of Sec. 4.1 (product of two 1D integrals, with their Q -> 0 limits)."""
    def one(k, L):
        # (exp(ikL) - 1)/(ik) with exp(ikL) - 1 = -2 sin^2(kL/2) + i sin(kL) (no cancellation)
        if k == 0:
            return L
        return (-2.0 * np.sin(0.5 * k * L) ** 2 + 1j * np.sin(k * L)) / (1j * k)
    return np.array([one(qx, a) * one(qy, b) for qx, qy in q])


def test_rectangle_closed_form(rng):
    q = np.concatenate([rng.uniform(-20, 20, (200, 2)),
                        [[0.0, 1.3], [2.1, 0.0], [0.0, 0.0], [1e-7, 3e-7], [1e-3, -2e-3]]])
    F = oracle.ft2d(synth.rectangle(A, B), q)
    ref = rect_closed_form(q)
    assert np.max(np.abs(F - ref)) < 1e-12 * A * B


def test_rectangle_edge_terms_match_paper():
    """The four segment terms printed in Sec. 4.1 (exponential-difference form, Eq. 4)."""
    a, b = A, B
    for qx, qy in [(0.7, -1.3), (3.0, 2.0), (-5.5, 0.25)]:
        q2 = qx * qx + qy * qy
        e = lambda x: np.exp(1j * x)
        printed = np.array([
            (qy * a) / (qx * a) * (e(qx * a) - 1.0),
            (-qx * b) / (qy * b) * (e(qx * a + qy * b) - e(qx * a)),
            (-qy * a) / (-qx * a) * (e(qy * b) - e(qx * a + qy * b)),
            (qx * b) / (-qy * b) * (1.0 - e(qy * b)),
        ]) / q2
        terms = oracle.seg_terms2d(synth.rectangle(a, b), (qx, qy))
        assert np.max(np.abs(terms - printed)) < 1e-13
        # and the closed form of the sum given after them
        total = (1.0 / q2) * (q2 / (qx * qy)) * (e(qy * b) + e(qx * a) - e(qx * a + qy * b) - 1.0)
        assert abs(terms.sum() - total) < 1e-12


@pytest.mark.parametrize("n,seed", [(5, 11), (9, 12), (17, 13)])
def test_star_vs_bruteforce_quadrature(n, seed, rng):
    v = synth.star_polygon(n, seed=seed, center=(0.3, -0.2))
    q = np.concatenate([rng.uniform(-6, 6, (12, 2)), [[0.0, 0.0], [1e-4, 0.0], [0.0, 4.0]]])
    F = oracle.ft2d(v, q)
    ref = quad.ft2d_fan(v.astype(np.float64), q, n=40)
    assert np.max(np.abs(F - ref)) < 1e-12


def test_regular_ngon_converges_to_disc():
    """N-gon -> disc 2 pi R J1(QR)/Q with error O(N^-2) (ratio ~4 per doubling)."""
    R = 1.0
    q = np.array([[0.9, 0.4], [3.0, -2.0], [7.5, 1.0]])
    Qn = np.linalg.norm(q, axis=1)
    disc = 2 * np.pi * R * j1(Qn * R) / Qn
    errs = []
    for n in (64, 128, 256, 512):
        v = synth.regular_polygon(n, R).astype(np.float64)
        # use exact (float64) vertices so that only the polygonal error remains
        th = 2 * np.pi * np.arange(n) / n
        v = np.stack([R * np.cos(th), R * np.sin(th)], 1)
        errs.append(np.max(np.abs(oracle.ft2d(v, q) - disc)))
        area = oracle.ft2d(v, [[0.0, 0.0]])[0]
        assert abs(area - 0.5 * n * R * R * np.sin(2 * np.pi / n)) < 1e-13
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 3.5) & (ratios < 4.5)), ratios


def test_invariances(rng):
    v = synth.star_polygon(23, seed=5).astype(np.float64)
    q = rng.uniform(-15, 15, (64, 2))
    F = oracle.ft2d(v, q)
    # translation: F_{P+t}(Q) = exp(iQ.t) F_P(Q)
    t = np.array([0.75, -1.25])
    assert np.max(np.abs(oracle.ft2d(v + t, q) - np.exp(1j * q @ t) * F)) < 1e-12
    # rotation by 90 degrees of both shape and Q
    rot = lambda a: np.stack([-a[:, 1], a[:, 0]], 1)
    assert np.max(np.abs(oracle.ft2d(rot(v), rot(q)) - F)) < 1e-12
    # Hermitian symmetry
    assert np.max(np.abs(oracle.ft2d(v, -q) - np.conj(F))) < 1e-12
    # scaling: F_{2P}(Q) = 4 F_P(2Q)
    assert np.max(np.abs(oracle.ft2d(2 * v, q) - 4 * oracle.ft2d(v, 2 * q))) < 1e-11
    # reversed orientation gives the negative
    assert np.max(np.abs(oracle.ft2d(v[::-1], q) + F)) < 1e-12


def test_centrosymmetric_is_real(rng):
    half = synth.star_polygon(8, seed=9).astype(np.float64)[:4]
    th = np.arctan2(half[:, 1], half[:, 0])
    assert np.all(np.diff(th) > 0)
    v = np.concatenate([half, -half])            # point-symmetric about the origin
    F = oracle.ft2d(v, rng.uniform(-10, 10, (50, 2)))
    assert np.max(np.abs(F.imag)) < 1e-13


def test_additivity_and_holes(rng):
    q = rng.uniform(-8, 8, (40, 2))
    sq = np.array([[0, 0], [2, 0], [2, 2], [0, 2]], dtype=np.float64)
    left = np.array([[0, 0], [1, 0], [1, 2], [0, 2]], dtype=np.float64)
    right = np.array([[1, 0], [2, 0], [2, 2], [1, 2]], dtype=np.float64)
    assert np.max(np.abs(oracle.ft2d(sq, q) - oracle.ft2d(left, q) - oracle.ft2d(right, q))) < 1e-12
    # a CW inner loop is a hole
    hole = np.array([[0.5, 0.5], [0.5, 1.5], [1.5, 1.5], [1.5, 0.5]], dtype=np.float64)
    both = np.concatenate([sq, hole])
    F = oracle.ft2d(both, q, loop_off=[0, 4, 8])
    assert np.max(np.abs(F - (oracle.ft2d(sq, q) + oracle.ft2d(hole, q)))) < 1e-12
    assert abs(oracle.ft2d(both, [[0, 0]], loop_off=[0, 4, 8])[0] - 3.0) < 1e-14


def test_small_q_branch_agrees_with_segment_sum():
    """The |Q| -> 0 series branch and the segment sum give the same value at the same Q.

    Translating the shape moves max|r| and so the branch taken, while the exact
    transform only picks up the phase exp(iQ.t).
    """
    v = synth.star_polygon(31, seed=2).astype(np.float64)
    rmax = np.max(np.linalg.norm(v, axis=1))
    d = np.array([0.6, 0.8])
    t = np.array([3.0, -4.0])
    for scale in (0.45, 0.3, 1e-3, 1e-7):
        Q = d * scale / rmax                     # |Q| rmax < 0.5: series for v
        assert np.linalg.norm(Q) * np.max(np.linalg.norm(v + t, axis=1)) > 0.5 or scale < 0.1
        a = oracle.ft2d(v, [Q])[0]
        b = oracle.ft2d(v + t, [Q])[0] * np.exp(-1j * (Q @ t))
        assert abs(a - b) < 1e-12 * (1.0 if scale > 0.1 else 1e3), (scale, a, b)
    area = oracle.ft2d(v, [[0, 0]])[0]
    assert abs(oracle.ft2d(v, [d * 1e-12])[0] - area) < 1e-11


def test_batched_matches_single(rng):
    v, off = synth.batched_star_polygons(6, seed=7, nmin=3, nmax=40)
    q = rng.uniform(-12, 12, (30, 2))
    Fb = oracle.ft2d_batched(v, off, q)
    for i in range(6):
        Fi = oracle.ft2d(v[off[i]:off[i + 1]], q)
        assert np.max(np.abs(Fb[i] - Fi)) == 0.0
    # per-polygon Q sets (CSR)
    q_off = np.array([0, 3, 3, 10, 12, 20, 30])
    Fc = oracle.ft2d_batched(v, off, q, q_off=q_off)
    for i in range(6):
        Fi = oracle.ft2d(v[off[i]:off[i + 1]], q[q_off[i]:q_off[i + 1]])
        assert np.max(np.abs(Fc[q_off[i]:q_off[i + 1]] - Fi), initial=0.0) == 0.0
