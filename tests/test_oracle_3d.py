"""Pins of the 3D oracle against what the paper and the mathematics fix.

oracle.ft3d sums the sign-corrected Eq. 14 (Sec. 3) over the faces of a closed
outward triangle mesh.  It is checked against the prism closed form and the
prism face values of Sec. 4.2, the sphere closed form of Sec. 4.3 (convergence
under refinement), brute-force tetrahedral quadrature (including the paper's own
two-sphere mesh of Sec. 4.4 when its text is available), exact invariances, the
2D <-> 3D extrusion identity and the limits Q -> 0 and Q parallel to a face normal.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2104_08309_gb300 import synth
from tests import quadrature as quad

A, B, C = 1.25, 0.75, 1.875     # exact in float32


def _e1(k, L):
    """(exp(ikL) - 1)/(ik) without cancellation, = L at k = 0."""
    if k == 0:
        return L
    return (-2.0 * np.sin(0.5 * k * L) ** 2 + 1j * np.sin(k * L)) / (1j * k)


def prism_closed_form(q, a=A, b=B, c=C):
    """Sec. 4.2: i (e^{iQx a}-1)(e^{iQy b}-1)(e^{iQz c}-1)/(Qx Qy Qz), i.e. the product of three 1D integrals."""
    return np.array([_e1(qx, a) * _e1(qy, b) * _e1(qz, c) for qx, qy, qz in q])


def test_prism_closed_form(rng):
    v, f = synth.box_mesh(A, B, C)
    q = np.concatenate([rng.uniform(-12, 12, (150, 3)),
                        [[0, 0, 0], [0, 0, 2.5], [1.5, 0, 0], [0, -3, 0], [1, 2, 0], [0, 1, 2],
                         [1e-5, 2e-5, -1e-5], [0.2, 0.1, 0.05]]])
    F = oracle.ft3d(v, f, q)
    ref = prism_closed_form(q)
    assert np.max(np.abs(F - ref)) < 1e-12 * A * B * C


def test_prism_face_values_match_paper(rng):
    """Top (z = c) and bottom (z = 0) face terms printed in Sec. 4.2."""
    v, f = synth.box_mesh(A, B, C)
    for Q in rng.uniform(-6, 6, (8, 3)):
        qx, qy, qz = Q
        q2 = Q @ Q
        base = (np.exp(1j * qx * A) - 1) * (np.exp(1j * qy * B) - 1) / (qx * qy)
        top = 1j * qz * np.exp(1j * qz * C) / q2 * base
        bottom = -1j * qz / q2 * base
        terms = oracle.face_terms3d(v, f, Q)
        assert abs(terms[0] + terms[1] - top) < 1e-13
        assert abs(terms[2] + terms[3] - bottom) < 1e-13
        # the sum of all six faces is the closed form
        assert abs(terms.sum() - prism_closed_form([Q])[0]) < 1e-12


def test_q_parallel_to_face_normal():
    """Q along z: the side faces have Q.N = 0, the top/bottom take the Q_perp = 0 limit."""
    v, f = synth.box_mesh(A, B, C)
    for qz in (0.3, 2.0, -7.0):
        F = oracle.ft3d(v, f, [[0.0, 0.0, qz]])[0]
        assert abs(F - A * B * _e1(qz, C)) < 1e-13


def test_icosphere_converges_to_sphere():
    """Sec. 4.3: 4 pi (sin QR - QR cos QR)/Q^3; the mesh error falls ~4x per subdivision."""
    q = np.array([[0.94, 0.1, -0.3], [2.0, 3.0, 1.0], [0.0, 0.0, 4.5]])
    Qn = np.linalg.norm(q, axis=1)
    exact = 4 * np.pi * (np.sin(Qn) - Qn * np.cos(Qn)) / Qn ** 3
    errs = []
    for level in (2, 3, 4, 5):
        v, f = synth._unit_icosphere(level)          # float64 vertices: pure mesh error
        errs.append(np.max(np.abs(oracle.ft3d(v, f, q) - exact)))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 3.5) & (ratios < 4.5)), ratios


@pytest.mark.parametrize("level,amp", [(1, 0.0), (1, 0.2), (2, 0.1)])
def test_mesh_vs_bruteforce_tets(level, amp, rng):
    v, f = synth.perturbed_icosphere(level, seed=level + 10, amp=amp)
    v = v.astype(np.float64) + np.array([0.3, -0.1, 0.2])
    q = np.concatenate([rng.uniform(-4, 4, (6, 3)), [[0, 0, 0], [1e-3, 0, 0], [0, 0, 2.0]]])
    F = oracle.ft3d(v, f, q)
    ref = quad.ft3d_tets(v, f, q, n=16)
    assert np.max(np.abs(F - ref)) < 1e-11


def _paper_mesh():
    """The two-sphere surface mesh of Sec. 4.4 (83 nodes, 160 triangles), stored as printed in the
    paper's appendix data under tests/golden/."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "two_spheres_mesh.txt")
    lines = [l for l in open(path).read().splitlines() if l and not l.startswith("#")]
    tag, n = lines[0].split()
    assert tag == "points"
    n = int(n)
    pts = np.array([[float(x) for x in line.split()] for line in lines[1:1 + n]])
    tag, m = lines[1 + n].split()
    assert tag == "triangles"
    m = int(m)
    tri = np.array([[int(x) for x in line.split()] for line in lines[2 + n:2 + n + m]]) - 1
    return pts, tri


def test_paper_two_sphere_mesh_vs_bruteforce(rng):
    """The two-sphere surface mesh of Sec. 4.4 (netgen output printed in the appendix)."""
    pts, tri = _paper_mesh()
    assert pts.shape == (83, 3) and tri.shape == (160, 3)
    q = np.concatenate([[[0.5, 0.3, 0.2], [3.0, -1.0, 2.0], [2.0, 1e-30, 1e-30], [0, 0, 0]],
                        rng.uniform(-5, 5, (4, 3))])
    F = oracle.ft3d(pts, tri, q)
    ref = quad.ft3d_tets(pts, tri, q, n=16)
    assert np.max(np.abs(F - ref)) < 1e-11
    assert F[3].real > 0                              # outward faces: positive volume


def test_invariances(rng):
    v, f = synth.perturbed_icosphere(2, seed=3, amp=0.15)
    v = v.astype(np.float64)
    q = rng.uniform(-8, 8, (48, 3))
    F = oracle.ft3d(v, f, q)
    t = np.array([0.5, -0.25, 1.5])
    assert np.max(np.abs(oracle.ft3d(v + t, f, q) - np.exp(1j * q @ t) * F)) < 1e-12
    rot = lambda a: np.stack([-a[:, 1], a[:, 0], a[:, 2]], 1)
    assert np.max(np.abs(oracle.ft3d(rot(v), f, rot(q)) - F)) < 1e-12
    assert np.max(np.abs(oracle.ft3d(v, f, -q) - np.conj(F))) < 1e-12
    assert np.max(np.abs(oracle.ft3d(2 * v, f, q) - 8 * oracle.ft3d(v, f, 2 * q))) < 1e-11
    assert np.max(np.abs(oracle.ft3d(v, f[:, ::-1], q) + F)) < 1e-12


def _extrude(poly, h):
    """Prism over a star polygon (centre-fan caps), outward triangles."""
    n = poly.shape[0]
    bot = np.concatenate([poly, np.zeros((n, 1))], 1)
    top = np.concatenate([poly, np.full((n, 1), h)], 1)
    v = np.concatenate([bot, top, [[0, 0, 0], [0, 0, h]]])
    cb, ct = 2 * n, 2 * n + 1
    faces = []
    for j in range(n):
        k = (j + 1) % n
        faces += [[cb, k, j], [ct, n + j, n + k], [j, k, n + k], [j, n + k, n + j]]
    return v, np.array(faces, dtype=np.int32)


def test_extrusion_2d_3d_identity(rng):
    poly = synth.star_polygon(12, seed=8).astype(np.float64)
    h = 0.8
    v, f = _extrude(poly, h)
    q = np.concatenate([rng.uniform(-6, 6, (30, 3)), [[1.0, 2.0, 0.0], [0.0, 0.0, 3.0]]])
    F3 = oracle.ft3d(v, f, q)
    F2 = oracle.ft2d(poly, q[:, :2])
    ref = F2 * np.array([_e1(qz, h) for qz in q[:, 2]])
    assert np.max(np.abs(F3 - ref)) < 1e-12


def test_union_is_sum_and_volume(rng):
    v, f = synth.sphere_union(3, 1, seed=1)
    nv, nf = v.shape[0] // 3, f.shape[0] // 3
    q = rng.uniform(-10, 10, (20, 3))
    F = oracle.ft3d(v, f, q)
    parts = sum(oracle.ft3d(v[i * nv:(i + 1) * nv], f[i * nf:(i + 1) * nf] - i * nv, q) for i in range(3))
    assert np.max(np.abs(F - parts)) < 1e-12
    vol = oracle.ft3d(v, f, [[0, 0, 0]])[0]
    p = v.astype(np.float64)[f]
    assert abs(vol - np.einsum("ij,ij->i", p[:, 0], np.cross(p[:, 1], p[:, 2])).sum() / 6) < 1e-13


def test_branches_agree_at_the_same_q():
    """Face series vs edge sum, and shape series vs face sum, at one Q via translation.

    Translating moves max|r| (and so the |Q| -> 0 branch) but not the exact result
    beyond the phase exp(iQ.t); rotating the Q direction slightly off a face normal
    moves a face across the small-spread threshold.
    """
    v, f = synth.icosphere(2)
    v = v.astype(np.float64)
    t = np.array([2.0, 1.0, -2.0])
    for scale in (0.45, 0.2):
        Q = np.array([0.36, 0.48, 0.8]) * scale / np.max(np.linalg.norm(v, axis=1))
        a = oracle.ft3d(v, f, [Q])[0]
        b = oracle.ft3d(v + t, f, [Q])[0] * np.exp(-1j * (Q @ t))
        assert abs(a - b) < 1e-12
    # a single face: thresholds of the face branch (spread = max |Q.d_l| = 1e-2)
    p = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    for qz in (0.9, 3.0):
        for eps in (0.9e-2, 1.1e-2, 0.5e-2, 2e-2):
            Q = np.array([eps, 0.0, qz])
            term = oracle.face_terms3d(p, tri, Q)[0]
            # direct quadrature of the face integral of Eq. 13 with -i Q_par/|Q|^2
            l1, l2, w = quad.tri_rule(20)
            pts = l1[:, None] * p[1] + l2[:, None] * p[2]
            integral = np.sum(w * np.exp(1j * pts @ Q))     # area 1/2 * 2 = weights sum 1/2
            ref = -1j * Q[2] / (Q @ Q) * integral
            assert abs(term - ref) < 1e-14, (qz, eps, term, ref)


def test_degenerate_faces_contribute_nothing(rng):
    """Zero-area faces (a repeated corner, or three collinear corners) add nothing."""
    v, f = synth.perturbed_icosphere(2, seed=6, amp=0.05)
    q = rng.uniform(-12, 12, (100, 3))
    base = oracle.ft3d(v, f, q)
    v2 = np.concatenate([v, [[0.25, 0.5, 0.75], [0.5, 1.0, 1.5], [0.75, 1.5, 2.25]]]).astype(np.float32)
    n = v.shape[0]
    extra = np.array([[0, 0, 5], [7, 3, 7], [n, n + 1, n + 2]], np.int32)
    got = oracle.ft3d(v2, np.concatenate([f, extra]), q)
    assert np.max(np.abs(got - base)) < 1e-13 * abs(oracle.ft3d(v, f, [[0.0, 0.0, 0.0]])[0])
