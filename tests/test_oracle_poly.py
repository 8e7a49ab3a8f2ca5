"""The oracle's polygon-face form of Eq. 14 (planar faces of any size, Newell normal) against
what fixes it independently: the box closed form, the 2D <-> 3D extrusion identity with the
2D oracle (convex and non-convex caps, Q along the cap normal), the volume at Q = 0, and the
triangle form of Eq. 14 on the fan-triangulated mesh (a different edge set, the same integral)."""
import numpy as np
import pytest

import oracle
from paper_2104_08309_gb300 import synth


def _seg(q, L):
    """(e^{iqL} - 1)/(iq) = L sinc(qL/2) e^{iqL/2}, written without cancellation at small q."""
    x = 0.5 * np.asarray(q) * L
    return L * np.sinc(x / np.pi) * np.exp(1j * x)


def _box_closed_form(Q, L):
    r = 1.0 + 0j
    for qc, lc in zip(Q, L):
        r *= _seg(qc, lc)
    return r


def _fan(idx, off):
    tris = []
    for m in range(off.size - 1):
        f = idx[off[m]:off[m + 1]]
        tris += [[f[0], f[k], f[k + 1]] for k in range(1, f.size - 1)]
    return np.array(tris, dtype=np.int32)


def _extrusion(F2, qz, h):
    return F2 * _seg(qz, h)


def test_box_quads_closed_form(rng):
    L = (1.25, 0.75, 1.875)
    v, idx, off = synth.box_quads(*L)
    q = np.concatenate([[[0, 0, 0], [1e-7, 0, 0], [0, 0, 2.0], [3.0, 0, 0], [1, 2, 3]], rng.uniform(-20, 20, (300, 3))])
    got = oracle.ft3d_poly(v, idx, off, q)
    ref = np.array([_box_closed_form(Q, L) for Q in q])
    assert np.max(np.abs(got - ref)) < 1e-12 * np.prod(L)


@pytest.mark.parametrize("cap", ["hexagon", "star"])
def test_extrusion_identity(cap, rng):
    """Prism over a cap polygon P with height h: F(Q) = F_P(Qx, Qy) (e^{iQz h} - 1)/(iQz)."""
    poly = synth.regular_polygon(6, 1.0) if cap == "hexagon" else synth.star_polygon(57, seed=9)
    poly = poly.astype(np.float32)          # the mesh holds FP32 coordinates; both sides use them
    h = 0.75
    v, idx, off = synth.extruded_polygon(poly, h)
    q = np.concatenate([[[0, 0, 0], [0, 0, 3.0], [0, 0, -7.5], [2.0, -1.0, 0.0], [1e-6, 2e-6, 1e-6]],
                        rng.uniform(-25, 25, (400, 3))])
    got = oracle.ft3d_poly(v, idx, off, q)
    ref = _extrusion(oracle.ft2d(poly, q[:, :2]), q[:, 2], h)
    area = abs(oracle.ft2d(poly, [[0.0, 0.0]])[0])
    assert np.max(np.abs(got - ref)) < 1e-12 * area * h
    assert abs(got[0] - area * h) < 1e-13 * area * h


def test_polygon_form_equals_triangle_form_on_the_fan(rng):
    """Eq. 14 over the polygon's own edges vs over its fan triangles' edges (interior edges
    cancel only analytically): the same transform to FP64 rounding."""
    star = synth.star_polygon(33, seed=2).astype(np.float32)
    v, idx, off = synth.extruded_polygon(star, 1.5, z0=-0.25)
    q = np.concatenate([[[0, 0, 4.0], [0.3, 0.1, 0.0]], rng.uniform(-30, 30, (300, 3))])
    a = oracle.ft3d_poly(v, idx, off, q)
    b = oracle.ft3d(v, _fan(idx, off), q)
    vol = abs(oracle.ft3d_poly(v, idx, off, [[0.0, 0.0, 0.0]])[0])
    assert abs(vol - 1.5 * abs(oracle.ft2d(star, [[0.0, 0.0]])[0])) < 1e-12 * vol
    assert np.max(np.abs(a - b)) < 1e-12 * vol


def test_malformed_faces_are_rejected():
    v, idx, off = synth.box_quads(1.0, 1.0, 1.0)
    with pytest.raises(ValueError):
        oracle.ft3d_poly(v, idx, np.array([0, 2, 24]), [[1.0, 0, 0]])      # a 2-vertex face
    bad = idx.copy()
    bad[3] = 99
    with pytest.raises(ValueError):
        oracle.ft3d_poly(v, bad, off, [[1.0, 0, 0]])
