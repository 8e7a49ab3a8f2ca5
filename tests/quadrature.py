"""Brute-force quadrature of exp(iQ.r) over triangles and tetrahedra (test helper).

Independent of both the oracle and the CUDA path: tensor Gauss-Legendre rules
mapped onto simplices with the collapsed (Duffy) coordinates, summed in numpy.
Signed fans from the origin turn a closed boundary into the area/volume
integral.
"""
import numpy as np


def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def tri_rule(n):
    """Points (barycentric l1, l2) and weights on the unit triangle (area 1/2)."""
    x, w = _gl(n)
    u, v = np.meshgrid(x, x, indexing="ij")
    wu, wv = np.meshgrid(w, w, indexing="ij")
    l1 = u
    l2 = (1.0 - u) * v
    return l1.ravel(), l2.ravel(), (wu * wv * (1.0 - u)).ravel()


def tet_rule(n):
    """Points (l1, l2, l3) and weights on the unit tetrahedron (volume 1/6)."""
    x, w = _gl(n)
    u, v, t = np.meshgrid(x, x, x, indexing="ij")
    wu, wv, wt = np.meshgrid(w, w, w, indexing="ij")
    l1 = u
    l2 = (1.0 - u) * v
    l3 = (1.0 - u) * (1.0 - v) * t
    return l1.ravel(), l2.ravel(), l3.ravel(), (wu * wv * wt * (1.0 - u) ** 2 * (1.0 - v)).ravel()


def ft2d_fan(verts, q, n=24):
    """Integral of exp(iQ.r) over a CCW polygon via signed triangles (0, p_j, p_{j+1})."""
    v = np.asarray(verts, dtype=np.float64)
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    l1, l2, w = tri_rule(n)
    p0, p1 = v, np.roll(v, -1, axis=0)
    det = p0[:, 0] * p1[:, 1] - p0[:, 1] * p1[:, 0]            # 2 x signed area
    pts = l1[None, :, None] * p0[:, None, :] + l2[None, :, None] * p1[:, None, :]   # [seg, pt, 2]
    out = np.empty(q.shape[0], dtype=np.complex128)
    for i, Q in enumerate(q):
        ph = np.exp(1j * (pts @ Q))                              # [seg, pt]
        out[i] = np.sum(det[:, None] * w[None, :] * ph)
    return out


def ft3d_tets(verts, faces, q, n=14):
    """Integral of exp(iQ.r) inside a closed outward mesh via signed tetrahedra (0, p0, p1, p2)."""
    v = np.asarray(verts, dtype=np.float64)
    f = np.asarray(faces)
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    l1, l2, l3, w = tet_rule(n)
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    det = np.einsum("ij,ij->i", a, np.cross(b, c))                # 6 x signed volume
    out = np.empty(q.shape[0], dtype=np.complex128)
    for i, Q in enumerate(q):
        qa, qb, qc = a @ Q, b @ Q, c @ Q
        ph = np.exp(1j * (l1[None, :] * qa[:, None] + l2[None, :] * qb[:, None] + l3[None, :] * qc[:, None]))
        out[i] = np.sum(det[:, None] * w[None, :] * ph)
    return out


def moment2d_fan(verts, q, n=24):
    """i times the first moment, i * integral of r exp(iQ.r) over a CCW polygon ([n_q, 2]): the
    Q-derivative of the transform, by the same signed triangles (0, p_j, p_{j+1})."""
    v = np.asarray(verts, dtype=np.float64)
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    l1, l2, w = tri_rule(n)
    p0, p1 = v, np.roll(v, -1, axis=0)
    det = p0[:, 0] * p1[:, 1] - p0[:, 1] * p1[:, 0]
    pts = l1[None, :, None] * p0[:, None, :] + l2[None, :, None] * p1[:, None, :]
    out = np.empty((q.shape[0], 2), dtype=np.complex128)
    for i, Q in enumerate(q):
        ph = (det[:, None] * w[None, :]) * np.exp(1j * (pts @ Q))
        out[i] = 1j * np.einsum("sp,spd->d", ph, pts)
    return out
