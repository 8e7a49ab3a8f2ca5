"""FP64 CPU oracle for the direct polygon / polyhedron Fourier transform.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library never does, and it
shares no code with the CUDA path.

The arithmetic lives in ``pft_oracle.c`` (plain C99, FP64, OpenMP over Q or
faces); this module compiles it with gcc on first use and wraps it with ctypes.
Sign convention: FT(Q) = integral of exp(+i Q.r) over the region (Sec. 2, Eq. 7).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pft_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile pft_oracle.c to a shared library (gcc -O2 -fopenmp, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_ft2d.argtypes = [_dp, _i64p, _i64, _dp, _i64, _dp, ctypes.c_int]
            lib.orc_seg_terms2d.argtypes = [_dp, _i64p, _i64, ctypes.c_double, ctypes.c_double, _dp]
            lib.orc_ft2d_batched.argtypes = [_dp, _i64p, _i64, _dp, _i64p, _i64, _dp, ctypes.c_int]
            lib.orc_ft3d.argtypes = [_dp, _i64, _i32p, _i64, _dp, _i64, _dp, ctypes.c_int]
            lib.orc_face_terms3d.argtypes = [_dp, _i64, _i32p, _i64, _dp, _dp]
            lib.orc_ft3d_poly.argtypes = [_dp, _i64, _i32p, _i64p, _i64, _dp, _i64, _dp, ctypes.c_int]
            lib.orc_grad2d.argtypes = [_dp, _i64p, _i64, _dp, _i64, _dp, _dp, ctypes.c_int]
            lib.orc_grad3d.argtypes = [_dp, _i64, _i32p, _i64, _dp, _i64, _dp, _i64p, _i64, _dp,
                                       ctypes.c_int]
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a, cols=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def _ptr(a, typ):
    return a.ctypes.data_as(typ)


def _threads(n):
    return int(n) if n else max(1, _load().orc_max_threads())


def _complex(out):
    return out[:, 0] + 1j * out[:, 1]


def _loops(verts, loop_off):
    v = _f64(verts, 2)
    off = np.ascontiguousarray(np.asarray(loop_off if loop_off is not None else [0, v.shape[0]],
                                          dtype=np.int64))
    return v, off


def ft2d(verts, q, loop_off=None, threads=None) -> np.ndarray:
    """FT_A(Q) of the region bounded by CCW loops (Eq. 6 summed over segments)."""
    v, off = _loops(verts, loop_off)
    q = _f64(q, 2)
    out = np.empty((q.shape[0], 2))
    _load().orc_ft2d(_ptr(v, _dp), _ptr(off, _i64p), off.size - 1, _ptr(q, _dp), q.shape[0],
                     _ptr(out, _dp), _threads(threads))
    return _complex(out)


def seg_terms2d(verts, qxy, loop_off=None) -> np.ndarray:
    """The individual segment terms of Eq. 4/6 at one Q (their sum is FT_A)."""
    v, off = _loops(verts, loop_off)
    out = np.empty((v.shape[0], 2))
    _load().orc_seg_terms2d(_ptr(v, _dp), _ptr(off, _i64p), off.size - 1, float(qxy[0]),
                            float(qxy[1]), _ptr(out, _dp))
    return _complex(out)


def ft2d_batched(verts, poly_off, q, q_off=None, threads=None) -> np.ndarray:
    """One FT_A per polygon; shared Q (q_off None, result [n_polys, n_q]) or per-polygon Q (CSR)."""
    v = _f64(verts, 2)
    off = np.ascontiguousarray(np.asarray(poly_off, dtype=np.int64))
    q = _f64(q, 2)
    npoly = off.size - 1
    if q_off is None:
        out = np.empty((npoly * q.shape[0], 2))
        qo = None
    else:
        qo = np.ascontiguousarray(np.asarray(q_off, dtype=np.int64))
        out = np.empty((q.shape[0], 2))
    _load().orc_ft2d_batched(_ptr(v, _dp), _ptr(off, _i64p), npoly, _ptr(q, _dp),
                             None if qo is None else _ptr(qo, _i64p), q.shape[0], _ptr(out, _dp),
                             _threads(threads))
    r = _complex(out)
    return r.reshape(npoly, -1) if q_off is None else r


def _mesh(verts, faces):
    v = _f64(verts, 3)
    f = np.ascontiguousarray(np.asarray(faces, dtype=np.int32).reshape(-1, 3))
    return v, f


def ft3d(verts, faces, q, threads=None) -> np.ndarray:
    """FT_V(Q) of a closed outward-oriented triangle surface (sign-corrected Eq. 14)."""
    v, f = _mesh(verts, faces)
    q = _f64(q, 3)
    out = np.empty((q.shape[0], 2))
    rc = _load().orc_ft3d(_ptr(v, _dp), v.shape[0], _ptr(f, _i32p), f.shape[0], _ptr(q, _dp),
                          q.shape[0], _ptr(out, _dp), _threads(threads))
    if rc:
        raise ValueError("face index out of range")
    return _complex(out)


def ft3d_poly(verts, face_idx, face_off, q, threads=None) -> np.ndarray:
    """FT_V(Q) of a closed surface of planar polygon faces in CSR form (face m: the vertex
    indices face_idx[face_off[m]:face_off[m+1]], counter-clockwise seen from outside);
    Eq. 14 over each face's own edges with its Newell normal."""
    v = _f64(verts, 3)
    idx = np.ascontiguousarray(np.asarray(face_idx, dtype=np.int32).reshape(-1))
    off = np.ascontiguousarray(np.asarray(face_off, dtype=np.int64).reshape(-1))
    if off.size < 1 or off[-1] != idx.size:
        raise ValueError("face_off must end at len(face_idx)")
    q = _f64(q, 3)
    out = np.empty((q.shape[0], 2))
    rc = _load().orc_ft3d_poly(_ptr(v, _dp), v.shape[0], _ptr(idx, _i32p), _ptr(off, _i64p), off.size - 1,
                               _ptr(q, _dp), q.shape[0], _ptr(out, _dp), _threads(threads))
    if rc == 2:
        raise ValueError("face index out of range")
    if rc:
        raise ValueError("malformed face offsets (each face needs at least 3 vertices)")
    return _complex(out)


def face_terms3d(verts, faces, Q) -> np.ndarray:
    """The per-face terms I_m of Eq. 14 (sign-corrected) at one Q != 0."""
    v, f = _mesh(verts, faces)
    Q = _f64(Q).reshape(3)
    out = np.empty((f.shape[0], 2))
    rc = _load().orc_face_terms3d(_ptr(v, _dp), v.shape[0], _ptr(f, _i32p), f.shape[0],
                                  _ptr(Q, _dp), _ptr(out, _dp))
    if rc:
        raise ValueError("face index out of range")
    return _complex(out)


def grad2d(verts, q, g, loop_off=None, threads=None) -> np.ndarray:
    """dL/dverts [n_v, 2] for g_Q = dL/dRe F + i dL/dIm F (shape derivative)."""
    v, off = _loops(verts, loop_off)
    q = _f64(q, 2)
    g = np.ascontiguousarray(np.stack([np.real(g), np.imag(g)], axis=1).astype(np.float64))
    out = np.empty((v.shape[0], 2))
    _load().orc_grad2d(_ptr(v, _dp), _ptr(off, _i64p), off.size - 1, _ptr(q, _dp), q.shape[0],
                       _ptr(g, _dp), _ptr(out, _dp), _threads(threads))
    return out


def grad3d(verts, faces, q, g, vsel=None, threads=None) -> np.ndarray:
    """dL/dverts [n_v, 3] (or [len(vsel), 3]) for g_Q = dL/dRe F + i dL/dIm F (shape derivative)."""
    v, f = _mesh(verts, faces)
    q = _f64(q, 3)
    g = np.ascontiguousarray(np.stack([np.real(g), np.imag(g)], axis=1).astype(np.float64))
    if vsel is not None:
        sel = np.ascontiguousarray(np.asarray(vsel, dtype=np.int64))
        out = np.empty((sel.size, 3))
        selp, nsel = _ptr(sel, _i64p), sel.size
    else:
        out = np.empty((v.shape[0], 3))
        selp, nsel = None, 0
    rc = _load().orc_grad3d(_ptr(v, _dp), v.shape[0], _ptr(f, _i32p), f.shape[0], _ptr(q, _dp),
                            q.shape[0], _ptr(g, _dp), selp, nsel, _ptr(out, _dp), _threads(threads))
    if rc:
        raise ValueError("oracle grad3d failed (bad index or out of memory)")
    return out


def qgrad3d(verts, faces, q, g, threads=None) -> np.ndarray:
    """dL/dQ [n_q, 3] = Re(conj(g_Q) dF/dQ) for g_Q = dL/dRe F + i dL/dIm F.

    The derivative is taken from its definition, as the limit of difference quotients of ft3d:
    central differences at steps h and h/2 combined by Richardson extrapolation (error O(h^4)),
    h = 1e-3 / max|r| (max over the vertices), in FP64.
    """
    v, f = _mesh(verts, faces)
    q = _f64(q, 3)
    g = np.asarray(g).reshape(-1)
    h = 1e-3 / max(float(np.max(np.linalg.norm(v, axis=1))), 1e-300)
    steps = []
    for j in range(3):
        for hh in (h, 0.5 * h):
            e = np.zeros(3)
            e[j] = hh
            steps += [q + e, q - e]
    F = ft3d(v, f, np.concatenate(steps), threads=threads).reshape(len(steps), q.shape[0])
    out = np.empty((q.shape[0], 3))
    for j in range(3):
        d1 = (F[4 * j] - F[4 * j + 1]) / (2 * h)
        d2 = (F[4 * j + 2] - F[4 * j + 3]) / h
        dF = (4.0 * d2 - d1) / 3.0
        out[:, j] = np.real(np.conj(g) * dF)
    return out


def qgrad2d(verts, q, g, loop_off=None, threads=None) -> np.ndarray:
    """dL/dQ [n_q, 2] = Re(conj(g_Q) dF/dQ) of the 2D transform, g_Q = dL/dRe F + i dL/dIm F.

    As qgrad3d: the derivative from its definition, central differences of ft2d at steps h and h/2
    combined by Richardson extrapolation (error O(h^4)), h = 1e-3 / max|r|, in FP64.
    """
    v, _ = _loops(verts, loop_off)
    q = _f64(q, 2)
    g = np.asarray(g).reshape(-1)
    h = 1e-3 / max(float(np.max(np.linalg.norm(v, axis=1))), 1e-300)
    steps = []
    for j in range(2):
        for hh in (h, 0.5 * h):
            e = np.zeros(2)
            e[j] = hh
            steps += [q + e, q - e]
    F = ft2d(verts, np.concatenate(steps), loop_off, threads=threads).reshape(len(steps), q.shape[0])
    out = np.empty((q.shape[0], 2))
    for j in range(2):
        d1 = (F[4 * j] - F[4 * j + 1]) / (2 * h)
        d2 = (F[4 * j + 2] - F[4 * j + 3]) / h
        out[:, j] = np.real(np.conj(g) * (4.0 * d2 - d1) / 3.0)
    return out


def _voxel_centres(occ, d):
    """Centres of the occupied cubes of side d on the grid centred on the origin: cube (i, j, k)
    spans [(i - n_x/2) d, (i + 1 - n_x/2) d] x ... (the layout of synth.voxel_surface)."""
    occ = np.asarray(occ, dtype=bool)
    n = np.array(occ.shape, dtype=np.float64)
    return (np.argwhere(occ).astype(np.float64) + 0.5 - 0.5 * n) * d


def ft3d_voxels(occ, d, q) -> np.ndarray:
    """FT of the solid union of the occupied cubes (the voxelised shape of Sec. 4.3), by its plain
    definition: the sum over the cubes of the integral of exp(iQ.r) over each, i.e. the box closed
    form of Sec. 4.2 for a = b = c = d about the cube's centre c_v,
    exp(iQ.c_v) prod_k d sin(Q_k d/2)/(Q_k d/2)."""
    c = _voxel_centres(occ, d)
    q = _f64(q, 3)
    u = 0.5 * d * q
    with np.errstate(invalid="ignore", divide="ignore"):
        s = np.where(u == 0.0, 1.0, np.sin(u) / np.where(u == 0.0, 1.0, u))
    box = d ** 3 * np.prod(s, axis=1)
    return box * np.exp(1j * (q @ c.T)).sum(axis=1)


def ft3d_voxel_points(occ, d, q) -> np.ndarray:
    """The gridded transform of the same voxels: each occupied cube taken as a point of weight d^3
    at its centre, d^3 sum_v exp(iQ.c_v) -- what a direct sum over the voxel grid (or a DFT of the
    occupancy) gives.  Shifting one component of Q by 2 pi / d multiplies every term by the same
phase (-1 when the grid has an even number of cubes along that axis), so |F| repeats with that
period: the replica of the Q = 0 peak is the gridding artefact."""
    c = _voxel_centres(occ, d)
    q = _f64(q, 3)
    return d ** 3 * np.exp(1j * (q @ c.T)).sum(axis=1)


def max_threads() -> int:
    return int(_load().orc_max_threads())
