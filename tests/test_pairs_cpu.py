"""The host pairing of triangles for the face_pairs option (pft3d_pair_faces; no GPU): the output is
the same surface, its leading pairs share their first edge in opposite directions, and faces that
cannot pair (an edge of three faces, two faces running an edge the same way) stay unpaired."""
import numpy as np
import pytest

from paper_2104_08309_gb300 import synth


def _pair(f):
    import paper_2104_08309_gb300 as pft
    return pft.pair_faces(f)


def _canon(f):
    """Each triangle as its rotation starting at the smallest index (orientation kept)."""
    out = []
    for t in np.asarray(f):
        k = int(np.argmin(t))
        out.append(tuple(int(t[(k + j) % 3]) for j in range(3)))
    return sorted(out)


@pytest.mark.parametrize("level", [0, 2, 4])
def test_icosphere_pairs_share_first_edges(level):
    _, f = synth.icosphere(level)
    out, n = _pair(f)
    assert _canon(out) == _canon(f)                          # the same oriented triangles
    assert n >= 0.9 * (f.shape[0] // 2)
    a, b = out[0:2 * n:2], out[1:2 * n:2]
    assert np.array_equal(a[:, 0], b[:, 1]) and np.array_equal(a[:, 1], b[:, 0])
    # the unpaired faces follow in input order, unrotated
    rest = out[2 * n:]
    pos = {tuple(t): i for i, t in enumerate(f.tolist())}
    idx = [pos[tuple(t)] for t in rest.tolist()]
    assert idx == sorted(idx)


def test_unpairable_faces_stay_unpaired():
    # edge (0, 1) held by three faces: none pairs across it; faces 3 and 4 run (5, 6) the same way
    f = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4], [5, 6, 7], [5, 6, 8]], np.int32)
    out, n = _pair(f)
    assert n == 0
    assert np.array_equal(out, f)
    # a proper pair among them is found: (2, 9, 1) holds (1, 2) reversed against (0, 1, 2)
    g = np.concatenate([f, [[2, 1, 9]]]).astype(np.int32)
    out, n = _pair(g)
    assert n == 1
    assert tuple(out[0]) == (1, 2, 0) and tuple(out[1]) == (2, 1, 9)


def test_pairing_arguments_checked():
    import ctypes
    from paper_2104_08309_gb300 import _capi
    lib = _capi.load()
    f = np.array([[0, 1, 2]], np.int32)
    out = np.empty_like(f)
    n = ctypes.c_int64(0)
    assert lib.pft3d_pair_faces(f.ctypes.data, -1, out.ctypes.data, ctypes.byref(n)) == 1
    assert lib.pft3d_pair_faces(f.ctypes.data, 1, f.ctypes.data, ctypes.byref(n)) == 1       # aliasing
    bad = np.array([[0, -1, 2]], np.int32)
    assert lib.pft3d_pair_faces(bad.ctypes.data, 1, out.ctypes.data, ctypes.byref(n)) == 1
    assert lib.pft3d_pair_faces(None, 0, None, ctypes.byref(n)) == 0 and n.value == 0
