"""A set of cubes (a voxelised ball) as a polygon mesh: the oracle's polygon-face transform of its
boundary against the plain sum over the cubes of the box closed form, prod_c (e^{iQ_c d} - 1)/(iQ_c)
times e^{iQ.r_v}.  Many coplanar faces and Q along the face normals exercise every limit branch."""
import numpy as np

import oracle
from paper_2104_08309_gb300 import synth


def voxel_ft(occ, d, q):
    n = np.array(occ.shape)
    r = (np.argwhere(occ) - 0.5 * n) * d
    out = np.empty(q.shape[0], dtype=complex)
    for i, Q in enumerate(q):
        box = np.prod([d * np.sinc(0.5 * Q[c] * d / np.pi) * np.exp(0.5j * Q[c] * d) for c in range(3)])
        out[i] = box * np.sum(np.exp(1j * (r @ Q)))
    return out


def test_voxel_ball_boundary_equals_voxel_sum(rng):
    d = 0.25
    occ = synth.voxel_ball(12, 1.3, d)
    assert 0 < occ.sum() < occ.size
    v, idx, off = synth.voxel_surface(occ, d)
    q = np.concatenate([[[0, 0, 0], [2.0, 0, 0], [0, 0, -5.0], [1e-5, 0, 0]], rng.uniform(-30, 30, (120, 3))])
    got = oracle.ft3d_poly(v, idx, off, q)
    ref = voxel_ft(occ, d, q)
    vol = occ.sum() * d ** 3
    assert abs(got[0] - vol) < 1e-12 * vol
    assert np.max(np.abs(got - ref)) < 1e-11 * vol
