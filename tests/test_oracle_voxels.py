"""Voxelised shapes (Sec. 4.3 compares the sphere with its voxelisation).

* ``oracle.ft3d_voxels`` (the solid union of cubes, by the box closed form per cube) is pinned to
  Sec. 4.2's prism formula (Eq. 19) for one cube, to the volume at Q = 0 and to additivity, and
  against the oracle's polygon-face transform of the voxels' boundary (many coplanar faces and Q
  along their normals exercise every limit branch).
* ``oracle.ft3d_voxel_points`` (each cube as a point at its centre: the gridded transform) is pinned
  to its (anti)periodicity: on a grid of even size every centre is a half-integer multiple of d, so a
  shift of Q by 2 pi / d along an axis flips the sign, and F(2 pi / d, 0, 0) = -V; and to the exact
  relation with the solid cubes: one cube's integral is the point term times
  prod_k sin(Q_k d/2)/(Q_k d/2).
"""
import numpy as np

import oracle
from paper_2104_08309_gb300 import synth


def _prism(q, a, b, c):
    """Eq. 19: the box [0,a]x[0,b]x[0,c] at Q with no zero component."""
    qx, qy, qz = q[:, 0], q[:, 1], q[:, 2]
    return (np.exp(1j * qx * a) - 1) * (np.exp(1j * qy * b) - 1) * (np.exp(1j * qz * c) - 1) / (1j ** 3 * qx * qy * qz)


def test_one_cube_is_the_prism_closed_form(rng):
    d = 0.3
    occ = np.zeros((2, 2, 2), bool)
    occ[1, 1, 1] = True                                  # the cube [0, d]^3
    q = rng.uniform(-40, 40, (64, 3))
    assert np.max(np.abs(oracle.ft3d_voxels(occ, d, q) - _prism(q, d, d, d))) < 1e-14
    assert abs(oracle.ft3d_voxels(occ, d, [[0, 0, 0]])[0] - d ** 3) < 1e-17


def test_voxel_sum_is_additive_and_gives_the_volume(rng):
    d = 0.2
    occ = synth.voxel_ball(10, 1.0, d)
    half = occ.copy()
    half[:5] = False
    q = np.concatenate([[[0, 0, 0]], rng.uniform(-60, 60, (40, 3))])
    F = oracle.ft3d_voxels(occ, d, q)
    assert abs(F[0] - occ.sum() * d ** 3) < 1e-14
    assert np.max(np.abs(F - oracle.ft3d_voxels(half, d, q) - oracle.ft3d_voxels(occ & ~half, d, q))) < 1e-13


def test_voxel_ball_boundary_equals_voxel_sum(rng):
    d = 0.25
    occ = synth.voxel_ball(12, 1.3, d)
    assert 0 < occ.sum() < occ.size
    v, idx, off = synth.voxel_surface(occ, d)
    q = np.concatenate([[[0, 0, 0], [2.0, 0, 0], [0, 0, -5.0], [1e-5, 0, 0]], rng.uniform(-30, 30, (120, 3))])
    got = oracle.ft3d_poly(v, idx, off, q)
    ref = oracle.ft3d_voxels(occ, d, q)
    vol = occ.sum() * d ** 3
    assert abs(got[0] - vol) < 1e-12 * vol
    assert np.max(np.abs(got - ref)) < 1e-11 * vol


def test_gridded_transform_period_and_replica(rng):
    d = 0.2
    occ = synth.voxel_ball(10, 1.0, d)
    V = occ.sum() * d ** 3
    g = 2 * np.pi / d
    q = rng.uniform(-20, 20, (30, 3))
    P = oracle.ft3d_voxel_points(occ, d, q)
    for e in np.eye(3):
        assert np.max(np.abs(oracle.ft3d_voxel_points(occ, d, q + g * e) + P)) < 1e-11
    # 10 cubes per axis: every centre at a half-integer multiple of d, so exp(i 2 pi x / d) = -1
    assert abs(oracle.ft3d_voxel_points(occ, d, [[g, 0, 0]])[0] + V) < 1e-12
    # the solid cubes: the point term times the product of sincs, exactly
    s = np.prod(np.sinc(0.5 * d * q / np.pi), axis=1)
    assert np.max(np.abs(oracle.ft3d_voxels(occ, d, q) - s * P)) < 1e-13
