"""GPU parity of pft3d_polymesh (closed surfaces of planar polygon faces, CSR) through the C ABI:
against the oracle's polygon form of Eq. 14, bitwise against pft3d_mesh on the same fan
triangles, and at full size against the 2D path through the extrusion identity.

Tolerances relative to F(0) = volume: FP32 path 1e-5, FP64 path 1e-12.
"""
import numpy as np
import pytest

import oracle
from paper_2104_08309_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08309_gb300 import build as pbuild
    pbuild.build()
    return torch, torch.device("cuda:0")


def _c(out):
    a = out.detach().cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def _run(td, v, idx, off, q, **opts):
    torch, dev = td
    import paper_2104_08309_gb300 as pft
    return _c(pft.pft3d_polymesh(torch.from_numpy(v).to(dev), torch.from_numpy(idx).to(dev),
                                 torch.from_numpy(off).to(dev), torch.from_numpy(np.asarray(q, np.float64)).to(dev),
                                 options=opts, check_status=True))


def _halving(idx, off):
    """The library's split of each face, built on the host: the chain p_i .. p_j closed by its
    diagonal is the triangle (p_i, p_m, p_j), m = (i + j) // 2, then the two halves, pre-order."""
    tris = []

    def rec(f, i, j):
        if j - i < 2:
            return
        m = (i + j) // 2
        tris.append([f[i], f[m], f[j]])
        rec(f, i, m)
        rec(f, m, j)

    for m in range(off.size - 1):
        f = idx[off[m]:off[m + 1]]
        rec(f, 0, f.size - 1)
    return np.array(tris, dtype=np.int32)


def _shapes():
    yield "box", synth.box_quads(1.25, 0.75, 1.875)
    yield "hexagon_prism", synth.extruded_polygon(synth.regular_polygon(6, 1.0).astype(np.float32), 0.75)
    yield "star_prism", synth.extruded_polygon(synth.star_polygon(200, seed=4).astype(np.float32), 1.5, z0=-0.5)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_polymesh_vs_oracle(torch_dev, prec, rng):
    q = np.concatenate([[[0, 0, 0], [1e-6, 0, 0], [0, 0, 3.0], [0, 0, -12.0], [2.0, 0, 0], [0.05, 0.02, -0.01]],
                        rng.uniform(-30, 30, (1500, 3))])
    for name, (v, idx, off) in _shapes():
        ref = oracle.ft3d_poly(v, idx, off, q)
        got = _run(torch_dev, v, idx, off, q, precision=prec)
        assert np.max(np.abs(got - ref)) / abs(ref[0]) < TOL[prec], (name, prec)


def test_polymesh_equals_mesh_on_its_triangles(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, idx, off = synth.extruded_polygon(synth.star_polygon(300, seed=7).astype(np.float32), 1.25)
    q = rng.uniform(-40, 40, (4000, 3))
    a = _run(torch_dev, v, idx, off, q)
    b = _c(pft.pft3d_mesh(torch.from_numpy(v).to(dev), torch.from_numpy(_halving(idx, off)).to(dev),
                          torch.from_numpy(q).to(dev), check_status=True))
    assert np.array_equal(a, b)


def test_malformed_offsets_are_reported(torch_dev):
    """A face with 2 vertices: the call runs, the device status reports malformed offsets."""
    torch, dev = torch_dev
    import ctypes
    import paper_2104_08309_gb300 as pft
    v, idx, _ = synth.box_quads(1.0, 1.0, 1.0)
    lib = pft.load()
    o = pft.make_options(None)
    for off, want in ((np.array([0, 2, 8, 12, 16, 20, 24]), 8), (np.array([0, 4, 8, 12, 16, 20, 24]), 0),
                      (np.array([1, 4, 8, 12, 16, 20, 24]), 8)):
        vd, idd, od = (torch.from_numpy(a).to(dev) for a in (v, idx, off.astype(np.int64)))
        q = torch.ones(5, 3, dtype=torch.float64, device=dev)
        nb = lib.pft3d_polymesh_workspace_size(v.shape[0], idx.size, off.size - 1, 5, ctypes.byref(o))
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        out = torch.empty(5, 2, dtype=torch.float64, device=dev)
        rc = lib.pft3d_polymesh(vd.data_ptr(), v.shape[0], idd.data_ptr(), idx.size, od.data_ptr(), off.size - 1,
                                q.data_ptr(), 5, out.data_ptr(), ws.data_ptr(), nb, ctypes.byref(o), None)
        assert rc == 0
        assert lib.pft_status(ws.data_ptr(), None) == want, off
    # fewer than 3 indices per face: refused before any device work
    assert lib.pft3d_polymesh(vd.data_ptr(), v.shape[0], idd.data_ptr(), 17, od.data_ptr(), 6, q.data_ptr(), 5,
                              out.data_ptr(), ws.data_ptr(), nb, ctypes.byref(o), None) == 1


def test_large_star_prism_extrusion_identity(torch_dev):
    """A 65,536-vertex non-convex star extruded (two 65,536-gon caps, 65,536 side quads: 262,140
    triangles) on a 64^3 grid: against the 2D path times (e^{iQz h} - 1)/(iQz) on every Q, and
    against the oracle on sampled Q."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    star = synth.star_polygon(65536, seed=11).astype(np.float32)
    h = 0.75
    v, idx, off = synth.extruded_polygon(star, h)
    q = synth.q_grid_3d(64, 30.0)
    got = _run(torch_dev, v, idx, off, q)
    q2 = np.unique(q[:, :2], axis=0)
    f2 = _c(pft.pft2d_polygons(torch.from_numpy(star).to(dev), torch.from_numpy(q2).to(dev), check_status=True))
    lookup = {tuple(k): val for k, val in zip(q2, f2)}
    x = 0.5 * q[:, 2] * h
    e = h * np.sinc(x / np.pi) * np.exp(1j * x)
    ref2 = np.array([lookup[(a, b)] for a, b in q[:, :2]]) * e
    vol = abs(got[np.flatnonzero(np.all(q == 0, axis=1))[0]])
    # two FP32 paths, each within 1e-5; the side quadrilaterals here are 0.75 x 1e-4 (aspect ~7,500),
    # where the edge sum of a sliver triangle keeps fewer digits (measured 1.7e-5 on a GB300)
    assert np.max(np.abs(got - ref2)) / vol < 3e-5
    rng = np.random.default_rng(12)
    sel = rng.choice(q.shape[0], 256, replace=False)
    ref = oracle.ft3d_poly(v, idx, off, q[sel])
    assert np.max(np.abs(got[sel] - ref)) / vol < TOL["fp32"]


def test_polymesh_backward(torch_dev, rng):
    """Vertex gradients of the polygon-face path: against the oracle's shape-derivative gradient of
    the same triangle split (1e-4 of max|grad|), bitwise against pft3d_mesh_backward on those
    triangles, and through the autograd wrapper."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, idx, off = synth.extruded_polygon(synth.star_polygon(120, seed=5).astype(np.float32), 1.25, z0=-0.5)
    q = np.concatenate([[[0, 0, 0], [0, 0, 2.0], [1e-4, 0, 2e-4]], rng.uniform(-20, 20, (1500, 3))])
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    gd = torch.from_numpy(np.ascontiguousarray(np.stack([g.real, g.imag], axis=1))).to(dev)
    vd, idd, od, qd = (torch.from_numpy(a).to(dev) for a in (v, idx, off, q))
    got = pft.pft3d_polymesh_backward(vd, idd, od, qd, gd, check_status=True).cpu().numpy()
    tris = _halving(idx, off)
    ref = oracle.grad3d(v, tris, q, g)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-4
    same = pft.pft3d_mesh_backward(vd, torch.from_numpy(tris).to(dev), qd, gd, check_status=True).cpu().numpy()
    assert np.array_equal(got, same)
    # autograd: L = sum |F|^2 w  ->  g = 2 w F
    vt = vd.clone().requires_grad_(True)
    w = torch.rand(q.shape[0], dtype=torch.float64, device=dev)
    F = pft.ft3d_poly(vt, idd, od, qd)
    (w * F.abs() ** 2).sum().backward()
    Fn = F.detach().cpu().numpy()
    ref2 = oracle.grad3d(v, tris, q, 2.0 * w.cpu().numpy() * Fn)
    assert np.max(np.abs(vt.grad.cpu().numpy() - ref2)) / np.max(np.abs(ref2)) < 1e-4


def test_polymesh_empty_and_single_face_types(torch_dev, rng):
    """No faces: zeros.  Triangles given as 3-vertex polygon faces: the triangle path, bitwise."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    q = rng.uniform(-10, 10, (200, 3))
    v = np.zeros((3, 3), np.float32)
    out = _run(torch_dev, v, np.zeros(0, np.int32), np.zeros(1, np.int64), q)
    assert np.all(out == 0)
    vi, fi = synth.icosphere(2)
    a = _run(torch_dev, vi, fi.reshape(-1), np.arange(0, 3 * fi.shape[0] + 1, 3, dtype=np.int64), q)
    b = _c(pft.pft3d_mesh(torch.from_numpy(vi).to(dev), torch.from_numpy(fi).to(dev), torch.from_numpy(q).to(dev)))
    assert np.array_equal(a, b)


def test_voxelised_ball_surface(torch_dev, rng):
    """The boundary of a voxelised ball (quadrilaterals on a cubic grid, many coplanar, Q along the
    face normals included) against the plain sum over its cubes of the box closed form."""
    d = 1.0 / 16.0
    occ = synth.voxel_ball(48, 1.3, d)
    v, idx, off = synth.voxel_surface(occ, d)
    q = np.concatenate([[[0, 0, 0], [8.0, 0, 0], [0, 0, -40.0], [0, 3.0, 0]], rng.uniform(-60, 60, (800, 3))])
    got = _run(torch_dev, v, idx, off, q)
    n = np.array(occ.shape)
    r = (np.argwhere(occ) - 0.5 * n) * d
    ref = np.empty(q.shape[0], dtype=complex)
    for i, Q in enumerate(q):
        box = np.prod([d * np.sinc(0.5 * Q[c] * d / np.pi) * np.exp(0.5j * Q[c] * d) for c in range(3)])
        ref[i] = box * np.sum(np.exp(1j * (r @ Q)))
    vol = occ.sum() * d ** 3
    assert np.max(np.abs(got - ref)) / vol < TOL["fp32"]
