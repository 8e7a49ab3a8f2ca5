"""GPU Q-gradient of the 2D transform, dL/dQ = Re(conj(g) dF/dQ), through the C ABI, against the
oracle's Richardson differences of the FP64 transform (oracle.qgrad2d).  Tolerance: 1e-5 of
max|g| A max|r| (a bound on |g dF/dQ|: |dF/dQ| <= int |r| dA), the FP32 path's budget; Q = 0 and
small |Q| come from the FP64 series and are held to 1e-9 of it."""
import numpy as np
import pytest

import oracle
from paper_2104_08309_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08309_gb300 import build as pbuild
    pbuild.build()
    return torch, torch.device("cuda:0")


def _scale(v, g, off=None):
    area = abs(oracle.ft2d(v, [[0.0, 0.0]], off)[0])
    return np.max(np.abs(g)) * area * float(np.max(np.linalg.norm(v.astype(np.float64), axis=1)))


def _qgrad(td, v, q, g, off=None):
    torch, dev = td
    import paper_2104_08309_gb300 as pft
    gd = torch.from_numpy(np.ascontiguousarray(np.stack([g.real, g.imag], axis=1))).to(dev)
    od = None if off is None else torch.from_numpy(off).to(dev)
    return pft.pft2d_polygons_qgrad(torch.from_numpy(v).to(dev),
                                    torch.from_numpy(np.ascontiguousarray(q, np.float64)).to(dev), gd, od,
                                    check_status=True).cpu().numpy()


def test_qgrad2d_vs_oracle_with_a_hole(torch_dev, rng):
    outer = synth.star_polygon(300, seed=4)
    hole = (0.3 * synth.star_polygon(31, seed=6))[::-1]
    v = (np.concatenate([outer, hole]) + np.float32(0.3)).astype(np.float32)   # off-centre: e^{iQ.c} matters
    off = np.array([0, 300, 331])
    q = np.concatenate([[[0.0, 0.0], [1e-4, 2e-4], [0.0, 0.05], [6.0, 0.0]],
                        rng.uniform(-40, 40, (3000, 2))]).astype(np.float32).astype(np.float64)
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    got = _qgrad(torch_dev, v, q, g, off)
    ref = oracle.qgrad2d(v, q, g, loop_off=off)
    s = _scale(v, g, off)
    assert np.max(np.abs(got - ref)) < 1e-5 * s
    assert np.max(np.abs(got[:3] - ref[:3])) < 1e-9 * s


def test_qgrad2d_c1_full_grid(torch_dev, rng):
    """The 64-vertex star on the full 128 x 128 grid over [-40, 40)^2 (Q = 0 included)."""
    w = synth.workload_c1()
    g = rng.normal(size=w.q.shape[0]) + 1j * rng.normal(size=w.q.shape[0])
    got = _qgrad(torch_dev, w.verts, w.q, g)
    ref = oracle.qgrad2d(w.verts, w.q, g)
    assert np.max(np.abs(got - ref)) < 1e-5 * _scale(w.verts, g)


def test_qgrad2d_many_small_q(torch_dev, rng):
    """Hundreds of Q with |Q| R < 0.25 (the FP64 series path, segments split into chunks per Q)."""
    v = (synth.star_polygon(500, seed=9) + np.float32(0.2)).astype(np.float32)
    r = float(np.max(np.linalg.norm(v.astype(np.float64), axis=1)))
    q = (rng.uniform(-1, 1, (400, 2)) * 0.1 / r).astype(np.float32).astype(np.float64)
    q[0] = 0.0
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    got = _qgrad(torch_dev, v, q, g)
    ref = oracle.qgrad2d(v, q, g)
    assert np.max(np.abs(got - ref)) < 1e-9 * _scale(v, g)


def test_autograd_ft2d_q_and_verts(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v = synth.star_polygon(90, seed=3)
    q = rng.uniform(-20, 20, (600, 2)).astype(np.float32).astype(np.float64)
    qt = torch.from_numpy(q).to(dev).requires_grad_(True)
    vt = torch.from_numpy(v).to(dev).requires_grad_(True)
    F = pft.ft2d(vt, qt)
    w = torch.rand(q.shape[0], dtype=torch.float64, device=dev)
    (w * F.abs() ** 2).sum().backward()
    Fn = F.detach().cpu().numpy()
    g = 2.0 * w.cpu().numpy() * Fn
    assert np.max(np.abs(qt.grad.cpu().numpy() - oracle.qgrad2d(v, q, g))) < 1e-5 * _scale(v, g)
    ref_v = oracle.grad2d(v, q, g)
    assert np.max(np.abs(vt.grad.cpu().numpy() - ref_v)) / np.max(np.abs(ref_v)) < 1e-4


def test_qgrad2d_bad_offsets_reported(torch_dev):
    torch, dev = torch_dev
    import ctypes
    from paper_2104_08309_gb300 import _capi
    lib = _capi.load()
    v = synth.star_polygon(40, seed=2)
    bad = np.array([0, 30, 20, 40], np.int64)             # decreasing offsets
    q = torch.from_numpy(np.array([[1.0, 2.0], [3.0, -1.0]])).to(dev)
    g = torch.ones(2, 2, dtype=torch.float64, device=dev)
    out = torch.empty(2, 2, dtype=torch.float64, device=dev)
    o = _capi.Options()
    nb = lib.pft2d_qgrad_workspace_size(40, 3, 2, ctypes.byref(o))
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    vd, bd = torch.from_numpy(v).to(dev), torch.from_numpy(bad).to(dev)
    rc = lib.pft2d_polygons_qgrad(vd.data_ptr(), 40, bd.data_ptr(), 3, q.data_ptr(), 2, g.data_ptr(),
                                  out.data_ptr(), ws.data_ptr(), nb, ctypes.byref(o), None)
    assert rc == 0
    assert lib.pft_status(ws.data_ptr(), None) == 8


def test_qgrad2d_empty_inputs(torch_dev):
    """No Q points: nothing to write; no vertices: dL/dQ = 0 for every Q."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v = torch.from_numpy(synth.star_polygon(12, seed=3)).to(dev)
    q0 = torch.empty(0, 2, dtype=torch.float64, device=dev)
    assert pft.pft2d_polygons_qgrad(v, q0, torch.empty(0, 2, dtype=torch.float64, device=dev)).shape == (0, 2)
    q = torch.from_numpy(np.array([[1.0, 2.0], [0.0, 0.0]])).to(dev)
    g = torch.ones(2, 2, dtype=torch.float64, device=dev)
    ve = torch.empty(0, 2, dtype=torch.float32, device=dev)
    out = pft.pft2d_polygons_qgrad(ve, q, g, torch.tensor([0, 0], dtype=torch.int64, device=dev),
                                   out=torch.full((2, 2), float("nan"), dtype=torch.float64, device=dev))
    assert torch.equal(out, torch.zeros_like(out))
