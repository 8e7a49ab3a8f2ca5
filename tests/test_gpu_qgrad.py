"""GPU Q-gradient dL/dQ = Re(conj(g) dF/dQ) (3D triangles) through the C ABI, against the oracle's
differences of the FP64 transform.  Tolerance: 1e-5 of max|g| V max|r| (a bound on |g dF/dQ|),
the FP32 path's budget."""
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


def _scale(v, f, g):
    vol = abs(oracle.ft3d(v, f, [[0.0, 0.0, 0.0]])[0])
    return np.max(np.abs(g)) * vol * float(np.max(np.linalg.norm(v.astype(np.float64), axis=1)))


def _qgrad(td, v, f, q, g, **opts):
    torch, dev = td
    import paper_2104_08309_gb300 as pft
    gd = torch.from_numpy(np.ascontiguousarray(np.stack([g.real, g.imag], axis=1))).to(dev)
    return pft.pft3d_mesh_qgrad(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev),
                                torch.from_numpy(np.ascontiguousarray(q, np.float64)).to(dev), gd,
                                options=opts, check_status=True).cpu().numpy()


@pytest.mark.parametrize("tau", [1.0, 3.0, 6.0])
def test_qgrad_vs_oracle(torch_dev, rng, tau):
    v, f = synth.perturbed_icosphere(3, seed=14, amp=0.08)
    v = (v + np.array([0.125, -0.25, 0.1875], np.float32)).astype(np.float32)   # off-centre: e^{iQ.c} matters
    q = np.concatenate([[[0, 0, 0], [1e-4, 0, 2e-4], [0, 0.05, 0], [0, 0, 4.0], [6.0, 0, 0]],
                        rng.uniform(-25, 25, (1200, 3))]).astype(np.float32).astype(np.float64)
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    got = _qgrad(torch_dev, v, f, q, g, face_series_tau=tau)
    ref = oracle.qgrad3d(v, f, q, g)
    assert np.max(np.abs(got - ref)) < 1e-5 * _scale(v, f, g)
    # Q = 0 and small |Q| come from the FP64 series: far tighter
    assert np.max(np.abs(got[:3] - ref[:3])) < 1e-9 * _scale(v, f, g)


def test_autograd_q(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f = synth.perturbed_icosphere(2, seed=3, amp=0.1)
    q = rng.uniform(-10, 10, (500, 3)).astype(np.float32).astype(np.float64)
    qt = torch.from_numpy(q).to(dev).requires_grad_(True)
    vt = torch.from_numpy(v).to(dev).requires_grad_(True)
    F = pft.ft3d(vt, torch.from_numpy(f).to(dev), qt)
    w = torch.rand(q.shape[0], dtype=torch.float64, device=dev)
    (w * F.abs() ** 2).sum().backward()
    Fn = F.detach().cpu().numpy()
    g = 2.0 * w.cpu().numpy() * Fn
    ref_q = oracle.qgrad3d(v, f, q, g)
    assert np.max(np.abs(qt.grad.cpu().numpy() - ref_q)) < 1e-5 * _scale(v, f, g)
    ref_v = oracle.grad3d(v, f, q, g)
    assert np.max(np.abs(vt.grad.cpu().numpy() - ref_v)) / np.max(np.abs(ref_v)) < 1e-4


def test_c4_size_sampled(torch_dev):
    """16 icospheres (81,920 faces) on the 32^3 grid with a seeded g: 48 sampled Q against the oracle."""
    w = synth.workload_c4()
    rng = np.random.default_rng(45)
    g = rng.normal(size=w.q.shape[0]) + 1j * rng.normal(size=w.q.shape[0])
    got = _qgrad(torch_dev, w.verts, w.faces, w.q, g)
    sel = np.sort(rng.choice(w.q.shape[0], 48, replace=False))
    ref = oracle.qgrad3d(w.verts, w.faces, w.q[sel], g[sel])
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got[sel] - ref)) < 1e-5 * _scale(w.verts, w.faces, g)


def test_many_small_q(torch_dev, rng):
    """Hundreds of Q with |Q| R < 0.25 (the FP64 series path, faces split into chunks per Q)."""
    v, f = synth.perturbed_icosphere(3, seed=15, amp=0.05)
    r = float(np.max(np.linalg.norm(v.astype(np.float64), axis=1)))
    q = (rng.uniform(-1, 1, (400, 3)) * 0.12 / r).astype(np.float32).astype(np.float64)
    q[0] = 0.0
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    got = _qgrad(torch_dev, v, f, q, g)
    ref = oracle.qgrad3d(v, f, q, g)
    assert np.max(np.abs(got - ref)) < 1e-9 * _scale(v, f, g)


def test_tiny_q_beside_large_q(torch_dev, rng):
    """A Q of size ~1e-25 as the first lane of every warp (one Q per thread), the other 31 lanes at
    |Q| up to 25: the tiny Q's P can round to -0 or a negative subnormal, and must not pull its
    warp onto the k <= 7 series.  Every entry against the oracle."""
    v, f = synth.perturbed_icosphere(3, seed=16, amp=0.08)
    v = (v + np.array([0.125, -0.25, 0.1875], np.float32)).astype(np.float32)
    q = rng.uniform(-25, 25, (1024, 3))
    d = rng.normal(size=(32, 3))
    q[::32] = d * 1e-25
    q = q.astype(np.float32).astype(np.float64)
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    got = _qgrad(torch_dev, v, f, q, g)
    ref = oracle.qgrad3d(v, f, q, g)
    assert np.max(np.abs(got - ref)) < 1e-5 * _scale(v, f, g)
    assert np.max(np.abs(got[::32] - ref[::32])) < 1e-9 * _scale(v, f, g)


def test_far_from_the_origin(torch_dev, rng):
    """dL/dQ of a mesh about 2,800 units from the origin at Q that float32 cannot represent: the
    factors and the phase take the caller's Q."""
    v, f = synth.perturbed_icosphere(2, seed=14, amp=0.08)
    v = (v.astype(np.float64) + np.array([1500.0, -2200.0, 800.0])).astype(np.float32)
    q = np.concatenate([[[1e-5, 0, 2e-5], [0.3, -0.2, 0.1]], rng.uniform(-25, 25, (800, 3))])
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    got = _qgrad(torch_dev, v, f, q, g)
    ref = oracle.qgrad3d(v, f, q, g)
    assert np.max(np.abs(got - ref)) < 1e-5 * _scale(v, f, g)
