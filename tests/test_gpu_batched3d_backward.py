"""Batched 3D adjoint (vertex gradients of many closed meshes in one call) through the C ABI: mesh by
mesh against the oracle's shape-derivative gradient and against the single-mesh adjoint, on a shared
Q list and on per-mesh Q lists, through autograd, and with malformed offsets.  Tolerance: 1e-4 of
each mesh's max |gradient| (the FP32 adjoint's budget)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2104_08309_gb300 import synth

pytestmark = pytest.mark.gpu

GTOL = 1e-4


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08309_gb300 import build as pbuild
    pbuild.build()
    return torch, torch.device("cuda:0")


def _batch():
    # 6 meshes of 80 .. 1,280 faces (a 1,280-face mesh spans ten pair blocks of 128 faces)
    return synth.mesh_batch(6, seed=27, levels=(1, 2, 3))


def _pairs(z):
    return np.ascontiguousarray(np.stack([z.real, z.imag], axis=-1))


def _qmix(rng, n):
    return np.concatenate([[[0.0, 0.0, 0.0], [1e-4, 0.0, 2e-4], [0.0, 0.0, 3.0]], rng.uniform(-25, 25, (n - 3, 3))])


def test_shared_q_vs_oracle_and_single_mesh_adjoint(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f, off = _batch()
    q = _qmix(rng, 700)
    n = off.size - 1
    g = rng.normal(size=(n, q.shape[0])) + 1j * rng.normal(size=(n, q.shape[0]))
    qd = torch.from_numpy(q).to(dev)
    got = pft.pft3d_meshes_batched_backward(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev), off, qd,
                                            torch.from_numpy(_pairs(g)).to(dev), check_status=True).cpu().numpy()
    for i in range(n):
        fi = f[off[i]:off[i + 1]]
        lo, hi = fi.min(), fi.max() + 1
        ref = oracle.grad3d(v[lo:hi], fi - lo, q, g[i])
        seg = got[lo:hi]
        assert np.max(np.abs(seg - ref)) / np.max(np.abs(ref)) < GTOL, i
        single = pft.pft3d_mesh_backward(torch.from_numpy(np.ascontiguousarray(v[lo:hi])).to(dev),
                                         torch.from_numpy(np.ascontiguousarray(fi - lo)).to(dev), qd,
                                         torch.from_numpy(_pairs(g[i])).to(dev)).cpu().numpy()
        assert np.max(np.abs(seg - single)) / np.max(np.abs(single)) < 1e-5, i


def test_per_mesh_q_lists_vs_oracle(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f, off = _batch()
    n = off.size - 1
    sizes = [200, 0, 450, 1, 129, 300][:n]
    qs = [_qmix(rng, s) if s >= 3 else rng.uniform(-20, 20, (s, 3)) for s in sizes]
    q = np.concatenate(qs)
    q_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    got = pft.pft3d_meshes_batched_backward(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev), off,
                                            torch.from_numpy(q).to(dev), torch.from_numpy(_pairs(g)).to(dev), q_off,
                                            check_status=True).cpu().numpy()
    for i in range(n):
        fi = f[off[i]:off[i + 1]]
        lo, hi = fi.min(), fi.max() + 1
        a, b = q_off[i], q_off[i + 1]
        if a == b:
            assert np.all(got[lo:hi] == 0.0), i
            continue
        ref = oracle.grad3d(v[lo:hi], fi - lo, q[a:b], g[a:b])
        assert np.max(np.abs(got[lo:hi] - ref)) / np.max(np.abs(ref)) < GTOL, i


def test_ft3d_batched_autograd(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f, off = _batch()
    q = _qmix(rng, 400)
    vt = torch.from_numpy(v).to(dev).requires_grad_(True)
    fd, qd = torch.from_numpy(f).to(dev), torch.from_numpy(q).to(dev)
    F = pft.ft3d_batched(vt, fd, off, qd)
    assert F.shape == (off.size - 1, q.shape[0]) and F.dtype == torch.complex128
    w = torch.rand(F.shape, dtype=torch.float64, device=dev)
    (w * F.abs() ** 2).sum().backward()
    g = (2.0 * w * F.detach()).cpu().numpy()
    direct = pft.pft3d_meshes_batched_backward(torch.from_numpy(v).to(dev), fd, off, qd,
                                               torch.from_numpy(_pairs(g)).to(dev)).cpu().numpy()
    assert np.array_equal(vt.grad.cpu().numpy(), direct)
    with pytest.raises(ValueError):
        pft.ft3d_batched(vt, fd, off, qd, options={"precision": "fp64"})


def test_bad_mesh_offsets_reported(torch_dev):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    lib = pft.load()
    v, f, off = _batch()
    bad = off.copy()
    bad[-1] -= 1                                       # the last mesh stops one face short
    n = off.size - 1
    q = torch.ones(8, 3, dtype=torch.float64, device=dev)
    g = torch.ones(n, 8, 2, dtype=torch.float64, device=dev)
    o = pft.make_options(None)
    nb = lib.pft3d_batched_backward_workspace_size(v.shape[0], f.shape[0], n, 8, 0, ctypes.byref(o))
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    out = torch.empty(v.shape[0], 3, dtype=torch.float32, device=dev)
    vd, fd, bd = (torch.from_numpy(a).to(dev) for a in (v, f, bad))
    rc = lib.pft3d_meshes_batched_backward(vd.data_ptr(), v.shape[0], fd.data_ptr(), f.shape[0], bd.data_ptr(), n,
                                           q.data_ptr(), None, 8, g.data_ptr(), out.data_ptr(), ws.data_ptr(), nb,
                                           ctypes.byref(o), None)
    assert rc == 0
    assert lib.pft_status(ws.data_ptr(), None) == 8


def test_empty_inputs(torch_dev):
    """No Q points, or no faces: every vertex gradient is 0."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f, off = _batch()
    vd, fd = torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev)
    n = off.size - 1
    q0 = torch.empty(0, 3, dtype=torch.float64, device=dev)
    g0 = torch.empty(n, 0, 2, dtype=torch.float64, device=dev)
    out = torch.full((v.shape[0], 3), float("nan"), dtype=torch.float32, device=dev)
    pft.pft3d_meshes_batched_backward(vd, fd, off, q0, g0, out=out, check_status=True)
    assert torch.equal(out, torch.zeros_like(out))
    q = torch.from_numpy(np.array([[1.0, 2.0, 0.5]])).to(dev)
    g = torch.ones(1, 1, 2, dtype=torch.float64, device=dev)
    out.fill_(float("nan"))
    pft.pft3d_meshes_batched_backward(vd, torch.empty(0, 3, dtype=torch.int32, device=dev), np.array([0, 0]), q, g,
                                      out=out)
    assert torch.equal(out, torch.zeros_like(out))
