"""Batched 2D adjoint (vertex gradients of many polygons, each with its own weights on a shared
Q set or on its own Q list) through the C ABI, polygon by polygon against the oracle's
shape-derivative gradient and the single-polygon adjoint.  Tolerance: 1e-4 of each polygon's max
|gradient|."""
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
    # pair blocks hold 256 segments (two per thread): 600 spans three, 257 ends one past a block,
    # 129 ends one past the first half of a block
    polys = [synth.star_polygon(3, seed=1), synth.star_polygon(600, seed=2, center=(0.5, -0.25)),
             synth.regular_polygon(17, 0.4), synth.star_polygon(129, seed=3, center=(-0.75, 0.5)),
             synth.star_polygon(40, seed=4), synth.star_polygon(257, seed=5, center=(0.25, 0.75))]
    off = np.concatenate([[0], np.cumsum([p.shape[0] for p in polys])]).astype(np.int64)
    return np.concatenate(polys).astype(np.float32), off


def _run(td, v, off, q, g):
    torch, dev = td
    import paper_2104_08309_gb300 as pft
    gd = np.ascontiguousarray(np.stack([g.real, g.imag], axis=-1))
    return pft.pft2d_polygons_batched_backward(torch.from_numpy(v).to(dev), torch.from_numpy(off).to(dev),
                                               torch.from_numpy(q).to(dev), torch.from_numpy(gd).to(dev),
                                               check_status=True).cpu().numpy()


def test_batched_backward_vs_oracle_and_single(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, off = _batch()
    q = np.concatenate([[[0.0, 0.0], [1e-4, 2e-4], [0.0, 0.05]], rng.uniform(-30, 30, (1500, 2))])
    g = rng.normal(size=(off.size - 1, q.shape[0])) + 1j * rng.normal(size=(off.size - 1, q.shape[0]))
    got = _run(torch_dev, v, off, q, g)
    for i in range(off.size - 1):
        vi = v[off[i]:off[i + 1]]
        ref = oracle.grad2d(vi, q, g[i])
        gi = got[off[i]:off[i + 1]]
        assert np.max(np.abs(gi - ref)) / np.max(np.abs(ref)) < GTOL, i
        single = pft.pft2d_polygons_backward(torch.from_numpy(vi).to(dev), torch.from_numpy(q).to(dev),
                                             torch.from_numpy(np.ascontiguousarray(np.stack([g[i].real, g[i].imag], 1))).to(dev),
                                             check_status=True).cpu().numpy()
        assert np.max(np.abs(gi - single)) / np.max(np.abs(ref)) < GTOL, i


def test_c3_batch_sampled(torch_dev):
    """4,096 polygons on the 64 x 64 grid with seeded weights: 8 sampled polygons against the oracle."""
    w = synth.workload_c3()
    rng = np.random.default_rng(46)
    n = w.poly_off.size - 1
    g = rng.normal(size=(n, w.q.shape[0])) + 1j * rng.normal(size=(n, w.q.shape[0]))
    got = _run(torch_dev, w.verts, w.poly_off, w.q, g)
    assert np.all(np.isfinite(got))
    for i in np.sort(rng.choice(n, 8, replace=False)):
        vi = w.verts[w.poly_off[i]:w.poly_off[i + 1]]
        ref = oracle.grad2d(vi, w.q, g[i])
        assert np.max(np.abs(got[w.poly_off[i]:w.poly_off[i + 1]] - ref)) / np.max(np.abs(ref)) < GTOL, i


def test_bad_offsets_reported(torch_dev):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, off = _batch()
    bad = off.copy()
    bad[-1] -= 1                                   # last offset short of n_verts
    lib = pft.load()
    o = pft.make_options(None)
    q = torch.ones(8, 2, dtype=torch.float64, device=dev)
    g = torch.ones(off.size - 1, 8, 2, dtype=torch.float64, device=dev)
    nb = lib.pft2d_batched_backward_workspace_size(v.shape[0], off.size - 1, 8, 0, ctypes.byref(o))
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    out = torch.empty(v.shape[0], 2, dtype=torch.float32, device=dev)
    vd, bd = torch.from_numpy(v).to(dev), torch.from_numpy(bad).to(dev)
    rc = lib.pft2d_polygons_batched_backward(vd.data_ptr(), v.shape[0], bd.data_ptr(), off.size - 1, q.data_ptr(),
                                             None, 8, g.data_ptr(), out.data_ptr(), ws.data_ptr(), nb,
                                             ctypes.byref(o), None)
    assert rc == 0
    assert lib.pft_status(ws.data_ptr(), None) == 8


def test_ft2d_batched_autograd(torch_dev, rng):
    """ft2d_batched under autograd: the vertex gradient of a linear loss equals the batched adjoint
    called directly (bitwise) and the oracle's gradient polygon by polygon."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, off = _batch()
    q = np.concatenate([[[0.0, 0.0]], rng.uniform(-25, 25, (700, 2))])
    w = rng.normal(size=(off.size - 1, q.shape[0], 2))
    vt = torch.from_numpy(v).to(dev).requires_grad_(True)
    qd = torch.from_numpy(q).to(dev)
    F = pft.ft2d_batched(vt, off, qd)
    assert F.shape == (off.size - 1, q.shape[0]) and F.dtype == torch.complex128
    wd = torch.from_numpy(w).to(dev)
    (F.real * wd[..., 0] + F.imag * wd[..., 1]).sum().backward()
    direct = pft.pft2d_polygons_batched_backward(torch.from_numpy(v).to(dev), off, qd, wd).cpu().numpy()
    got = vt.grad.cpu().numpy()
    assert np.array_equal(got, direct)
    g = w[..., 0] + 1j * w[..., 1]
    for i in range(off.size - 1):
        ref = oracle.grad2d(v[off[i]:off[i + 1]], q, g[i])
        assert np.max(np.abs(got[off[i]:off[i + 1]] - ref)) / np.max(np.abs(ref)) < GTOL, i


def test_ft2d_batched_refuses_fp64_gradient(torch_dev):
    """The batched adjoint has only an FP32 path: asking for a gradient of an FP64 forward raises
    instead of silently differentiating in FP32; without grad the FP64 forward runs."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, off = _batch()
    qd = torch.from_numpy(np.array([[0.0, 0.0], [1.5, -2.0]])).to(dev)
    vt = torch.from_numpy(v).to(dev).requires_grad_(True)
    with pytest.raises(ValueError):
        pft.ft2d_batched(vt, off, qd, options={"precision": "fp64"})
    F = pft.ft2d_batched(vt.detach(), off, qd, options={"precision": "fp64"})
    ref = oracle.ft2d_batched(v, off, qd.cpu().numpy())
    assert np.max(np.abs(F.cpu().numpy() - ref)) < 1e-12 * np.max(np.abs(ref))


def _per_polygon_q(rng, n_polys):
    """Each polygon its own Q list (sizes 0 .. 900, Q = 0 and a small |Q| in some), CSR."""
    sizes = [300, 0, 900, 1, 257, 129][:n_polys]
    qs = []
    for i, n in enumerate(sizes):
        qi = rng.uniform(-30, 30, (n, 2))
        if n > 2 and i % 2 == 0:
            qi[0] = 0.0
            qi[1] = [1e-4, -2e-4]
        qs.append(qi)
    q_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(qs), q_off


def test_per_polygon_q_sets_vs_oracle(torch_dev, rng):
    """q_off: polygon i on its own Q list; each polygon's gradient against the oracle's, and the
    call against the shared-Q call where every list is the same."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, off = _batch()
    q, q_off = _per_polygon_q(rng, off.size - 1)
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    gp = np.ascontiguousarray(np.stack([g.real, g.imag], axis=1))
    got = pft.pft2d_polygons_batched_backward(torch.from_numpy(v).to(dev), off, torch.from_numpy(q).to(dev),
                                              torch.from_numpy(gp).to(dev), q_off, check_status=True).cpu().numpy()
    for i in range(off.size - 1):
        a, b = q_off[i], q_off[i + 1]
        seg = got[off[i]:off[i + 1]]
        if a == b:
            assert np.all(seg == 0.0), i
            continue
        ref = oracle.grad2d(v[off[i]:off[i + 1]], q[a:b], g[a:b])
        assert np.max(np.abs(seg - ref)) / np.max(np.abs(ref)) < GTOL, i
    # the same Q list for every polygon: equal to the shared-Q call
    qs = rng.uniform(-20, 20, (200, 2))
    n = off.size - 1
    gs = rng.normal(size=(n, 200, 2))
    shared = pft.pft2d_polygons_batched_backward(torch.from_numpy(v).to(dev), off, torch.from_numpy(qs).to(dev),
                                                 torch.from_numpy(gs).to(dev)).cpu().numpy()
    lists = pft.pft2d_polygons_batched_backward(torch.from_numpy(v).to(dev), off,
                                                torch.from_numpy(np.tile(qs, (n, 1))).to(dev),
                                                torch.from_numpy(gs.reshape(-1, 2)).to(dev),
                                                np.arange(n + 1, dtype=np.int64) * 200).cpu().numpy()
    assert np.max(np.abs(lists - shared)) <= 1e-6 * np.max(np.abs(shared))


def test_ft2d_batched_autograd_per_polygon_q(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, off = _batch()
    q, q_off = _per_polygon_q(rng, off.size - 1)
    w = rng.normal(size=(q.shape[0], 2))
    vt = torch.from_numpy(v).to(dev).requires_grad_(True)
    F = pft.ft2d_batched(vt, off, torch.from_numpy(q).to(dev), q_off=q_off)
    assert F.shape == (q.shape[0],)
    wd = torch.from_numpy(w).to(dev)
    (F.real * wd[:, 0] + F.imag * wd[:, 1]).sum().backward()
    direct = pft.pft2d_polygons_batched_backward(torch.from_numpy(v).to(dev), off, torch.from_numpy(q).to(dev), wd,
                                                 q_off).cpu().numpy()
    assert np.array_equal(vt.grad.cpu().numpy(), direct)


def test_malformed_q_off_reported(torch_dev):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    lib = pft.load()
    v, off = _batch()
    n = off.size - 1
    q_off = np.arange(n + 1, dtype=np.int64) * 2
    q_off[3] = 1                                           # decreasing
    q = torch.ones(2 * n, 2, dtype=torch.float64, device=dev)
    g = torch.ones(2 * n, 2, dtype=torch.float64, device=dev)
    o = pft.make_options(None)
    nb = lib.pft2d_batched_backward_workspace_size(v.shape[0], n, 2 * n, 1, ctypes.byref(o))
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    out = torch.empty(v.shape[0], 2, dtype=torch.float32, device=dev)
    vd, od, qod = (torch.from_numpy(a).to(dev) for a in (v, off, q_off))
    rc = lib.pft2d_polygons_batched_backward(vd.data_ptr(), v.shape[0], od.data_ptr(), n, q.data_ptr(),
                                             qod.data_ptr(), 2 * n, g.data_ptr(), out.data_ptr(), ws.data_ptr(), nb,
                                             ctypes.byref(o), None)
    assert rc == 0
    assert lib.pft_status(ws.data_ptr(), None) == 8
