"""GPU adjoints (vertex gradients) against the oracle's shape-derivative gradient and
central finite differences of the FP64 forward.

The GPU differentiates the forward formulas term by term (reverse mode); the
oracle integrates the boundary flux of the moving surface.  Tolerance: 1e-4 of
max |gradient| (the FP32 path's error budget for a gradient).
"""
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


def _g_pairs(g):
    return np.ascontiguousarray(np.stack([g.real, g.imag], axis=1))


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_2d_backward_vs_oracle(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    outer = synth.star_polygon(200, seed=4)
    hole = (0.3 * synth.star_polygon(31, seed=6))[::-1]
    v = (np.concatenate([outer, hole]) + np.float32(0.3)).astype(np.float32)
    off = np.array([0, 200, 231])
    q = np.concatenate([[[0.0, 0.0], [1e-4, 2e-4], [0.0, 0.05]], rng.uniform(-30, 30, (3000, 2))])
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    ref = oracle.grad2d(v, q, g, loop_off=off)
    got = pft.pft2d_polygons_backward(torch.from_numpy(v).to(dev), torch.from_numpy(q).to(dev),
                                      torch.from_numpy(_g_pairs(g)).to(dev), torch.from_numpy(off).to(dev),
                                      check_status=True).cpu().numpy()
    assert _rel(got, ref) < GTOL


@pytest.mark.parametrize("tau", [1.0, 0.05, 3.0, 6.0])
def test_3d_backward_vs_oracle(torch_dev, rng, tau):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f = synth.perturbed_icosphere(3, seed=12, amp=0.08)
    v = (v + np.array([0.2, -0.1, 0.3], np.float32)).astype(np.float32)
    q = np.concatenate([[[0, 0, 0], [1e-4, 0, 2e-4], [0, 0, 4.0], [6.0, 0, 0]], rng.uniform(-25, 25, (2500, 3))])
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    ref = oracle.grad3d(v, f, q, g)
    got = pft.pft3d_mesh_backward(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev),
                                  torch.from_numpy(q).to(dev), torch.from_numpy(_g_pairs(g)).to(dev),
                                  options={"face_series_tau": tau}, check_status=True).cpu().numpy()
    assert _rel(got, ref) < GTOL


def test_3d_loss_gradient_vs_fd_of_fp64_forward(torch_dev):
    """C4-style loss sum_Q (|F|^2 - I)^2 on a union of small spheres: the adjoint against central
    differences of the GPU FP64 forward, and against the oracle's analytic gradient."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f = synth.sphere_union(3, 2, seed=4)
    vt, _ = synth.sphere_union(3, 2, seed=4, perturb=0.02, perturb_seed=44)
    q = synth.q_grid_3d(12, 30.0)
    target = np.abs(oracle.ft3d(vt, f, q)) ** 2
    F = oracle.ft3d(v, f, q)
    g = 4.0 * (np.abs(F) ** 2 - target) * F
    qd, fd = torch.from_numpy(q).to(dev), torch.from_numpy(f).to(dev)
    got = pft.pft3d_mesh_backward(torch.from_numpy(v).to(dev), fd, qd, torch.from_numpy(_g_pairs(g)).to(dev),
                                  check_status=True).cpu().numpy()
    ref = oracle.grad3d(v, f, q, g)
    assert _rel(got, ref) < GTOL

    def loss(vv):
        out = pft.pft3d_mesh(torch.from_numpy(vv).to(dev), fd, qd, options={"precision": "fp64"}).cpu().numpy()
        Fv = out[:, 0] + 1j * out[:, 1]
        return np.sum((np.abs(Fv) ** 2 - target) ** 2)

    rng = np.random.default_rng(8)
    scale = np.max(np.abs(ref))
    h = 1e-3   # float32 vertices: steps that are exact multiples of the coordinate spacing
    for j in rng.choice(v.shape[0], 6, replace=False):
        for c in range(3):
            vp, vm = v.copy(), v.copy()
            vp[j, c] += np.float32(h)
            vm[j, c] -= np.float32(h)
            step = float(vp[j, c]) - float(vm[j, c])
            fdv = (loss(vp) - loss(vm)) / step
            assert abs(fdv - got[j, c]) < 1e-4 * scale + 2e-3 * abs(fdv), (j, c, fdv, got[j, c])


def test_autograd_ft3d(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f = synth.perturbed_icosphere(2, seed=3, amp=0.1)
    q = rng.uniform(-10, 10, (700, 3))
    vt = torch.from_numpy(v).to(dev).requires_grad_(True)
    F = pft.ft3d(vt, torch.from_numpy(f).to(dev), torch.from_numpy(q).to(dev))
    target = torch.rand(q.shape[0], dtype=torch.float64, device=dev)
    L = ((F.abs() ** 2 - target) ** 2).sum()
    L.backward()
    Fn = F.detach().cpu().numpy()
    g = 4.0 * (np.abs(Fn) ** 2 - target.cpu().numpy()) * Fn
    ref = oracle.grad3d(v, f, q, g)
    assert _rel(vt.grad.cpu().numpy(), ref) < GTOL


def test_c4_full_size_sampled_vertices(torch_dev):
    """16 icospheres (81,920 faces) on the full 32^3 grid with a seeded random g:
    64 sampled vertices against the oracle (each needs only its incident faces)."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    w = synth.workload_c4()
    rng = np.random.default_rng(44)
    g = rng.normal(size=w.q.shape[0]) + 1j * rng.normal(size=w.q.shape[0])
    got = pft.pft3d_mesh_backward(torch.from_numpy(w.verts).to(dev), torch.from_numpy(w.faces).to(dev),
                                  torch.from_numpy(w.q).to(dev), torch.from_numpy(_g_pairs(g)).to(dev),
                                  check_status=True).cpu().numpy()
    sel = np.sort(rng.choice(w.verts.shape[0], 64, replace=False))
    ref = oracle.grad3d(w.verts, w.faces, w.q, g, vsel=sel)
    assert np.all(np.isfinite(got))
    assert _rel(got[sel], ref) < GTOL
    # reproducible
    again = pft.pft3d_mesh_backward(torch.from_numpy(w.verts).to(dev), torch.from_numpy(w.faces).to(dev),
                                    torch.from_numpy(w.q).to(dev), torch.from_numpy(_g_pairs(g)).to(dev)).cpu().numpy()
    assert np.array_equal(got, again)


def test_far_from_the_origin(torch_dev, rng):
    """The adjoints of shapes thousands of units from the origin, at Q that float32 cannot represent:
    the Q records' weights g e^{-iQ.c}/|Q|^2 take the caller's Q, as the forward's finish does."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v = synth.star_polygon(200, seed=4, center=(2500.0, -1800.0)).astype(np.float32)
    q = np.concatenate([[[1e-5, 2e-5], [0.3, -0.2]], rng.uniform(-30, 30, (1500, 2))])
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    ref = oracle.grad2d(v, q, g)
    got = pft.pft2d_polygons_backward(torch.from_numpy(v).to(dev), torch.from_numpy(q).to(dev),
                                      torch.from_numpy(_g_pairs(g)).to(dev), check_status=True).cpu().numpy()
    assert _rel(got, ref) < GTOL
    v, f = synth.perturbed_icosphere(2, seed=12, amp=0.08)
    v = (v.astype(np.float64) + np.array([1500.0, -2200.0, 800.0])).astype(np.float32)
    q = np.concatenate([[[1e-5, 0, 2e-5], [0.3, -0.2, 0.1]], rng.uniform(-25, 25, (1200, 3))])
    g = rng.normal(size=q.shape[0]) + 1j * rng.normal(size=q.shape[0])
    ref = oracle.grad3d(v, f, q, g)
    got = pft.pft3d_mesh_backward(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev),
                                  torch.from_numpy(q).to(dev), torch.from_numpy(_g_pairs(g)).to(dev),
                                  check_status=True).cpu().numpy()
    assert _rel(got, ref) < GTOL
