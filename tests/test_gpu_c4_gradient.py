"""Gradient parity on the full differentiation workload: 16 icospheres of subdivision 4 (81,920
triangles, 40,992 vertices) on the 32^3 Q grid over [-30, 30)^3, loss
L(v) = sum_Q (|F(Q; v)|^2 - I_target(Q))^2 with I_target = |F|^2 of the copy whose vertices are moved
radially by 2 %.

The adjoint kernel (FP32 with compensated sums) is checked

* against central differences of the FP64 GPU forward, extrapolated from the steps h and h/2
  (Richardson: D = (4 D(h/2) - D(h)) / 3 cancels the O(h^2) term), on 32 seeded vertex coordinates and
  along one random direction of the coordinates (all whose moves are exact in float32); both steps
  are exact in float32 at the coordinates' exponents, so the differenced vertices are exactly v +- h;
* against the oracle's shape-derivative gradient under the same loss (weights g from the oracle's
  transform), on 64 sampled vertices.

Per coordinate the bar is |fd - adj| <= 1e-4 * max(|fd|, FLOOR * max|adj|): relative 1e-4, with an
absolute floor for coordinates whose derivative is tiny against the largest one (the FP32 adjoint's
error scales with the size of the terms it sums, not with their sum).

For one coordinate only the triangles at that vertex move, so F(v +- h e) = F(v) + [F_inc(v +- h e) -
F_inc(v)], F_inc the sum over the incident triangles.  F_inc is evaluated by the same FP64 GPU call on
that sub-list of triangles with the full vertex array; the sampled vertices are away from the bounding
box's faces (the centre c the library measures phases from does not move) and from c (no Q but Q = 0
takes the small-|Q| series, so every Q takes the same branch at v, v + h e and v - h e).  The random
direction moves every vertex and uses the full FP64 forward.
"""
import numpy as np
import pytest

import oracle
from paper_2104_08309_gb300 import synth

pytestmark = pytest.mark.gpu

REL = 1e-4         # spec bar: adjoint vs finite differences, relative
FLOOR = 1e-2       # below FLOOR * max|grad| a coordinate is held to REL * FLOOR * max|grad| (absolute)
H = 2.0 ** -11     # Richardson steps H and H/2 (exact float32 moves at the sampled coordinates)
N_COORDS = 32


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08309_gb300 import build as pbuild
    pbuild.build()
    return torch, torch.device("cuda:0")


@pytest.fixture(scope="module")
def c4(torch_dev):
    """Workload, oracle target and oracle transform (FP64 CPU; about a minute on 16 cores)."""
    w = synth.workload_c4()
    target = np.abs(oracle.ft3d(w.verts_target, w.faces, w.q)) ** 2
    F_or = oracle.ft3d(w.verts, w.faces, w.q)
    return w, target, F_or


def _pairs(z):
    return np.ascontiguousarray(np.stack([z.real, z.imag], axis=1))


def _f64(td, v, f, q):
    torch, dev = td
    import paper_2104_08309_gb300 as pft
    out = pft.pft3d_mesh(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev), q,
                         options={"precision": "fp64"}, check_status=True).cpu().numpy()
    return out[:, 0] + 1j * out[:, 1]


def _dloss(F_plus, F_minus, F0, target):
    """L(F_plus) - L(F_minus) for L(F) = sum (|F|^2 - I)^2, from the differences directly:
    (a^2 - b^2) = (a - b)(a + b), a - b = Re((F+ - F-) conj(F+ + F-))."""
    d = F_plus - F_minus
    s = F_plus + F_minus
    a_minus_b = np.real(d * np.conj(s))
    a_plus_b = np.abs(F_plus) ** 2 + np.abs(F_minus) ** 2 - 2.0 * target
    return float(np.sum(a_minus_b * a_plus_b))


def test_c4_adjoint_vs_richardson_fd_of_fp64_forward(torch_dev, c4):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    w, target, _ = c4
    v, f = w.verts, w.faces
    qd = torch.from_numpy(w.q).to(dev)
    F0 = _f64(torch_dev, v, f, qd)
    g = 4.0 * (np.abs(F0) ** 2 - target) * F0
    adj = pft.pft3d_mesh_backward(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev), qd,
                                  torch.from_numpy(_pairs(g)).to(dev), check_status=True).cpu().numpy()
    assert np.all(np.isfinite(adj))
    scale = float(np.max(np.abs(adj)))

    # sampled coordinates: vertices 0.05 inside the bounding box on every axis and 0.2 from its centre
    v64 = v.astype(np.float64)
    lo, hi = v64.min(axis=0), v64.max(axis=0)
    c = 0.5 * (lo + hi)
    ok = np.all((v64 - lo > 0.05) & (hi - v64 > 0.05), axis=1) & (np.linalg.norm(v64 - c, axis=1) > 0.2)
    rng = np.random.default_rng(2104)
    verts_sel = rng.choice(np.flatnonzero(ok), N_COORDS, replace=False)
    axes = rng.integers(0, 3, N_COORDS)
    rows = []
    for j, ax in zip(verts_sel, axes):
        inc = np.ascontiguousarray(f[np.any(f == j, axis=1)])
        finc0 = _f64(torch_dev, v, inc, qd)
        d = {}
        for step in (H, H / 2):
            vp, vm = v.copy(), v.copy()
            vp[j, ax] += np.float32(step)
            vm[j, ax] -= np.float32(step)
            assert float(vp[j, ax]) - float(v[j, ax]) == step and float(v[j, ax]) - float(vm[j, ax]) == step
            Fp = F0 + (_f64(torch_dev, vp, inc, qd) - finc0)
            Fm = F0 + (_f64(torch_dev, vm, inc, qd) - finc0)
            d[step] = _dloss(Fp, Fm, F0, target) / (2.0 * step)
        fd = (4.0 * d[H / 2] - d[H]) / 3.0
        rows.append((int(j), int(ax), fd, float(adj[j, ax]), d[H], d[H / 2]))
    fd = np.array([r[2] for r in rows])
    got = np.array([r[3] for r in rows])
    tol = REL * np.maximum(np.abs(fd), FLOOR * scale)
    err = np.abs(fd - got)
    worst = int(np.argmax(err / tol))
    assert np.all(err <= tol), (rows[worst], float(err[worst] / np.maximum(np.abs(fd[worst]), 1e-300)), scale)

    # one random direction (signs +-1) over every coordinate whose moves by +-H and +-H/2 are exact in
    # float32 (not those near zero or just below a power of two): full FP64 forwards at v +- h delta
    delta = rng.choice(np.array([-1.0, 1.0], np.float32), size=v.shape)
    for step in (H, H / 2):
        for sign in (1.0, -1.0):
            moved = (v + np.float32(sign * step)).astype(np.float64)
            delta[moved - v64 != sign * step] = 0.0
    assert np.mean(delta != 0) > 0.9
    dd = {}
    for step in (H, H / 2):
        vp = (v + np.float32(step) * delta).astype(np.float32)
        vm = (v - np.float32(step) * delta).astype(np.float32)
        assert np.array_equal(vp.astype(np.float64) - v64, step * delta.astype(np.float64))
        assert np.array_equal(v64 - vm.astype(np.float64), step * delta.astype(np.float64))
        dd[step] = _dloss(_f64(torch_dev, vp, f, qd), _f64(torch_dev, vm, f, qd), F0, target) / (2.0 * step)
    fd_dir = (4.0 * dd[H / 2] - dd[H]) / 3.0
    adj_dir = float(np.sum(adj.astype(np.float64) * delta))
    assert abs(fd_dir - adj_dir) <= REL * abs(fd_dir), (fd_dir, adj_dir, dd)


def test_c4_adjoint_vs_oracle_gradient_under_the_loss(torch_dev, c4):
    """The same loss with the oracle's transform in the weights: the adjoint against the oracle's
    shape-derivative gradient on 64 sampled vertices (each needs only its incident triangles)."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    w, target, F_or = c4
    g = 4.0 * (np.abs(F_or) ** 2 - target) * F_or
    got = pft.pft3d_mesh_backward(torch.from_numpy(w.verts).to(dev), torch.from_numpy(w.faces).to(dev),
                                  torch.from_numpy(w.q).to(dev), torch.from_numpy(_pairs(g)).to(dev),
                                  check_status=True).cpu().numpy()
    sel = np.sort(np.random.default_rng(45).choice(w.verts.shape[0], 64, replace=False))
    ref = oracle.grad3d(w.verts, w.faces, w.q, g, vsel=sel)
    scale = float(np.max(np.abs(got)))
    err = np.abs(got[sel] - ref)
    assert np.all(err <= REL * np.maximum(np.abs(ref), FLOOR * scale)), float(np.max(err / np.abs(ref)))
