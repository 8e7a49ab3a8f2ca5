"""The Q order of the main kernels (q_order option, pft_q_order): the slot -> Q map against a host
mirror of its definition (bit-exact: it is index work), the compactness of the groups it forms on a
grid, and the forward calls in that order against the caller's order (bitwise in 2D, where the
arithmetic of a pair does not depend on the other Q points of its group; to rounding in 3D, where
the group chooses between the series and the edge sum) and against the oracle."""
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


def _spread(c, d):
    """Bit b of c moved to bit d*b (Morton interleave for d coordinates)."""
    out = np.zeros(c.shape, np.uint64)
    for b in range(10 if d == 3 else 16):
        out |= ((c.astype(np.uint64) >> np.uint64(b)) & np.uint64(1)) << np.uint64(d * b)
    return out


def mirror_perm(q, r, nt):
    """The slot -> Q map as the header defines it: FP32 coordinates quantised over their bounding
    box (NaN skipped for the box and put on level 0), Morton keys, a stable sort, runs of 32 r
    sorted points dealt to the groups of whole blocks, the ragged last block in sorted order."""
    qf = q.astype(np.float32)
    n, d = qf.shape
    levels = np.float32(1 << (10 if d == 3 else 16))
    key = np.zeros(n, np.uint64)
    for k in range(d):
        x = qf[:, k]
        fin = x[~np.isnan(x)]
        lo, hi = (fin.min(), fin.max()) if fin.size else (np.float32(np.nan), np.float32(np.nan))
        with np.errstate(invalid="ignore", divide="ignore"):
            t = (x - lo) / (hi - lo) if hi > lo else np.zeros(n, np.float32)
            lev = np.where(t > 0, np.minimum(t * levels, levels - np.float32(1)), np.float32(0))
        key |= _spread(lev.astype(np.uint32), d) << np.uint64(k)
    order = np.argsort(key, kind="stable")
    per_block = r * nt
    full = n // per_block * per_block
    p = np.arange(n)
    g, o = p // (32 * r), p % (32 * r)
    wpb = nt // 32
    slot = np.where(p < full, (g // wpb) * per_block + (o // 32) * nt + (g % wpb) * 32 + o % 32, p)
    perm = np.empty(n, np.int64)
    perm[slot] = order
    return perm


def _perm(td, q, r, nt):
    torch, dev = td
    import paper_2104_08309_gb300 as pft
    return pft.q_order(torch.from_numpy(np.ascontiguousarray(q, np.float64)).to(dev), r, nt).cpu().numpy()


@pytest.mark.parametrize("d", [2, 3])
def test_q_order_matches_its_definition(torch_dev, rng, d):
    """Random Q with duplicates, a NaN coordinate and a ragged last block, for every launch shape."""
    q = rng.uniform(-40, 40, (5000, d))
    q[100:140] = q[7]                       # duplicates keep the caller's order among themselves
    q[3, 0] = np.nan
    q[11] = 0.0
    for r in (1, 2, 4, 8):
        for nt in (128, 256, 512):
            got = _perm(torch_dev, q, r, nt)
            assert np.array_equal(np.sort(got), np.arange(q.shape[0])), (r, nt)
            assert np.array_equal(got, mirror_perm(q, r, nt)), (r, nt)


def test_q_order_degenerate_sets(torch_dev):
    """All Q equal (an empty box: every key 0, so the caller's order), one point, none."""
    q = np.tile([[1.5, -2.0, 3.0]], (3000, 1))
    assert np.array_equal(_perm(torch_dev, q, 4, 128), mirror_perm(q, 4, 128))
    assert np.array_equal(_perm(torch_dev, q[:1], 4, 128), [0])
    assert _perm(torch_dev, q[:0], 4, 128).shape == (0,)


def test_q_order_groups_are_compact_on_a_grid(torch_dev):
    """On a 32^3 grid each group of 32 threads x 4 Q points gets a 4 x 4 x 8 block of the grid
    (128 consecutive Morton codes); in the caller's row order the same slots span a 1 x 13 x 32 slab."""
    q = synth.q_grid_3d(32, 30.0)
    perm = _perm(torch_dev, q, 4, 128)
    step = 60.0 / 32
    idx = np.rint((q[perm] + 30.0) / step).astype(int)
    n = q.shape[0]
    slots = (np.arange(n // 512)[:, None, None, None] * 512 + np.arange(4)[None, :, None, None] * 32
             + np.arange(4)[None, None, :, None] * 128 + np.arange(32)[None, None, None, :]).reshape(-1, 128)
    ext = idx[slots].max(axis=1) - idx[slots].min(axis=1)          # [groups, 3] extents in grid steps
    assert np.all(np.sort(ext, axis=1) == [3, 3, 7])


def test_tiled_forward_2d_bitwise(torch_dev, rng):
    """4,096 segments x 512^2 Q (1.1e9 pairs, above the ordering threshold): the library's order
    equals the caller's bitwise, a shuffled Q array gives the shuffled result bitwise, and a sample
    agrees with the oracle."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v = synth.star_polygon(4096, seed=11)
    g = np.linspace(-40.0, 40.0, 512, endpoint=False)
    q = np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    vd, qd = torch.from_numpy(v).to(dev), torch.from_numpy(q).to(dev)
    a = pft.pft2d_polygons(vd, qd, check_status=True).cpu().numpy()
    b = pft.pft2d_polygons(vd, qd, options={"q_order": "as_given"}, check_status=True).cpu().numpy()
    assert np.array_equal(a, b)
    s = rng.permutation(q.shape[0])
    c = pft.pft2d_polygons(vd, torch.from_numpy(q[s]).to(dev), check_status=True).cpu().numpy()
    assert np.array_equal(c, a[s])
    sel = rng.choice(q.shape[0], 200, replace=False)
    ref = oracle.ft2d(v, q[sel])
    got = a[sel, 0] + 1j * a[sel, 1]
    assert np.max(np.abs(got - ref)) / abs(oracle.ft2d(v, [[0.0, 0.0]])[0]) < 1e-5


def test_tiled_forward_3d(torch_dev, rng):
    """20,480 faces x 64^3 Q (5.4e9 pairs): the library's order against the caller's order (1e-6 of
    the volume: a group may switch a face between the series and the edge sum) and, on sampled Q
    including Q = 0, against the oracle; a shuffled Q array gives the shuffled result to rounding."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f = synth.icosphere(5)
    q = synth.q_grid_3d(64, 30.0)
    vd, fd, qd = torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev), torch.from_numpy(q).to(dev)
    a = pft.pft3d_mesh(vd, fd, qd, check_status=True).cpu().numpy()
    b = pft.pft3d_mesh(vd, fd, qd, options={"q_order": "as_given"}, check_status=True).cpu().numpy()
    i0 = int(np.flatnonzero(np.all(q == 0, axis=1))[0])
    vol = abs(a[i0, 0])
    assert np.max(np.abs(a - b)) / vol < 1e-6
    s = rng.permutation(q.shape[0])
    c = pft.pft3d_mesh(vd, fd, torch.from_numpy(q[s]).to(dev), check_status=True).cpu().numpy()
    assert np.max(np.abs(c - a[s])) / vol < 1e-6
    sel = np.concatenate([[i0], rng.choice(q.shape[0], 255, replace=False)])
    ref = oracle.ft3d(v, f, q[sel])
    got = a[sel, 0] + 1j * a[sel, 1]
    assert np.max(np.abs(got - ref)) / abs(ref[0]) < 1e-5


def test_tiled_batched_2d_bitwise_and_graph(torch_dev):
    """The 4,096-polygon batch on its shared 64 x 64 grid (1.1e10 pairs): the library's order equals
    the caller's bitwise, also when the call (ordering included) is replayed from a CUDA graph."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    w = synth.workload_c3()
    vd, qd = torch.from_numpy(w.verts).to(dev), torch.from_numpy(w.q).to(dev)
    offd = torch.from_numpy(w.poly_off).to(dev)
    p1 = pft.pft2d_batched_prepare(w.poly_off, w.q.shape[0], device=dev)
    p0 = pft.pft2d_batched_prepare(w.poly_off, w.q.shape[0], options={"q_order": "as_given"}, device=dev)
    a = pft.pft2d_polygons_batched(vd, offd, qd, prepared=p1)
    b = pft.pft2d_polygons_batched(vd, offd, qd, prepared=p0)
    assert torch.equal(a, b)
    assert pft.pft_status(p1.ws) == 0
    out = torch.empty_like(a)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        pft.pft2d_polygons_batched(vd, offd, qd, prepared=p1, out=out)
    torch.cuda.current_stream(dev).wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pft.pft2d_polygons_batched(vd, offd, qd, prepared=p1, out=out)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, a)


def test_tiled_batched_3d_against_caller_order(torch_dev, rng):
    """1,024 meshes on a shared 32^3 grid (5.5e10 pairs): the library's order against the caller's
    within the FP32 bar (1e-5 of each mesh's volume: both are FP32 evaluations, and another grouping
    can move a face between the series and the edge sum, whose FP32 error on these small meshes
    reaches ~1e-6 of the volume), and sampled meshes and Q points against the oracle."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f, off = synth.mesh_batch(1024, seed=21)
    q = synth.q_grid_3d(32, 30.0)
    vd, fd, qd, offd = (torch.from_numpy(x).to(dev) for x in (v, f, q, off))
    p1 = pft.pft3d_batched_prepare(off, q.shape[0], device=dev)
    p0 = pft.pft3d_batched_prepare(off, q.shape[0], options={"q_order": "as_given"}, device=dev)
    a = pft.pft3d_meshes_batched(vd, fd, offd, qd, prepared=p1).cpu().numpy()
    b = pft.pft3d_meshes_batched(vd, fd, offd, qd, prepared=p0).cpu().numpy()
    i0 = int(np.flatnonzero(np.all(q == 0, axis=1))[0])
    vol = np.abs(b[:, i0, 0])
    assert np.all(np.max(np.abs(a - b), axis=(1, 2)) / vol < 1e-5)
    for m in rng.choice(off.size - 1, 4, replace=False):
        sel = np.concatenate([[i0], rng.choice(q.shape[0], 63, replace=False)])
        ref = oracle.ft3d(v, f[off[m]:off[m + 1]], q[sel])
        got = a[m, sel, 0] + 1j * a[m, sel, 1]
        assert np.max(np.abs(got - ref)) / abs(ref[0]) < 1e-5, m


def test_tiled_qgrad(torch_dev, rng):
    """Q-gradients above the ordering threshold: in 2D (4,096 segments x 512^2 Q) the library's order
    gives the caller's result bitwise (one Q point per thread, no per-group choice that changes a
    pair's arithmetic); in 3D on the differentiation workload (81,920 faces x 32^3 Q) it agrees within
    the Q-gradient bar, 1e-5 of max|g| V max|r|, and a sample agrees with the oracle's Richardson
    differences."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v = synth.star_polygon(4096, seed=11)
    g1 = np.linspace(-40.0, 40.0, 512, endpoint=False)
    q = np.stack(np.meshgrid(g1, g1, indexing="ij"), axis=-1).reshape(-1, 2)
    gw = rng.normal(size=(q.shape[0], 2))
    vd, qd, gd = (torch.from_numpy(x).to(dev) for x in (v, q, gw))
    a = pft.pft2d_polygons_qgrad(vd, qd, gd, check_status=True)
    b = pft.pft2d_polygons_qgrad(vd, qd, gd, options={"q_order": "as_given"}, check_status=True)
    assert torch.equal(a, b)
    w = synth.workload_c4()
    vd, fd, qd = (torch.from_numpy(x).to(dev) for x in (w.verts, w.faces, w.q))
    g = rng.normal(size=w.q.shape[0]) + 1j * rng.normal(size=w.q.shape[0])
    gd = torch.from_numpy(np.ascontiguousarray(np.stack([g.real, g.imag], axis=1))).to(dev)
    a = pft.pft3d_mesh_qgrad(vd, fd, qd, gd, check_status=True).cpu().numpy()
    b = pft.pft3d_mesh_qgrad(vd, fd, qd, gd, options={"q_order": "as_given"}, check_status=True).cpu().numpy()
    vol = abs(oracle.ft3d(w.verts, w.faces, [[0.0, 0.0, 0.0]])[0])
    scale = np.max(np.abs(g)) * vol * float(np.max(np.linalg.norm(w.verts.astype(np.float64), axis=1)))
    assert np.max(np.abs(a - b)) < 1e-5 * scale
    sel = rng.choice(w.q.shape[0], 16, replace=False)
    ref = oracle.qgrad3d(w.verts, w.faces, w.q[sel], g[sel])
    assert np.max(np.abs(a[sel] - ref)) < 1e-5 * scale
