"""GPU parity of the batched 2D transform (one persistent launch over a CSR of polygons)."""
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


def _mixed_batch():
    """Polygons of 3..5000 vertices (one above the 4096-segment chunk), some far from the origin."""
    rng = np.random.default_rng(17)
    sizes = [3, 4, 8, 5000, 17, 300, 9, 1024, 4096, 4097, 64, 3]
    parts = [synth.star_polygon(n, seed=100 + i, center=tuple(rng.uniform(-3, 3, 2)))
             for i, n in enumerate(sizes)]
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    return np.concatenate(parts).astype(np.float32), off


def _c(a):
    a = a.detach().cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def _areas(v, off):
    return np.array([abs(oracle.ft2d(v[off[i]:off[i + 1]], [[0.0, 0.0]])[0]) for i in range(off.size - 1)])


# the FP64 path keeps at most 2 Q points per thread (larger shapes are refused synchronously)
@pytest.mark.parametrize("prec,r,nt", [(p, r, nt) for p in ("fp32", "fp64")
                                       for r, nt in ((4, 128), (1, 256), (2, 128), (4, 512))
                                       if p == "fp32" or (r <= 2 and nt < 512)])
def test_shared_grid_vs_oracle(torch_dev, prec, r, nt):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, off = _mixed_batch()
    rng = np.random.default_rng(3)
    q = np.concatenate([[[0, 0], [1e-5, 0], [0, 0.02], [30.0, 0]], rng.uniform(-40, 40, (900, 2))])
    out = pft.pft2d_polygons_batched(torch.from_numpy(v).to(dev), torch.from_numpy(off), torch.from_numpy(q).to(dev),
                                     options={"precision": prec, "q_per_thread": r, "block_threads": nt},
                                     check_status=True)
    got = _c(out)
    ref = oracle.ft2d_batched(v, off, q)
    areas = _areas(v, off)
    err = np.max(np.abs(got - ref), axis=1) / areas
    assert np.all(err < TOL[prec]), err


def test_per_polygon_q_sets(torch_dev):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, off = _mixed_batch()
    rng = np.random.default_rng(5)
    counts = np.array([5, 0, 700, 3, 1, 64, 513, 2, 0, 40, 1000, 6])
    q_off = np.zeros(counts.size + 1, dtype=np.int64)
    q_off[1:] = np.cumsum(counts)
    q = rng.uniform(-25, 25, (q_off[-1], 2))
    q[q_off[2]] = 0.0
    out = pft.pft2d_polygons_batched(torch.from_numpy(v).to(dev), torch.from_numpy(off), torch.from_numpy(q).to(dev),
                                     q_off=torch.from_numpy(q_off), check_status=True)
    got = _c(out)
    ref = oracle.ft2d_batched(v, off, q, q_off=q_off)
    areas = _areas(v, off)
    for i in range(counts.size):
        sl = slice(q_off[i], q_off[i + 1])
        if counts[i]:
            assert np.max(np.abs(got[sl] - ref[sl])) / areas[i] < TOL["fp32"], i


def test_c3_full_batch_sampled_and_graph_replay(torch_dev):
    """4,096 polygons (log-uniform 8..4096 vertices) on the shared 64x64 grid: one prepared schedule,
    captured in a CUDA graph and replayed; 40 seeded polygons checked against the oracle on every Q."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    w = synth.workload_c3()
    vd, qd = torch.from_numpy(w.verts).to(dev), torch.from_numpy(w.q).to(dev)
    offd = torch.from_numpy(w.poly_off).to(dev)
    prep = pft.pft2d_batched_prepare(w.poly_off, w.q.shape[0], device=dev)
    direct = pft.pft2d_polygons_batched(vd, offd, qd, prepared=prep, check_status=True).clone()
    out = torch.empty(w.poly_off.size - 1, w.q.shape[0], 2, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):          # warm the library on the capture stream
        pft.pft2d_polygons_batched(vd, offd, qd, prepared=prep, out=out)
    torch.cuda.current_stream(dev).wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pft.pft2d_polygons_batched(vd, offd, qd, prepared=prep, out=out)
    out.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert pft.pft_status(prep.ws) == 0
    assert torch.equal(out, direct)                 # deterministic schedule: bitwise equal
    rng = np.random.default_rng(33)
    sel = np.sort(rng.choice(w.poly_off.size - 1, 40, replace=False))
    got = _c(direct)[sel]
    for k, i in enumerate(sel):
        vi = w.verts[w.poly_off[i]:w.poly_off[i + 1]]
        ref = oracle.ft2d(vi, w.q)
        area = abs(oracle.ft2d(vi, [[0.0, 0.0]])[0])
        assert np.max(np.abs(got[k] - ref)) / area < TOL["fp32"], i


def test_c3_full_batch_fp32_vs_fp64_gpu(torch_dev):
    """Every one of the 4,096 polygons on every Q: the FP32-compensated path, in each launch shape
    the autotuner may pick for the benchmark, against the FP64 GPU path (itself held to 1e-12 of the
    oracle above), relative to each polygon's area."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    from paper_2104_08309_gb300 import autotune
    w = synth.workload_c3()
    vd, qd = torch.from_numpy(w.verts).to(dev), torch.from_numpy(w.q).to(dev)
    offd = torch.from_numpy(w.poly_off).to(dev)
    prep = pft.pft2d_batched_prepare(w.poly_off, w.q.shape[0], options={"precision": "fp64"}, device=dev)
    ref = _c(pft.pft2d_polygons_batched(vd, offd, qd, prepared=prep, check_status=True))
    q0 = int(np.flatnonzero(np.all(w.q == 0, axis=1))[0])
    area = np.abs(ref[:, q0])
    for r, nt in autotune.CANDIDATES_BATCHED_FP32:
        prep = pft.pft2d_batched_prepare(w.poly_off, w.q.shape[0], options={"q_per_thread": r, "block_threads": nt},
                                         device=dev)
        got = _c(pft.pft2d_polygons_batched(vd, offd, qd, prepared=prep, check_status=True))
        err = np.max(np.abs(got - ref), axis=1) / area
        assert np.all(err < TOL["fp32"]), (r, nt)
        assert err.max() < 1e-6, (r, nt)          # measured 3.1e-7 on a GB300


def test_plan_mismatch_is_rejected(torch_dev):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, off = _mixed_batch()
    q = torch.zeros(10, 2, dtype=torch.float64, device=dev)
    prep = pft.pft2d_batched_prepare(off, 10, device=dev)
    with pytest.raises(pft.PFTError):
        pft.pft2d_polygons_batched(torch.from_numpy(v).to(dev), torch.from_numpy(off), q[:7], prepared=prep)
    # device-side check: same sizes, different offsets
    off2 = off.copy()
    off2[1] += 1
    with pytest.raises(pft.PFTError, match="offsets"):
        pft.pft2d_polygons_batched(torch.from_numpy(v).to(dev), torch.from_numpy(off2).to(dev), q, prepared=prep,
                                   check_status=True)


def test_default_shape_on_a_large_shared_grid(torch_dev):
    """On a shared Q set of 4 x 512 points or more the default launch shape is one block of 512
    threads per SM (bit for bit the same as asking for it).  Every Q point's sum runs over the same
    segments in the same order in any launch shape, but the 512-thread shapes sum over tiles of 256
    segments rather than 128 (the FP32 sums are compensated across tiles): the 4 x 128 and 4 x 256
    shapes agree with each other bit for bit and with the default to rounding, and all with the
    oracle on sampled polygons."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, off = synth.batched_star_polygons(96, seed=8)
    q = synth.q_grid_2d(48, 40.0)                   # 2,304 points, one ragged 2,048-point tile
    vd, qd, offd = torch.from_numpy(v).to(dev), torch.from_numpy(q).to(dev), torch.from_numpy(off).to(dev)
    outs = {}
    for name, opts in (("default", None), ("4x128", {"q_per_thread": 4, "block_threads": 128}),
                       ("4x256", {"q_per_thread": 4, "block_threads": 256}),
                       ("4x512", {"q_per_thread": 4, "block_threads": 512})):
        prep = pft.pft2d_batched_prepare(off, q.shape[0], options=opts, device=dev)
        outs[name] = pft.pft2d_polygons_batched(vd, offd, qd, prepared=prep, check_status=True).clone()
    assert torch.equal(outs["default"], outs["4x512"])
    assert torch.equal(outs["4x128"], outs["4x256"])
    got, alt = _c(outs["default"]), _c(outs["4x128"])
    area = np.abs(got[:, np.flatnonzero(np.all(q == 0, axis=1))[0]])
    assert np.max(np.abs(got - alt).max(axis=1) / area) < 1e-6
    for i in (0, 17, 95):
        vi = v[off[i]:off[i + 1]]
        ref = oracle.ft2d(vi, q)
        assert np.max(np.abs(got[i] - ref)) / abs(ref[np.flatnonzero(np.all(q == 0, axis=1))[0]]) < TOL["fp32"], i


@pytest.mark.parametrize("shape", [None, (4, 128)])
def test_far_from_the_origin_phase_reduction(torch_dev, shape):
    """Polygons centred about 3e3 and 1e5 from the origin: the translation phase Q.c reaches about
    1.7e5 rad, which the FP32 finish reduces from a float-float Q.c in two parts, and about 6e6 rad,
    beyond 2^20 rad, where it takes the FP64 finish; one polygon of 5,000 vertices (two chunks) goes
    through the multi-chunk finish.  Every polygon against the oracle within 1e-5 of its area."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    specs = [(64, (2500.0, -1800.0)), (5000, (-3100.0, 2000.0)), (300, (90000.0, -60000.0)), (17, (1.5, 0.5))]
    parts = [synth.star_polygon(n, seed=40 + k, center=c) for k, (n, c) in enumerate(specs)]
    off = np.zeros(len(parts) + 1, dtype=np.int64)
    off[1:] = np.cumsum([p.shape[0] for p in parts])
    v = np.concatenate(parts).astype(np.float32)
    rng = np.random.default_rng(41)
    q = np.concatenate([[[0.0, 0.0], [0.3, -0.2]], rng.uniform(-40, 40, (600, 2))])
    opts = None if shape is None else {"q_per_thread": shape[0], "block_threads": shape[1]}
    got = _c(pft.pft2d_polygons_batched(torch.from_numpy(v).to(dev), torch.from_numpy(off),
                                        torch.from_numpy(q).to(dev), options=opts, check_status=True))
    areas = _areas(v, off)
    for i in range(len(parts)):
        ref = oracle.ft2d(v[off[i]:off[i + 1]], q)
        assert np.max(np.abs(got[i] - ref)) / areas[i] < TOL["fp32"], i


def test_per_polygon_q_sets_one_block_per_sm(torch_dev):
    """Per-polygon Q lists (short ones among them: 2,048-point Q tiles mostly empty) with one block of
    512 threads per SM asked for: the default launch shape's result to rounding (the 512-thread shapes
    sum over tiles of 256 segments, the others 128), and the oracle."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, off = _mixed_batch()
    rng = np.random.default_rng(6)
    counts = np.array([5, 0, 700, 3, 1, 64, 2100, 2, 0, 40, 1000, 6])
    q_off = np.zeros(counts.size + 1, dtype=np.int64)
    q_off[1:] = np.cumsum(counts)
    q = rng.uniform(-25, 25, (q_off[-1], 2))
    args = (torch.from_numpy(v).to(dev), torch.from_numpy(off), torch.from_numpy(q).to(dev))
    a = pft.pft2d_polygons_batched(*args, q_off=torch.from_numpy(q_off), check_status=True)
    b = pft.pft2d_polygons_batched(*args, q_off=torch.from_numpy(q_off), options={"q_per_thread": 4,
                                   "block_threads": 512}, check_status=True)
    areas = _areas(v, off)
    ca, cb = _c(a), _c(b)
    for i in range(counts.size):
        sl = slice(q_off[i], q_off[i + 1])
        if counts[i]:
            assert np.max(np.abs(ca[sl] - cb[sl])) / areas[i] < 1e-6, i
    got = cb
    ref = oracle.ft2d_batched(v, off, q, q_off=q_off)
    for i in range(counts.size):
        sl = slice(q_off[i], q_off[i + 1])
        if counts[i]:
            assert np.max(np.abs(got[sl] - ref[sl])) / areas[i] < TOL["fp32"], i
