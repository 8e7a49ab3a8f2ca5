"""GPU parity of the forward transforms against the FP64 CPU oracle (through the C ABI).

Tolerances (relative to max|F| = F(0) = area or volume, since |F(Q)| <= F(0)):
FP32-compensated path 1e-5, FP64 path 1e-12.
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


def run3d(td, v, f, q, **opts):
    torch, dev = td
    import paper_2104_08309_gb300 as pft
    out = pft.pft3d_mesh(torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev),
                         torch.from_numpy(np.ascontiguousarray(f, np.int32)).to(dev),
                         torch.from_numpy(np.ascontiguousarray(q, np.float64)).to(dev), options=opts,
                         check_status=True)
    return _c(out)


def run2d(td, v, q, loop_off=None, **opts):
    torch, dev = td
    import paper_2104_08309_gb300 as pft
    lo = None if loop_off is None else torch.tensor(loop_off, dtype=torch.int64, device=dev)
    out = pft.pft2d_polygons(torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev),
                             torch.from_numpy(np.ascontiguousarray(q, np.float64)).to(dev), lo,
                             options=opts, check_status=True)
    return _c(out)


def rel_err(got, ref, measure):
    return float(np.max(np.abs(got - ref)) / abs(measure))


def _q3_mix(rng, n, scale):
    q = rng.uniform(-scale, scale, (n, 3))
    special = [[0, 0, 0], [1e-6, 0, 0], [0, 2e-3, 1e-3], [0, 0, 3.0], [4.0, 0, 0], [0, -5.0, 0],
               [1, 1, 0], [0.05, 0.02, -0.01]]
    return np.concatenate([special, q])


# the FP64 path keeps at most 2 Q points per thread (larger shapes are refused synchronously)
@pytest.mark.parametrize("prec,r,nt", [(p, r, nt) for p in ("fp32", "fp64")
                                       for r, nt in ((1, 128), (2, 256), (4, 256), (8, 128))
                                       if p == "fp32" or r <= 2])
def test_3d_ragged_tiles_vs_oracle(torch_dev, prec, r, nt, rng):
    v, f = synth.perturbed_icosphere(2, seed=21, amp=0.15)       # 320 faces: 5 tiles of 64, 10 of 32
    v = (v + np.array([0.7, -0.3, 0.2], np.float32)).astype(np.float32)
    q = _q3_mix(rng, 3001, 15.0)                                  # ragged against every block size
    ref = oracle.ft3d(v, f, q)
    got = run3d(torch_dev, v, f, q, precision=prec, q_per_thread=r, block_threads=nt)
    assert rel_err(got, ref, ref[0]) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_3d_box_normals_and_limits(torch_dev, prec):
    v, f = synth.box_mesh(1.25, 0.75, 1.875)
    q = np.array([[0, 0, 0], [0, 0, 2.5], [0, 0, -7.0], [1.5, 0, 0], [0, 3, 0], [1e-7, 0, 0],
                  [2.0, 3.0, 0.0], [0.3, -0.2, 0.9], [40.0, 0, 0], [0, 0, 1e-3]])
    ref = oracle.ft3d(v, f, q)
    got = run3d(torch_dev, v, f, q, precision=prec)
    assert rel_err(got, ref, ref[0]) < TOL[prec]
    assert abs(got[0] - 1.25 * 0.75 * 1.875) < 1e-12


@pytest.mark.parametrize("tau", [1e-3, 0.25, 1.0, 2.0, 3.0, 4.5, 6.0])
def test_3d_face_branch_threshold(torch_dev, tau, rng):
    """Both per-face branches (edge sum of Eq. 14, series of Eq. 13) agree with the oracle."""
    v, f = synth.perturbed_icosphere(3, seed=5, amp=0.05)
    q = _q3_mix(rng, 1500, 40.0)
    ref = oracle.ft3d(v, f, q)
    for prec in ("fp32", "fp64"):
        got = run3d(torch_dev, v, f, q, precision=prec, face_series_tau=tau)
        assert rel_err(got, ref, ref[0]) < TOL[prec], (prec, tau)


def test_3d_every_series_form(torch_dev):
    """Each Q point repeated over a whole block (R x NT = 4 x 128), so for every face a warp's P values
    are equal and the ladder takes exactly the form for that P. |Q| sweeps the box's faces across all
    five series bounds (k <= 7, 9, 11, 13, 17 for P < 1/4, 1, 9/4, 4, 9) and past tau^2/4 = 9 (edge sum);
    every output matches the oracle."""
    v, f = synth.box_mesh(1.25, 0.75, 1.875)
    d = np.array([0.48, -0.6, 0.64])
    qd = np.linspace(0.05, 6.0, 120)[:, None] * d[None, :]
    got = run3d(torch_dev, v, f, np.repeat(qd, 512, axis=0), q_per_thread=4, block_threads=128,
                face_series_tau=6.0)
    ref = oracle.ft3d(v, f, qd)
    assert rel_err(got, np.repeat(ref, 512), 1.25 * 0.75 * 1.875) < TOL["fp32"]
    # P = a0^2 + a0 a1 + a1^2 of the corner phases about each face's centroid, for every (face, Q)
    p = v.astype(np.float64)[f]
    g = p.mean(axis=1)
    a0, a1 = (np.einsum("kj,fj->kf", qd, p[:, i] - g) for i in (0, 1))
    P = (a0 * a0 + a0 * a1 + a1 * a1).ravel()
    edges = [0.0, 0.25, 1.0, 2.25, 4.0, 9.0, np.inf]
    for lo, hi in zip(edges[:-1], edges[1:]):
        assert np.count_nonzero((P > lo) & (P < hi)) >= 5, (lo, hi)


def test_3d_short_series_taken_whatever_tau(torch_dev, rng):
    """Small faces at small |Q| (every P < 1/4): the short series serves every warp for any
    tau >= 1, so tau = 1, 2, 3 and 6 give bitwise the same FP32 result; the default is tau = 6."""
    v, f = synth.icosphere(5)                        # edges ~0.06: P < 1/4 for |Q| < ~8
    q = rng.uniform(-4.0, 4.0, (3000, 3))
    q[0] = 0.0
    a = run3d(torch_dev, v, f, q, face_series_tau=1.0, k_splits=2)
    for tau in (2.0, 3.0, 6.0, 0.0):
        b = run3d(torch_dev, v, f, q, face_series_tau=tau, k_splits=2)
        assert np.array_equal(a, b), tau
    ref = oracle.ft3d(v, f, q[:200])
    assert rel_err(a[:200], ref, ref[0]) < TOL["fp32"]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_2d_loops_and_limits(torch_dev, prec, rng):
    outer = synth.star_polygon(300, seed=2)
    hole = (0.3 * synth.star_polygon(37, seed=3))[::-1]          # clockwise: a hole
    v = np.concatenate([outer, hole]).astype(np.float32) + np.float32(0.4)
    off = [0, 300, 337]
    q = np.concatenate([[[0, 0], [1e-6, 0], [0, 0.01], [25.0, 0], [0, -25.0]], rng.uniform(-40, 40, (2500, 2))])
    ref = oracle.ft2d(v, q, loop_off=off)
    got = run2d(torch_dev, v, q, off, precision=prec)
    assert rel_err(got, ref, ref[0]) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_c1_star64_full_grid(torch_dev, prec):
    w = synth.workload_c1()
    ref = oracle.ft2d(w.verts, w.q)
    got = run2d(torch_dev, w.verts, w.q, precision=prec)
    iz = np.flatnonzero(np.all(w.q == 0, axis=1))[0]
    assert rel_err(got, ref, ref[iz]) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_c2_icosphere5_full_grid_sampled(torch_dev, prec):
    """Full 64^3 grid on the GPU in the default launch; the oracle checks 2,048 sampled Q."""
    w = synth.workload_c2()
    got = run3d(torch_dev, w.verts, w.faces, w.q, precision=prec)
    rng = np.random.default_rng(2)
    idx = np.concatenate([np.flatnonzero(np.all(w.q == 0, axis=1)), rng.choice(w.q.shape[0], 2047, replace=False)])
    ref = oracle.ft3d(w.verts, w.faces, w.q[idx])
    assert rel_err(got[idx], ref, ref[0]) < TOL[prec]
    assert np.all(np.isfinite(got))


def test_c5_full_size_sampled(torch_dev):
    """1.31M-face mesh on the full 128^3 grid in the benchmark's launch: the FP32 path and the plain
    FP64 GPU path against the oracle on the seeded 4,096-point Q subsample (Q = 0 included), every
    point within the FP32 / FP64 bar of the volume; the FP32 path also against the FP64 GPU path there."""
    torch, dev = torch_dev
    w = synth.workload_c5()
    got = run3d(torch_dev, w.verts, w.faces, w.q)
    assert np.all(np.isfinite(got))
    sub = synth.c5_subsample_indices(w.q)
    assert sub.size == 4096 and np.any(np.all(w.q[sub] == 0, axis=1))
    ref = oracle.ft3d(w.verts, w.faces, w.q[sub])
    vol = ref[np.flatnonzero(np.all(w.q[sub] == 0, axis=1))[0]].real
    assert rel_err(got[sub], ref, vol) < TOL["fp32"]
    got64 = run3d(torch_dev, w.verts, w.faces, w.q[sub], precision="fp64")
    assert rel_err(got64, ref, vol) < TOL["fp64"]
    assert rel_err(got[sub], got64, vol) < TOL["fp32"]


def test_bitwise_determinism_and_split_independence(torch_dev, rng):
    v, f = synth.perturbed_icosphere(3, seed=8, amp=0.1)
    q = _q3_mix(rng, 5000, 30.0)
    a = run3d(torch_dev, v, f, q, k_splits=3)
    b = run3d(torch_dev, v, f, q, k_splits=3)
    assert np.array_equal(a, b)
    # another launch shape keeps the per-Q summation order (it depends only on the chunking) but
    # groups other Q points into a warp, and the 3D branch is chosen per warp: rounding-level only
    c = run3d(torch_dev, v, f, q, k_splits=3, q_per_thread=1, block_threads=128)
    assert rel_err(c, a, a[0]) < 1e-6
    # in 2D there is no per-warp branch choice that changes the arithmetic: bitwise equal
    v2 = synth.star_polygon(300, seed=3)
    q2 = rng.uniform(-40, 40, (3000, 2))
    d2 = run2d(torch_dev, v2, q2, k_splits=2)
    e2 = run2d(torch_dev, v2, q2, k_splits=2, q_per_thread=1, block_threads=128)
    assert np.array_equal(d2, e2)
    d = run3d(torch_dev, v, f, q, k_splits=7)
    assert rel_err(d, a, a[0]) < 1e-6


def test_empty_inputs(torch_dev):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v = torch.zeros(0, 3, dtype=torch.float32, device=dev)
    f = torch.zeros(0, 3, dtype=torch.int32, device=dev)
    q = torch.randn(17, 3, dtype=torch.float64, device=dev)
    out = pft.pft3d_mesh(v, f, q, check_status=True)
    assert torch.count_nonzero(out).item() == 0
    out = pft.pft3d_mesh(torch.ones(3, 3, device=dev), torch.tensor([[0, 1, 2]], dtype=torch.int32, device=dev),
                         torch.zeros(0, 3, dtype=torch.float64, device=dev), check_status=True)
    assert out.shape == (0, 2)


def test_device_detected_errors(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f = synth.icosphere(1)
    q = torch.from_numpy(rng.uniform(-3, 3, (64, 3))).to(dev)
    fb = f.copy()
    fb[5, 1] = v.shape[0] + 3
    with pytest.raises(pft.PFTError, match="index"):
        pft.pft3d_mesh(torch.from_numpy(v).to(dev), torch.from_numpy(fb).to(dev), q, check_status=True)
    vb = v.copy()
    vb[3, 2] = np.nan
    with pytest.raises(pft.PFTError, match="non-finite"):
        pft.pft3d_mesh(torch.from_numpy(vb).to(dev), torch.from_numpy(f).to(dev), q, check_status=True)
    p = torch.from_numpy(synth.star_polygon(20, seed=1)).to(dev)
    q2 = torch.zeros(8, 2, dtype=torch.float64, device=dev)
    bad = torch.tensor([0, 12, 9, 20], dtype=torch.int64, device=dev)   # not non-decreasing
    with pytest.raises(pft.PFTError, match="offsets"):
        pft.pft2d_polygons(p, q2, bad, check_status=True)
    # the workspace is reusable after an error: a clean call reports ok
    out = pft.pft3d_mesh(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev), q, check_status=True)
    assert torch.isfinite(out).all()


def test_main_kernel_events(torch_dev):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f = synth.icosphere(3)
    q = torch.from_numpy(synth.q_grid_3d(24, 20.0)).to(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    e1.record()           # materialise the event handles
    o = pft.make_options({"main_start_event": e0.cuda_event, "main_stop_event": e1.cuda_event})
    pft.pft3d_mesh(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev), q, options=o)
    torch.cuda.synchronize()
    assert e0.elapsed_time(e1) > 0.0
    assert pft.launch_count() >= 4


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_degenerate_faces_and_segments(torch_dev, prec, rng):
    """Zero-area faces (repeated or collinear corners) and zero-length segments (repeated vertices)
    contribute nothing: the results match the shapes without them."""
    v, f = synth.perturbed_icosphere(3, seed=6, amp=0.05)
    q = _q3_mix(rng, 800, 20.0)
    n = v.shape[0]
    v2 = np.concatenate([v, [[0.25, 0.5, 0.75], [0.5, 1.0, 1.5], [0.75, 1.5, 2.25]]]).astype(np.float32)
    extra = np.array([[0, 0, 5], [7, 3, 7], [n, n + 1, n + 2]] * 20, np.int32)
    ref = oracle.ft3d(v, f, q)
    got = run3d(torch_dev, v2, np.concatenate([f, extra]), q, precision=prec)
    assert rel_err(got, ref, ref[0]) < TOL[prec]
    p = synth.star_polygon(50, seed=8)
    p2 = np.repeat(p, 2, axis=0)                       # every vertex twice: 50 zero-length segments
    q2 = np.concatenate([[[0.0, 0.0]], rng.uniform(-30, 30, (600, 2))])
    ref2 = oracle.ft2d(p, q2)
    got2 = run2d(torch_dev, p2, q2, precision=prec)
    assert rel_err(got2, ref2, ref2[0]) < TOL[prec]


def test_far_from_the_origin(torch_dev, rng):
    """Shapes thousands of units from the origin, at Q that float32 cannot represent: the FP32 pair sums
    run at Q rounded to float in coordinates centred on the shape, and the translation phase e^{iQ.c},
    1/|Q|^2 and the small-|Q| FP64 series take the caller's Q (Q rounded to float would move the phase
    by |c| times the rounding, 3e-5 rad here).  Against the oracle within 1e-5 of F(0)."""
    q2 = np.concatenate([[[0.0, 0.0], [1e-5, -2e-5], [0.3, -0.2]], rng.uniform(-40, 40, (800, 2))])
    for c in ((2500.0, -1800.0), (90000.0, -60000.0)):
        v = synth.star_polygon(200, seed=8, center=c).astype(np.float32)
        ref = oracle.ft2d(v, q2)
        assert rel_err(run2d(torch_dev, v, q2), ref, ref[0]) < TOL["fp32"], c
    v, f = synth.perturbed_icosphere(3, seed=9, amp=0.05)
    v = (v.astype(np.float64) + np.array([1500.0, -2200.0, 800.0])).astype(np.float32)
    q3 = np.concatenate([[[0.0, 0.0, 0.0], [1e-5, 0.0, 2e-5], [0.3, -0.2, 0.1]], rng.uniform(-25, 25, (600, 3))])
    ref = oracle.ft3d(v, f, q3)
    assert rel_err(run3d(torch_dev, v, f, q3), ref, ref[0]) < TOL["fp32"]
