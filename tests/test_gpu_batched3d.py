"""Batched 3D (many closed triangle meshes in one persistent launch) against the FP64 oracle,
per mesh, through the C ABI: shared and per-mesh Q sets, meshes larger than one 4,096-face chunk,
small |Q|, CUDA-graph replay, plan mismatches.

Tolerances relative to each mesh's volume: FP32 path 1e-5, FP64 path 1e-12.
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


def _c(a):
    a = a.detach().cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def _mesh(v, f, off, i):
    """Mesh i of a batch with its own vertex array (the oracle's input)."""
    fi = f[off[i]:off[i + 1]]
    used = np.unique(fi)
    remap = np.full(v.shape[0], -1, dtype=np.int64)
    remap[used] = np.arange(used.size)
    return v[used], remap[fi].astype(np.int32)


def _q_mix(rng, n, scale):
    return np.concatenate([[[0, 0, 0], [1e-4, 0, 2e-4], [0, 0, 0.2], [3.0, 0, 0], [0, -5.0, 1.0]],
                           rng.uniform(-scale, scale, (n, 3))])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_shared_q_vs_oracle(torch_dev, prec, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f, off = synth.mesh_batch(12, seed=3, levels=(0, 1, 2, 3))
    # one mesh above a 4,096-face chunk: a level-5 icosphere (20,480 faces, 5 chunks)
    v5, f5 = synth.perturbed_icosphere(5, seed=9, amp=0.03, radius=0.7)
    f = np.concatenate([f, f5 + v.shape[0]]).astype(np.int32)
    v = np.concatenate([v, v5 + np.float32(0.25)]).astype(np.float32)
    off = np.append(off, off[-1] + f5.shape[0])
    q = _q_mix(rng, 700, 25.0)
    got = _c(pft.pft3d_meshes_batched(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev), off,
                                      torch.from_numpy(q).to(dev), options={"precision": prec}, check_status=True))
    assert got.shape == (off.size - 1, q.shape[0])
    for i in range(off.size - 1):
        vi, fi = _mesh(v, f, off, i)
        ref = oracle.ft3d(vi, fi, q)
        assert np.max(np.abs(got[i] - ref)) / abs(ref[0]) < TOL[prec], (i, prec)


def test_per_mesh_q_sets(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f, off = synth.mesh_batch(9, seed=5)
    counts = rng.integers(1, 400, off.size - 1)
    q_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    q = rng.uniform(-20, 20, (int(q_off[-1]), 3))
    q[q_off[:-1]] = 0.0                                   # every mesh's first Q is 0 -> its volume
    got = _c(pft.pft3d_meshes_batched(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev), off,
                                      torch.from_numpy(q).to(dev), q_off, check_status=True))
    for i in range(off.size - 1):
        vi, fi = _mesh(v, f, off, i)
        sl = slice(q_off[i], q_off[i + 1])
        ref = oracle.ft3d(vi, fi, q[sl])
        assert np.max(np.abs(got[sl] - ref)) / abs(ref[0]) < TOL["fp32"], i


def test_full_batch_graph_replay_and_sampled_parity(torch_dev):
    """1,024 meshes (80..5,120 faces, 1.68M faces) on a shared 32^3 grid: one prepared schedule
    captured in a CUDA graph and replayed (bitwise equal to the direct call); 12 seeded meshes
    against the oracle on every Q."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f, off = synth.mesh_batch(1024, seed=21)
    q = synth.q_grid_3d(32, 30.0)
    vd, fd, qd = (torch.from_numpy(a).to(dev) for a in (v, f, q))
    offd = torch.from_numpy(off).to(dev)
    prep = pft.pft3d_batched_prepare(off, q.shape[0], device=dev)
    direct = pft.pft3d_meshes_batched(vd, fd, offd, qd, prepared=prep, check_status=True).clone()
    out = torch.empty(off.size - 1, q.shape[0], 2, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        pft.pft3d_meshes_batched(vd, fd, offd, qd, prepared=prep, out=out)
    torch.cuda.current_stream(dev).wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pft.pft3d_meshes_batched(vd, fd, offd, qd, prepared=prep, out=out)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert pft.pft_status(prep.ws) == 0
    assert torch.equal(out, direct)
    got = _c(direct)
    rng = np.random.default_rng(22)
    for i in np.sort(rng.choice(off.size - 1, 12, replace=False)):
        vi, fi = _mesh(v, f, off, i)
        ref = oracle.ft3d(vi, fi, q)
        vol = abs(oracle.ft3d(vi, fi, [[0.0, 0.0, 0.0]])[0])
        assert np.max(np.abs(got[i] - ref)) / vol < TOL["fp32"], i


def test_plan_mismatch_and_bad_offsets(torch_dev):
    torch, dev = torch_dev
    import ctypes
    import paper_2104_08309_gb300 as pft
    v, f, off = synth.mesh_batch(4, seed=7, levels=(1,))
    q = torch.ones(10, 3, dtype=torch.float64, device=dev)
    vd, fd = torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev)
    prep2 = pft.pft2d_batched_prepare(np.array([0, 3, 7]), 10, device=dev)     # a 2D plan
    lib = pft.load()
    out = torch.empty(4, 10, 2, dtype=torch.float64, device=dev)
    offd = torch.from_numpy(off).to(dev)
    rc = lib.pft3d_meshes_batched(vd.data_ptr(), v.shape[0], fd.data_ptr(), f.shape[0], offd.data_ptr(), 4,
                                  q.data_ptr(), None, 10, out.data_ptr(), prep2.ws.data_ptr(), prep2.ws.numel(),
                                  ctypes.byref(prep2.plan), None)
    assert rc == 1
    # device offsets that differ from the prepared ones: reported, nothing read out of range
    prep = pft.pft3d_batched_prepare(off, 10, device=dev)
    bad = off.copy()
    bad[2] += 3
    pft.pft3d_meshes_batched(vd, fd, torch.from_numpy(bad).to(dev), q, prepared=prep, out=out)
    assert pft.pft_status(prep.ws) == 8


def test_empty_mesh_in_batch(torch_dev, rng):
    """A mesh with no faces between two others: its transform is 0 everywhere, the others unchanged."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f, off = synth.mesh_batch(2, seed=8, levels=(2,))
    off3 = np.array([0, off[1], off[1], off[2]], dtype=np.int64)
    q = _q_mix(rng, 300, 15.0)
    got = _c(pft.pft3d_meshes_batched(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev), off3,
                                      torch.from_numpy(q).to(dev), check_status=True))
    assert np.all(got[1] == 0)
    for k, i in ((0, 0), (2, 1)):
        vi, fi = _mesh(v, f, off, i)
        ref = oracle.ft3d(vi, fi, q)
        assert np.max(np.abs(got[k] - ref)) / abs(ref[0]) < TOL["fp32"]


def test_default_shape_on_a_large_shared_grid(torch_dev):
    """On a shared Q set of 4 x 512 points or more the default launch shape is one block of 512
    threads per SM (the same result bit for bit as asking for it).  The series form of a face is
    chosen per warp from the largest P over the warp's Q points, and without the library's Q order
    (too few pairs here) a warp of another block size holds other Q points: the 4 x 128 shape then
    agrees to rounding, and both agree with the oracle on sampled meshes."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f, off = synth.mesh_batch(24, seed=6, levels=(1, 2, 3))
    q = synth.q_grid_3d(14, 20.0)                   # 2,744 points, one ragged 2,048-point tile
    vd, fd, qd = (torch.from_numpy(a).to(dev) for a in (v, f, q))
    outs = {}
    for name, opts in (("default", None), ("4x128", {"q_per_thread": 4, "block_threads": 128}),
                       ("4x512", {"q_per_thread": 4, "block_threads": 512})):
        prep = pft.pft3d_batched_prepare(off, q.shape[0], options=opts, device=dev)
        outs[name] = pft.pft3d_meshes_batched(vd, fd, torch.from_numpy(off).to(dev), qd, prepared=prep,
                                              check_status=True).clone()
    assert torch.equal(outs["default"], outs["4x512"])
    got, alt = _c(outs["default"]), _c(outs["4x128"])
    for i in range(off.size - 1):
        vol = abs(got[i][np.flatnonzero(np.all(q == 0, axis=1))[0]])
        assert np.max(np.abs(got[i] - alt[i])) / vol < 1e-6, i
    for i in (0, 11, 23):
        vi, fi = _mesh(v, f, off, i)
        ref = oracle.ft3d(vi, fi, q)
        vol = abs(oracle.ft3d(vi, fi, [[0.0, 0.0, 0.0]])[0])
        assert np.max(np.abs(got[i] - ref)) / vol < TOL["fp32"], i


def test_far_from_the_origin_phase_reduction(torch_dev, rng):
    """Meshes centred about 2e3 and 6e4 from the origin: Q.c reaches about 1e5 rad (the FP32 finish's
    float-float reduction) and about 3e6 rad (beyond 2^20 rad: the FP64 finish); a 20,480-face mesh
    (5 chunks) goes through the multi-chunk finish.  Each mesh against the oracle within 1e-5 of its
    volume."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    shifts = [((1500.0, -2200.0, 800.0), 2), ((-1200.0, 900.0, 1700.0), 5), ((40000.0, 30000.0, -50000.0), 1)]
    vs, fs, off = [], [], [0]
    base = 0
    for k, (sh, level) in enumerate(shifts):
        vk, fk = synth.perturbed_icosphere(level, seed=50 + k, amp=0.03)
        vs.append((vk.astype(np.float64) + np.array(sh)).astype(np.float32))
        fs.append(fk + base)
        base += vk.shape[0]
        off.append(off[-1] + fk.shape[0])
    v = np.concatenate(vs).astype(np.float32)
    f = np.concatenate(fs).astype(np.int32)
    off = np.array(off, dtype=np.int64)
    q = _q_mix(rng, 400, 25.0)
    got = _c(pft.pft3d_meshes_batched(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev), off,
                                      torch.from_numpy(q).to(dev), check_status=True))
    for i in range(off.size - 1):
        vi, fi = _mesh(v, f, off, i)
        ref = oracle.ft3d(vi, fi, q)
        assert np.max(np.abs(got[i] - ref)) / abs(ref[0]) < TOL["fp32"], i


def test_per_mesh_q_sets_one_block_per_sm(torch_dev, rng):
    """Per-mesh Q lists with one block of 512 threads per SM asked for (the 2,048-point Q tiles of the
    short lists mostly empty), against the oracle."""
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f, off = synth.mesh_batch(9, seed=7)
    counts = rng.integers(1, 2500, off.size - 1)
    q_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    q = rng.uniform(-20, 20, (int(q_off[-1]), 3))
    q[q_off[:-1]] = 0.0
    got = _c(pft.pft3d_meshes_batched(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev), off,
                                      torch.from_numpy(q).to(dev), q_off,
                                      options={"q_per_thread": 4, "block_threads": 512}, check_status=True))
    for i in range(off.size - 1):
        vi, fi = _mesh(v, f, off, i)
        sl = slice(q_off[i], q_off[i + 1])
        ref = oracle.ft3d(vi, fi, q[sl])
        assert np.max(np.abs(got[sl] - ref)) / abs(ref[0]) < TOL["fp32"], i
