"""Autotuner: selection, caching and keys (CPU, with a fake timer) and a real run on the GPU."""
import json

import numpy as np
import pytest

from paper_2104_08309_gb300 import autotune


def test_bucket_and_key():
    assert autotune.bucket(1, 2, 1000) == "0x1x10"
    k1 = autotune.make_key("GB300", "mesh3d", "fp32", 1310720, 2097152)
    k2 = autotune.make_key("GB300", "mesh3d", "fp32", 1300000, 2100000)
    assert k1 == k2                       # same size class
    assert k1 != autotune.make_key("GB300", "mesh3d", "fp64", 1310720, 2097152)


def test_pick_is_fastest_and_deterministic():
    t = {(1, 128): 3.0, (2, 128): 2.0, (4, 256): 2.0, (8, 256): None}
    assert autotune.pick(t) == (2, 128)
    with pytest.raises(RuntimeError):
        autotune.pick({(1, 128): None})


def test_tune_caches_choice(tmp_path):
    path = str(tmp_path / "tune.json")
    calls = []

    def run_for(c):
        if c == (8, 256):
            raise ValueError("unsupported")
        return lambda: calls.append(c)

    fake = {(1, 128): 5.0, (2, 128): 1.5, (4, 128): 2.0}
    timer = lambda fn: (fn(), fake.get(calls[-1], 9.0))[1]
    best = autotune.tune("k", run_for, autotune.CANDIDATES_FP32, timer=timer, path=path)
    assert best == (2, 128)
    data = json.load(open(path))
    assert data["k"]["best"] == [2, 128] and "8x256" not in data["k"]["ms"]
    n = len(calls)
    assert autotune.tune("k", run_for, autotune.CANDIDATES_FP32, timer=timer, path=path) == (2, 128)
    assert len(calls) == n                # served from the cache


@pytest.mark.gpu
def test_tune_batched_on_gpu(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_2104_08309_gb300 as pft
    from paper_2104_08309_gb300 import build as pbuild, synth
    pbuild.build()
    dev = torch.device("cuda:0")
    v, off = synth.batched_star_polygons(64, seed=9, nmin=8, nmax=512)
    q = synth.q_grid_2d(32, 20.0)
    vd, qd = torch.from_numpy(v).to(dev), torch.from_numpy(q).to(dev)
    opts = autotune.tune_batched2d(vd, off, qd, path=str(tmp_path / "t.json"))
    assert (opts["q_per_thread"], opts["block_threads"]) in autotune.CANDIDATES_FP32
    out = pft.pft2d_polygons_batched(vd, off, qd, options=opts, check_status=True).cpu().numpy()
    ref = oracle.ft2d_batched(v, off, q[:50])
    got = out[:, :50, 0] + 1j * out[:, :50, 1]
    areas = np.abs(ref[:, np.flatnonzero(np.all(q[:50] == 0, axis=1))]) if np.any(np.all(q[:50] == 0, axis=1)) \
        else np.array([[abs(oracle.ft2d(v[off[i]:off[i + 1]], [[0, 0]])[0])] for i in range(64)])
    assert np.all(np.max(np.abs(got - ref), axis=1) / areas[:, 0] < 1e-5)
