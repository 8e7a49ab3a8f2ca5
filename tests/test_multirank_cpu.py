"""The N > 1 host logic of bench.py on CPU with two gloo ranks: each rank transforms its own mesh
(independent problems, no collective on the data path), the timings are reduced to the slowest
rank's, and the whole-job rate counts every rank's pairs over that time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2104_08309_gb300 import synth
        assert bench.dist_env() == (rank, rank, world)
        # each rank its own problem: same size, different vertices
        v, _ = synth.perturbed_icosphere(2, seed=bench.replica_seed(rank), amp=0.05)
        gathered = [None] * world
        dist.all_gather_object(gathered, v.tobytes())
        # per-rank step times: the reduction returns the slowest on every rank
        mine = [10.0 + rank, 3.0 - rank]
        red = bench.max_over_ranks(mine, torch.device("cpu"))
        results[rank] = (gathered[0] != gathered[1], red)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), results), nprocs=world, start_method="spawn")
    for r in range(world):
        distinct, red = results[r]
        assert distinct
        assert red == [11.0, 3.0]


def test_single_process_paths():
    import bench
    assert bench.max_over_ranks([1.5, 2.5], None) == [1.5, 2.5]      # no process group: identity
    assert bench.whole_job_rate(4, 1e12, 2000.0) == pytest.approx(2000.0)
    assert bench.replica_seed(0) == 5 and bench.replica_seed(3) == 8
    assert np.isclose(bench.whole_job_rate(1, 2.75e12, 4160.0), 661.06, rtol=1e-4)
