"""Q-sharding of one transform over ranks (shard.py): the slab partition, and the two collectives
(gathering the per-rank slabs of a per-Q result; summing per-rank vertex gradients in rank order)
run as gloo ranks on CPU.  The per-rank transform is the library's job on a GPU; here each rank
fills its slab with a stand-in function of its Q rows, so that the gathered result can be checked
row by row."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2104_08309_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("n_q,world,align", [(0, 3, 512), (1, 4, 512), (2097152, 8, 512), (1000, 3, 64),
                                             (4097, 2, 512), (10, 1, 4), (13, 5, 1)])
def test_slabs_partition_the_q_rows(n_q, world, align):
    slabs = [shard.q_slab(n_q, r, world, align) for r in range(world)]
    assert slabs[0][0] == 0 and slabs[-1][1] == n_q
    for (a, b), (c, _) in zip(slabs, slabs[1:]):
        assert b == c and a <= b
    for a, b in slabs:
        assert a % align == 0 or a == n_q
    units = [-(-(b - a) // align) for a, b in slabs]
    assert max(units) - min(units) <= 1 or n_q < align * world


def test_slab_arguments_checked():
    for bad in ((10, 2, 2, 4), (10, -1, 2, 4), (10, 0, 0, 4), (-1, 0, 1, 4), (10, 0, 1, 0)):
        with pytest.raises(ValueError):
            shard.q_slab(*bad)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n_q, align = 1300, 64
        q = torch.arange(3 * n_q, dtype=torch.float64).reshape(n_q, 3)
        a, b = shard.q_slab(n_q, rank, world, align)
        local = torch.stack([q[a:b, 0] * 2.0, -q[a:b, 2]], dim=1)       # stand-in per-Q result
        full = shard.gather_slabs(local, n_q, align)
        grad = torch.full((7, 3), float(rank + 1), dtype=torch.float64) / 3.0   # per-rank vertex gradient
        total = shard.sum_over_ranks(grad)
        results[rank] = (full.numpy(), total.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_gather_and_sum(world):
    mgr = mp.get_context("spawn").Manager()
    results = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), results), nprocs=world, start_method="spawn")
    n_q = 1300
    q = np.arange(3 * n_q, dtype=np.float64).reshape(n_q, 3)
    want = np.stack([q[:, 0] * 2.0, -q[:, 2]], axis=1)
    expect_sum = sum(np.full((7, 3), float(r + 1)) / 3.0 for r in range(world))
    for r in range(world):
        full, total = results[r]
        assert np.array_equal(full, want)                # every row from its owner, in Q order
        assert np.array_equal(total, results[0][1])      # the same sum on every rank
        assert np.allclose(total, expect_sum, rtol=0, atol=1e-15)


def test_single_process_is_identity():
    x = torch.randn(5, 2)
    assert shard.gather_slabs(x, 5) is x
    assert shard.sum_over_ranks(x) is x
