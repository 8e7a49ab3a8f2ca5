"""Q-sharding on one GPU: the slabs shard.q_slab gives 3 ranks, each transformed by its own
library call (as each rank would on its own GPU), concatenated in Q order, against the oracle and
the unsharded call; per-slab adjoints summed in rank order against the unsharded adjoint."""
import numpy as np
import pytest

import oracle
from paper_2104_08309_gb300 import shard, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08309_gb300 import build as pbuild
    pbuild.build()
    return torch, torch.device("cuda:0")


def test_three_slabs_on_one_gpu(torch_dev, rng):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    v, f = synth.perturbed_icosphere(4, seed=31, amp=0.05)
    q = np.concatenate([[[0.0, 0.0, 0.0]], rng.uniform(-30, 30, (5000, 3))])
    vd, fd, qd = (torch.from_numpy(a).to(dev) for a in (v, f, q))
    whole = pft.pft3d_mesh(vd, fd, qd, check_status=True)
    parts, grads = [], []
    g = torch.from_numpy(rng.normal(size=(q.shape[0], 2))).to(dev)
    for r in range(3):
        a, b = shard.q_slab(q.shape[0], r, 3)
        parts.append(pft.pft3d_mesh(vd, fd, qd[a:b].contiguous(), check_status=True))
        grads.append(pft.pft3d_mesh_backward(vd, fd, qd[a:b].contiguous(), g[a:b].contiguous()).double())
    joined = torch.cat(parts).cpu().numpy()
    vol = abs(whole[0, 0].item())
    ref = oracle.ft3d(v, f, q)
    assert np.max(np.abs(joined[:, 0] + 1j * joined[:, 1] - ref)) < 1e-5 * vol
    assert np.max(np.abs(joined - whole.cpu().numpy())) < 1e-6 * vol
    gsum = (grads[0] + grads[1] + grads[2]).cpu().numpy()
    gwhole = pft.pft3d_mesh_backward(vd, fd, qd, g).double().cpu().numpy()
    assert np.max(np.abs(gsum - gwhole)) < 1e-5 * np.max(np.abs(gwhole))
