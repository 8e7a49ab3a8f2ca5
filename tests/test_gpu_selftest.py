"""The failure handling around the bulk copies, exercised on the GPU without a fault: a bounded
mbarrier wait that nothing completes runs out, sets the timeout bit of the status word and returns;
pft_status() reports PFT_ERR_TIMEOUT, and the context stays usable for the next transform."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2104_08309_gb300 import synth

pytestmark = pytest.mark.gpu

PFT_OK, PFT_ERR_TIMEOUT = 0, 6


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_08309_gb300 import build as pbuild
    pbuild.build()
    return torch, torch.device("cuda:0")


def test_bounded_wait_runs_out_and_reports(torch_dev):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    lib = pft.load()
    ws = torch.empty(512, dtype=torch.uint8, device=dev)
    assert ws.data_ptr() % 256 == 0
    st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    # nothing arrives: 4,096 polls of an incomplete phase, then the timeout bit
    assert lib.pft_selftest_wait(ctypes.c_void_p(ws.data_ptr()), ws.numel(), 4096, 0, st) == PFT_OK
    assert lib.pft_status(ctypes.c_void_p(ws.data_ptr()), st) == PFT_ERR_TIMEOUT
    # the block arrives first: the same wait succeeds and the (cleared) status stays clear
    assert lib.pft_selftest_wait(ctypes.c_void_p(ws.data_ptr()), ws.numel(), 4096, 1, st) == PFT_OK
    assert lib.pft_status(ctypes.c_void_p(ws.data_ptr()), st) == PFT_OK
    # the context is still usable: a transform right after matches the oracle
    v, f = synth.icosphere(2)
    q = np.random.default_rng(5).uniform(-8, 8, (300, 3))
    out = pft.pft3d_mesh(torch.from_numpy(v).to(dev), torch.from_numpy(f).to(dev),
                         torch.from_numpy(q).to(dev), check_status=True).cpu().numpy()
    ref = oracle.ft3d(v, f, q)
    assert np.max(np.abs(out[:, 0] + 1j * out[:, 1] - ref)) < 1e-5 * abs(ref).max()
