"""The allocation-free entry point pft3d_mesh_noalloc, called through the C ABI.

It serves callers that cannot allocate device memory when they need a
transform (stream capture, host applications that own all device memory).
Its result must equal pft3d_mesh with a caller workspace bit for bit, on two
calls in a row (the second sees the first call's leftovers in the shared
scratch), and
problems too large for its fixed 32 MiB scratch must be refused up front.
This file is named to run last, so a failure here cannot hide other tests.
"""
import ctypes

import numpy as np
import pytest

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


def test_noalloc_matches_workspace_call_twice(torch_dev):
    torch, dev = torch_dev
    from paper_2104_08309_gb300 import _capi
    lib = _capi.load()
    v, f = synth.perturbed_icosphere(4, seed=3, amp=0.05)                 # 5,120 faces
    q = synth.q_grid_3d(24, 30.0)                                          # 13,824 Q incl. Q = 0
    vd, fd, qd = (torch.from_numpy(a).to(dev) for a in (v, f, q))
    stream = torch.cuda.current_stream(dev).cuda_stream
    opts = _capi.Options()
    need = lib.pft3d_workspace_size(v.shape[0], f.shape[0], q.shape[0], ctypes.byref(opts))
    assert 0 < need <= 32 << 20
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    ref = torch.empty(q.shape[0], 2, dtype=torch.float64, device=dev)
    assert lib.pft3d_mesh(vd.data_ptr(), v.shape[0], fd.data_ptr(), f.shape[0], qd.data_ptr(), q.shape[0],
                          ref.data_ptr(), ws.data_ptr(), need, ctypes.byref(opts), stream) == 0
    assert lib.pft_status(ws.data_ptr(), stream) == 0
    for call in range(2):
        out = torch.full((q.shape[0], 2), float("nan"), dtype=torch.float64, device=dev)
        rc = lib.pft3d_mesh_noalloc(vd.data_ptr(), v.shape[0], fd.data_ptr(), f.shape[0], qd.data_ptr(),
                                    q.shape[0], out.data_ptr(), ctypes.byref(opts), stream)
        assert rc == 0, (call, lib.pft_status_string(rc))
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        # the same kernels with the same launch plan in a fixed summation order: bit for bit
        assert torch.equal(out, ref), (call, (out - ref).abs().max().item())


def test_noalloc_with_the_q_order(torch_dev):
    """A problem large enough for the library's Q order (81,920 faces x 32^3 Q, 2.7e9 pairs) whose
    workspace, ordering scratch included, fits the fixed scratch: bitwise the workspace call."""
    torch, dev = torch_dev
    from paper_2104_08309_gb300 import _capi
    lib = _capi.load()
    v, f = synth.icosphere(6)
    q = synth.q_grid_3d(32, 30.0)
    vd, fd, qd = (torch.from_numpy(a).to(dev) for a in (v, f, q))
    stream = torch.cuda.current_stream(dev).cuda_stream
    tiled, given = _capi.Options(), _capi.Options(q_order=1)
    need = lib.pft3d_workspace_size(v.shape[0], f.shape[0], q.shape[0], ctypes.byref(tiled))
    assert lib.pft3d_workspace_size(v.shape[0], f.shape[0], q.shape[0], ctypes.byref(given)) < need <= 32 << 20
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    ref = torch.empty(q.shape[0], 2, dtype=torch.float64, device=dev)
    assert lib.pft3d_mesh(vd.data_ptr(), v.shape[0], fd.data_ptr(), f.shape[0], qd.data_ptr(), q.shape[0],
                          ref.data_ptr(), ws.data_ptr(), need, ctypes.byref(tiled), stream) == 0
    out = torch.full((q.shape[0], 2), float("nan"), dtype=torch.float64, device=dev)
    rc = lib.pft3d_mesh_noalloc(vd.data_ptr(), v.shape[0], fd.data_ptr(), f.shape[0], qd.data_ptr(),
                                q.shape[0], out.data_ptr(), ctypes.byref(tiled), stream)
    assert rc == 0, lib.pft_status_string(rc)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_noalloc_refuses_problems_beyond_its_scratch(torch_dev):
    torch, dev = torch_dev
    from paper_2104_08309_gb300 import _capi
    lib = _capi.load()
    fake = ctypes.c_void_p(256)          # never dereferenced: the size check comes first
    # 3M Q points: their partial sums alone (3e6 x 16 B = 45.8 MiB) exceed the 32 MiB
    rc = lib.pft3d_mesh_noalloc(fake, 3, fake, 1, fake, 3_000_000, fake, None, None)
    assert rc == 9
    assert b"32 MiB" in lib.pft_status_string(rc)
    # what pft3d_mesh refuses is refused with its code: a negative size, an unsupported launch shape
    assert lib.pft3d_mesh_noalloc(fake, -1, fake, 1, fake, 1, fake, None, None) == 1
    bad = _capi.Options()
    bad.q_per_thread = 3
    assert lib.pft3d_mesh_noalloc(fake, 3, fake, 1, fake, 1, fake, ctypes.byref(bad), None) == 7
