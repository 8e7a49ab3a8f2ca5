"""Paired faces (face_pairs option): faces 2k, 2k+1 share their first edge, whose sinc the FP32
kernel evaluates once for both where a warp takes the edge sum for both.  Checked against the
oracle (FP32 1e-5, FP64 1e-12 of the volume) and against the unpaired call, at face_series_tau 1
(mostly edge sums), 3 and 6 (mostly series, mixed pairs); a pair that does not share its first edge
is reported and left out."""
import ctypes

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


def _run(td, v, f, q, **opts):
    torch, dev = td
    import paper_2104_08309_gb300 as pft
    out = pft.pft3d_mesh(torch.from_numpy(v).to(dev), torch.from_numpy(np.ascontiguousarray(f)).to(dev),
                         torch.from_numpy(q).to(dev), options=opts, check_status=True).cpu().numpy()
    return out[:, 0] + 1j * out[:, 1]


@pytest.mark.parametrize("tau", [1.0, 3.0, 6.0])
@pytest.mark.parametrize("r", [2, 4])
def test_paired_faces_vs_oracle_and_unpaired(torch_dev, rng, tau, r):
    import paper_2104_08309_gb300 as pft
    v, f = synth.perturbed_icosphere(4, seed=19, amp=0.08)
    v = (v + np.array([0.25, -0.125, 0.0625], np.float32)).astype(np.float32)
    fp, n = pft.pair_faces(f)
    assert n > 2400
    q = np.concatenate([[[0, 0, 0], [1e-4, 0, 2e-4], [0, 0, 5.0], [7.0, 0, 0]], rng.uniform(-45, 45, (6000, 3))])
    ref = oracle.ft3d(v, f, q)
    vol = ref[0].real
    paired = _run(torch_dev, v, fp, q, face_pairs=n, face_series_tau=tau, q_per_thread=r)
    plain = _run(torch_dev, v, fp, q, face_series_tau=tau, q_per_thread=r)
    assert np.max(np.abs(paired - ref)) < 1e-5 * vol
    assert np.max(np.abs(paired - plain)) < 1e-6 * vol
    f64 = _run(torch_dev, v, fp, q, face_pairs=n, precision="fp64")
    assert np.max(np.abs(f64 - ref)) < 1e-12 * vol


def test_bad_pair_reported_and_left_out(torch_dev):
    torch, dev = torch_dev
    import paper_2104_08309_gb300 as pft
    from paper_2104_08309_gb300 import _capi
    v, f = synth.perturbed_icosphere(2, seed=20, amp=0.05)
    fp, n = pft.pair_faces(f)
    bad = fp.copy()
    bad[3] = bad[3][[1, 2, 0]]                       # the second face of pair 1 rotated: first edges differ
    q = np.array([[1.0, 2.0, -0.5], [4.0, 0.0, 3.0]])
    vd, fd, qd = (torch.from_numpy(a).to(dev) for a in (v, bad, q))
    lib = _capi.load()
    o = _capi.Options()
    o.face_pairs = n
    nb = lib.pft3d_workspace_size(v.shape[0], bad.shape[0], 2, ctypes.byref(o))
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    out = torch.empty(2, 2, dtype=torch.float64, device=dev)
    assert lib.pft3d_mesh(vd.data_ptr(), v.shape[0], fd.data_ptr(), bad.shape[0], qd.data_ptr(), 2, out.data_ptr(),
                          ws.data_ptr(), nb, ctypes.byref(o), None) == 0
    assert lib.pft_status(ws.data_ptr(), None) == 10
    # the pair is left out: the rest equals the transform of the surface without those two faces
    keep = np.delete(bad, [2, 3], axis=0)
    ref = oracle.ft3d(v, keep, q)
    got = out.cpu().numpy()
    assert np.max(np.abs(got[:, 0] + 1j * got[:, 1] - ref)) < 1e-5 * abs(oracle.ft3d(v, f, [[0, 0, 0]])[0])
    # options the paired kernel has no shape for, and more pairs than faces allow
    o.q_per_thread = 8
    assert lib.pft3d_mesh(vd.data_ptr(), v.shape[0], fd.data_ptr(), bad.shape[0], qd.data_ptr(), 2, out.data_ptr(),
                          ws.data_ptr(), nb, ctypes.byref(o), None) == 7
    o.q_per_thread = 0
    o.face_pairs = bad.shape[0] // 2 + 1
    assert lib.pft3d_mesh(vd.data_ptr(), v.shape[0], fd.data_ptr(), bad.shape[0], qd.data_ptr(), 2, out.data_ptr(),
                          ws.data_ptr(), nb, ctypes.byref(o), None) == 1
