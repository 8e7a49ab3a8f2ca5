"""Host-side checks of libpft that need no GPU.

The shared library builds for sm_103a, loads, and exports every entry point
that include/pft.h declares; workspace sizing and argument validation answer
without touching a device.
"""
import ctypes
import os
import re

import pytest

from paper_2104_08309_gb300 import _capi
from paper_2104_08309_gb300 import build as pbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pft.h")


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return _capi.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pft\w+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("pft2d_polygons", "pft2d_polygons_batched", "pft3d_mesh", "pft2d_polygons_backward",
              "pft3d_mesh_backward", "pft_status"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # and the ctypes table covers exactly the declared set
    assert sorted(_capi.SIGNATURES) == declared_functions()


def test_options_struct_layout_matches_header():
    # int32 x5, float, two pointers (8-aligned at offset 24), int32[4]
    assert ctypes.sizeof(_capi.Options) == 24 + 16 + 16
    assert _capi.Options.main_start_event.offset == 24
    assert (_capi.Options.face_pairs.offset, _capi.Options.q_order.offset) == (40, 44)


def test_status_strings_and_version(lib):
    assert lib.pft_status_string(0) == b"ok"
    assert b"index" in lib.pft_status_string(2)
    assert lib.pft_status_string(999) == b"unknown status code"
    assert lib.pft_version() >= 100


def test_workspace_sizes(lib):
    o = _capi.Options()
    s3 = lib.pft3d_workspace_size(10242, 20480, 262144, ctypes.byref(o))
    assert s3 >= 256 + 20480 * 48 + 262144 * 16
    assert s3 % 256 == 0
    o64 = _capi.Options(precision=1)
    assert lib.pft3d_workspace_size(10242, 20480, 262144, ctypes.byref(o64)) > s3   # 96-byte records
    assert lib.pft2d_workspace_size(64, 1, 16384, None) >= 256 + 64 * 16 + 16384 * 16
    assert lib.pft3d_workspace_size(-1, 3, 3, None) == 0
    assert lib.pft3d_polymesh_workspace_size(8, 24, 6, 100, ctypes.byref(o)) >= s3 * 0 + 256 + 12 * 48
    assert lib.pft3d_polymesh_workspace_size(8, 17, 6, 100, ctypes.byref(o)) == 0     # < 3 indices per face
    bad = _capi.Options(face_series_tau=6.5)
    assert lib.pft3d_workspace_size(3, 1, 1, ctypes.byref(bad)) == 0
    # adjoint-side sizes: Q records (32 B) and small-row lists (4 B) per (polygon, Q) row, segment records
    # and FP64 partials per vertex; the adjoints run in FP32 only, so FP64 options size to 0
    nv, npol, nq = 2675209, 4096, 4096
    sb = lib.pft2d_batched_backward_workspace_size(nv, npol, nq, 0, ctypes.byref(o))
    assert sb >= 256 + 36 * npol * nq + 16 * nv + 32 * nv and sb % 256 == 0
    assert lib.pft2d_batched_backward_workspace_size(nv, npol, nq, 0, ctypes.byref(o64)) == 0
    assert lib.pft2d_batched_backward_workspace_size(-1, npol, nq, 0, ctypes.byref(o)) == 0
    # per-polygon Q lists: n_q rows in all instead of n_polys x n_q
    sp = lib.pft2d_batched_backward_workspace_size(nv, npol, nq * 16, 1, ctypes.byref(o))
    assert 256 + 36 * nq * 16 + 16 * nv <= sp < sb
    sq = lib.pft3d_qgrad_workspace_size(40992, 81920, 32768, ctypes.byref(o))
    assert sq >= 256 + 81920 * 48 + 32768 * 32 and sq % 256 == 0
    assert lib.pft3d_qgrad_workspace_size(40992, 81920, 32768, ctypes.byref(o64)) == 0


def test_q_order_option_and_workspace(lib):
    """The Q ordering adds workspace only where it runs (two blocks of Q points and about 1e9 pairs
    or more, PFT_Q_TILED); PFT_Q_AS_GIVEN never orders; other values are refused."""
    tiled, given = _capi.Options(), _capi.Options(q_order=1)
    big = lib.pft3d_workspace_size(655362, 1310720, 2097152, ctypes.byref(tiled))
    plain = lib.pft3d_workspace_size(655362, 1310720, 2097152, ctypes.byref(given))
    assert big - plain >= 2097152 * (4 + 16) + lib.pft_q_order_workspace_size(0)
    assert big - plain >= lib.pft_q_order_workspace_size(2097152)
    # a small problem (1e6 pairs) is not ordered
    assert (lib.pft2d_workspace_size(64, 1, 16384, ctypes.byref(tiled))
            == lib.pft2d_workspace_size(64, 1, 16384, ctypes.byref(given)))
    assert lib.pft3d_workspace_size(10, 16, 100, ctypes.byref(_capi.Options(q_order=2))) == 0
    assert lib.pft3d_workspace_size(10, 16, 100, ctypes.byref(_capi.Options(q_order=-1))) == 0
    assert lib.pft_q_order_workspace_size(-1) == 0
    # pft_q_order checks its arguments before any device work
    fake = ctypes.c_void_p(256)
    assert lib.pft_q_order(fake, 10, 4, 4, 128, fake, fake, 1 << 20, None) == 1             # dim
    assert lib.pft_q_order(fake, 10, 3, 3, 128, fake, fake, 1 << 20, None) == 7             # R
    assert lib.pft_q_order(fake, 10, 3, 4, 64, fake, fake, 1 << 20, None) == 7              # NT
    assert lib.pft_q_order(None, 10, 3, 4, 128, fake, fake, 1 << 20, None) == 1
    assert lib.pft_q_order(fake, 10, 3, 4, 128, fake, fake, 16, None) == 4                  # workspace
    assert lib.pft_q_order(fake, 0, 3, 4, 128, None, None, 0, None) == 0                     # nothing to do


def test_batched_default_launch_shape(lib):
    """Batched FP32 calls default to one block of 512 threads (4 Q points each) on a shared Q set of
    4 x 512 points or more, else to 4 x 128; FP64 keeps 1 x 128.  Seen here through the plan's item
    count (polygons x Q tiles of R x NT points) in the workspace size."""
    npol = 1000
    off = (ctypes.c_int64 * (npol + 1))(*[16 * i for i in range(npol + 1)])
    nv = 16 * npol

    def size(n_q, q_off=None, **kw):
        o = _capi.Options(**kw)
        return lib.pft2d_batched_workspace_size(nv, off, npol, q_off, n_q, ctypes.byref(o))

    assert size(4096) == size(4096, q_per_thread=4, block_threads=512)
    assert size(4096) < size(4096, q_per_thread=4, block_threads=128)
    assert size(2047) == size(2047, q_per_thread=4, block_threads=128)       # below 4 x 512 points
    qo = (ctypes.c_int64 * (npol + 1))(*[5 * i for i in range(npol + 1)])
    assert size(5 * npol, qo) == size(5 * npol, qo, q_per_thread=4, block_threads=128)   # per-polygon lists
    assert size(4096, precision=1) == size(4096, precision=1, q_per_thread=1, block_threads=128)
    assert size(4096, q_per_thread=2, block_threads=512) == 0               # 512 threads: 4 Q points only
    assert size(4096, precision=1, q_per_thread=1, block_threads=512) == 0
    mo = (ctypes.c_int64 * (npol + 1))(*[20 * i for i in range(npol + 1)])
    o, o512 = _capi.Options(), _capi.Options(q_per_thread=4, block_threads=512)
    assert (lib.pft3d_batched_workspace_size(20 * npol, mo, npol, None, 4096, ctypes.byref(o))
            == lib.pft3d_batched_workspace_size(20 * npol, mo, npol, None, 4096, ctypes.byref(o512)))


def test_argument_errors_are_synchronous(lib):
    """Rejected before any device work: negative sizes, bad options, short or misaligned workspace."""
    fake = ctypes.c_void_p(256)     # never dereferenced: every call below fails its host checks
    o = _capi.Options()
    assert lib.pft3d_mesh(fake, -1, fake, 1, fake, 1, fake, fake, 1 << 20, ctypes.byref(o), None) == 1
    assert lib.pft3d_mesh(fake, 3, fake, 1, fake, 1, fake, None, 1 << 20, ctypes.byref(o), None) == 4
    assert lib.pft3d_mesh(fake, 3, fake, 1, fake, 1, fake, ctypes.c_void_p(256 + 8), 1 << 20,
                          ctypes.byref(o), None) == 4
    assert lib.pft3d_mesh(fake, 3, fake, 1, fake, 1, fake, fake, 16, ctypes.byref(o), None) == 4
    bad = _capi.Options(q_per_thread=3)
    assert lib.pft3d_mesh(fake, 3, fake, 1, fake, 1, fake, fake, 1 << 20, ctypes.byref(bad), None) == 7
    bad = _capi.Options(precision=1, q_per_thread=4, block_threads=256)      # FP64: at most 2 Q per thread
    assert lib.pft3d_mesh(fake, 3, fake, 1, fake, 1, fake, fake, 1 << 20, ctypes.byref(bad), None) == 7
    bad = _capi.Options(precision=5)
    assert lib.pft2d_polygons(fake, 3, fake, 1, fake, 1, fake, fake, 1 << 20, ctypes.byref(bad), None) == 1
    assert lib.pft2d_polygons(None, 3, fake, 1, fake, 1, fake, fake, 1 << 20, None, None) == 1
    # the bounded-wait self-test checks its arguments before any device work
    assert lib.pft_selftest_wait(None, 256, 64, 0, None) == 4
    assert lib.pft_selftest_wait(ctypes.c_void_p(256 + 8), 256, 64, 0, None) == 4
    assert lib.pft_selftest_wait(fake, 16, 64, 0, None) == 4
    assert lib.pft_selftest_wait(fake, 256, 0, 0, None) == 1
    assert lib.pft_selftest_wait(fake, 256, (1 << 20) + 1, 0, None) == 1
    assert lib.pft_selftest_wait(fake, 256, 64, 2, None) == 1


def test_python_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    import paper_2104_08309_gb300 as pft
    with pytest.raises(ValueError, match="CUDA"):
        pft.pft3d_mesh(torch.zeros(3, 3), torch.zeros(1, 3, dtype=torch.int32), torch.zeros(1, 3, dtype=torch.float64))
