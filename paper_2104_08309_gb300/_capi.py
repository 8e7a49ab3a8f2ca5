"""ctypes declarations of libpft (include/pft.h).  Argument marshalling only.

The library is loaded from this package's ``_build/`` directory.  There is no
fallback: if the shared library is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpft.so")

PFT_OK = 0
PFT_FP32_COMPENSATED = 0
PFT_FP64 = 1

c_i64 = ctypes.c_int64
c_vp = ctypes.c_void_p
c_size = ctypes.c_size_t


class Options(ctypes.Structure):
    """pft_options: zero means default for every field."""
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("q_per_thread", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("k_splits", ctypes.c_int32),
        ("tile_items", ctypes.c_int32),
        ("face_series_tau", ctypes.c_float),
        ("main_start_event", ctypes.c_void_p),
        ("main_stop_event", ctypes.c_void_p),
        ("face_pairs", ctypes.c_int32),
        ("q_order", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 2),
    ]


# name -> (restype, argtypes); exactly the entry points include/pft.h declares.
SIGNATURES = {
    "pft2d_workspace_size": (c_size, [c_i64, c_i64, c_i64, c_vp]),
    "pft_q_order_workspace_size": (c_size, [c_i64]),
    "pft_q_order": (ctypes.c_int, [c_vp, c_i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_vp, c_vp, c_size, c_vp]),
    "pft2d_batched_workspace_size": (c_size, [c_i64, c_vp, c_i64, c_vp, c_i64, c_vp]),
    "pft2d_batched_prepare": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_size, c_vp, c_vp, c_vp]),
    "pft_batched_last_launch_count": (ctypes.c_int, []),
    "pft3d_workspace_size": (c_size, [c_i64, c_i64, c_i64, c_vp]),
    "pft2d_polygons": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_size, c_vp, c_vp]),
    "pft2d_polygons_batched": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp, c_size,
                                              c_vp, c_vp]),
    "pft3d_mesh": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_size, c_vp, c_vp]),
    "pft_selftest_wait": (ctypes.c_int, [c_vp, c_size, ctypes.c_uint32, ctypes.c_int, c_vp]),
    "pft3d_batched_workspace_size": (c_size, [c_i64, c_vp, c_i64, c_vp, c_i64, c_vp]),
    "pft3d_batched_prepare": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_size, c_vp, c_vp, c_vp]),
    "pft3d_meshes_batched": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp,
                                            c_size, c_vp, c_vp]),
    "pft3d_pair_faces": (ctypes.c_int, [c_vp, c_i64, c_vp, c_vp]),
    "pft3d_polymesh_workspace_size": (c_size, [c_i64, c_i64, c_i64, c_i64, c_vp]),
    "pft3d_polymesh": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_size,
                                      c_vp, c_vp]),
    "pft2d_backward_workspace_size": (c_size, [c_i64, c_i64, c_i64, c_vp]),
    "pft3d_backward_workspace_size": (c_size, [c_i64, c_i64, c_i64, c_vp]),
    "pft2d_batched_backward_workspace_size": (c_size, [c_i64, c_i64, c_i64, ctypes.c_int, c_vp]),
    "pft2d_polygons_batched_backward": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp, c_vp,
                                                       c_vp, c_size, c_vp, c_vp]),
    "pft3d_batched_backward_workspace_size": (c_size, [c_i64, c_i64, c_i64, c_i64, ctypes.c_int, c_vp]),
    "pft3d_meshes_batched_backward": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_i64,
                                                     c_vp, c_vp, c_vp, c_size, c_vp, c_vp]),
    "pft3d_qgrad_workspace_size": (c_size, [c_i64, c_i64, c_i64, c_vp]),
    "pft3d_mesh_qgrad": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp, c_size, c_vp, c_vp]),
    "pft2d_qgrad_workspace_size": (c_size, [c_i64, c_i64, c_i64, c_vp]),
    "pft2d_polygons_qgrad": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp, c_size,
                                            c_vp, c_vp]),
    "pft3d_polymesh_backward_workspace_size": (c_size, [c_i64, c_i64, c_i64, c_i64, c_vp]),
    "pft3d_polymesh_backward": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp,
                                               c_vp, c_size, c_vp, c_vp]),
    "pft2d_polygons_backward": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp, c_size,
                                               c_vp, c_vp]),
    "pft3d_mesh_noalloc": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp]),
    "pft3d_mesh_backward": (ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_vp, c_vp, c_size,
                                           c_vp, c_vp]),
    "pft_status": (ctypes.c_int, [c_vp, c_vp]),
    "pft_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "pft_version": (ctypes.c_int, []),
    "pft_last_launch_count": (ctypes.c_int, []),
    "pft_backward_last_launch_count": (ctypes.c_int, []),
}

_lock = threading.Lock()
_lib = None


class BatchedPlan(ctypes.Structure):
    """pft_batched_plan: opaque host-side handle filled by pft2d_batched_prepare."""
    _fields_ = [("opaque", ctypes.c_int64 * 24)]


class PFTError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (code {code})")


def load(path: str | None = None):
    """Load libpft.so (once).  Raises if it is missing: there is no CPU fallback."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libpft.so not built ({p}); run __graft_entry__.build() first")
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_string(code: int) -> str:
    try:
        return load().pft_status_string(int(code)).decode()
    except Exception:   # library not loadable: still give a readable message
        return "status"


def check(code: int, where: str) -> None:
    if code != PFT_OK:
        raise PFTError(code, where)
