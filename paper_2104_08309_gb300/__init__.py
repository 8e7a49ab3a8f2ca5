"""pft -- direct Fourier transform of polygonal areas and closed triangulated
surfaces on an NVIDIA GB300 (sm_103a), after Maranville, arXiv 2104.08309.

This module is the thin Python face of ``libpft.so`` (C ABI in include/pft.h).
PyTorch supplies device memory and streams; every step of the computation runs
in the library's CUDA kernels.  There is no CPU fallback: calls on CPU tensors,
or without the built library, raise.

Functions named like the C entry points take CUDA tensors and return float64
[n_q, 2] (re, im) tensors; ``ft2d`` / ``ft3d`` wrap them as differentiable
complex128 results (``torch.autograd``) whose backward runs the adjoint kernels.
"""
from __future__ import annotations

import ctypes

from . import synth  # noqa: F401  (seeded inputs; no transform arithmetic)
from ._capi import (PFT_FP32_COMPENSATED, PFT_FP64, BatchedPlan, Options, PFTError, check, load,  # noqa: F401
                    status_string)

__all__ = [
    "pft2d_polygons", "pft2d_batched_prepare", "pft2d_polygons_batched", "BatchedPrepared", "pft3d_mesh",
    "pft3d_polymesh", "pft3d_polymesh_backward", "ft3d_poly", "pft2d_polygons_batched_backward", "pft3d_batched_prepare", "pft3d_meshes_batched",
    "pft2d_polygons_backward",
    "pft3d_mesh_backward", "pft3d_mesh_qgrad", "pft2d_polygons_qgrad", "pair_faces", "q_order",
    "pft3d_meshes_batched_backward", "ft3d_batched", "pft3d_mesh_noalloc", "pft_status", "ft2d", "ft2d_batched", "ft3d", "make_options", "Options",
    "PFTError",
    "launch_count", "version",
]


def _torch():
    import torch
    return torch


def make_options(options=None) -> Options:
    """Build a pft_options struct from None, an Options, or a dict of its fields.

    ``precision`` may be "fp32" (FP32 with compensated sums, the default) or "fp64"; ``q_order``
    "tiled" (the default: the library orders the Q points for the main kernel) or "as_given".
    """
    if isinstance(options, Options):
        return options
    o = Options()
    for k, v in (options or {}).items():
        if k == "precision":
            v = {"fp32": PFT_FP32_COMPENSATED, "fp64": PFT_FP64}.get(v, v)
        if k == "q_order":
            v = {"tiled": 0, "as_given": 1}.get(v, v)
        if not hasattr(o, k):
            raise KeyError(f"unknown pft option {k!r}")
        setattr(o, k, v)
    return o


def _dev(t, dtype, name, cols=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (libpft has no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
        raise ValueError(f"{name} must have shape [n, {cols}], got {tuple(t.shape)}")
    return t.contiguous()


def _stream(stream, device):
    torch = _torch()
    if stream is None:
        return torch.cuda.current_stream(device).cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ws(nbytes, device, ws):
    torch = _torch()
    if ws is None:
        ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    elif ws.numel() < nbytes:
        raise ValueError(f"workspace of {ws.numel()} bytes < {nbytes} required")
    return ws


def pft2d_polygons(verts, q, loop_off=None, *, options=None, out=None, ws=None, stream=None,
                   check_status=False):
    """FT_A(Q) of the region bounded by closed loops (Eq. 6).  Returns float64 [n_q, 2]."""
    torch = _torch()
    v = _dev(verts, torch.float32, "verts", 2)
    qq = _dev(q, torch.float64, "q", 2)
    if loop_off is None:
        loop_off = torch.tensor([0, v.shape[0]], dtype=torch.int64, device=v.device)
    off = _dev(loop_off.to(v.device) if loop_off.device != v.device else loop_off, torch.int64, "loop_off")
    o = make_options(options)
    lib = load()
    nv, nl, nq = v.shape[0], off.numel() - 1, qq.shape[0]
    nb = lib.pft2d_workspace_size(nv, nl, nq, ctypes.byref(o))
    ws = _ws(nb, v.device, ws)
    out = torch.empty(nq, 2, dtype=torch.float64, device=v.device) if out is None else out
    st = _stream(stream, v.device)
    check(lib.pft2d_polygons(v.data_ptr(), nv, off.data_ptr(), nl, qq.data_ptr(), nq, out.data_ptr(),
                             ws.data_ptr(), ws.numel(), ctypes.byref(o), st), "pft2d_polygons")
    if check_status:
        check(lib.pft_status(ws.data_ptr(), st), "pft2d_polygons (device status)")
    return out


class BatchedPrepared:
    """Workspace and schedule from pft2d_batched_prepare or pft3d_batched_prepare, reusable while the
    offsets stay the same."""

    def __init__(self, ws, plan, n_verts, n_polys, n_q, shared):
        self.ws, self.plan = ws, plan
        self.n_verts, self.n_polys, self.n_q, self.shared = n_verts, n_polys, n_q, shared


def _host_i64(x):
    torch = _torch()
    if isinstance(x, torch.Tensor):
        return x.detach().to("cpu", torch.int64).contiguous()
    return torch.as_tensor(x, dtype=torch.int64).contiguous()


def pft2d_batched_prepare(poly_off, n_q, q_off=None, *, options=None, device=None, stream=None):
    """Build the cost-sorted static schedule for a batch of polygons (host) and copy it to a new workspace.

    Synchronises the stream; call it outside CUDA-graph capture.  The returned object is
    passed to pft2d_polygons_batched as ``prepared``.
    """
    torch = _torch()
    off_h = _host_i64(poly_off)
    qo_h = None if q_off is None else _host_i64(q_off)
    device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    o = make_options(options)
    lib = load()
    n_polys = off_h.numel() - 1
    n_verts = int(off_h[-1]) if n_polys > 0 else 0
    qo_ptr = None if qo_h is None else qo_h.data_ptr()
    nb = lib.pft2d_batched_workspace_size(n_verts, off_h.data_ptr(), n_polys, qo_ptr, int(n_q), ctypes.byref(o))
    if nb == 0:
        raise ValueError("pft2d_batched_workspace_size rejected the offsets, sizes or options")
    ws = torch.empty(int(nb), dtype=torch.uint8, device=device)
    plan = BatchedPlan()
    check(lib.pft2d_batched_prepare(off_h.data_ptr(), n_polys, qo_ptr, int(n_q), ws.data_ptr(), ws.numel(),
                                    ctypes.byref(o), ctypes.byref(plan), _stream(stream, device)),
          "pft2d_batched_prepare")
    return BatchedPrepared(ws, plan, n_verts, n_polys, int(n_q), q_off is None)


def pft2d_polygons_batched(verts, poly_off, q, q_off=None, *, prepared=None, options=None, out=None, stream=None,
                           check_status=False):
    """One FT_A per polygon (Eq. 6 per segment) in one persistent launch.

    With q_off None every polygon uses all Q and the result is [n_polys, n_q, 2];
    otherwise polygon i uses q[q_off[i]:q_off[i+1]] and the result is [n_q, 2].
    Pass ``prepared`` (from pft2d_batched_prepare) to reuse a schedule; this call
    then only launches kernels and can be captured into a CUDA graph.
    """
    torch = _torch()
    v = _dev(verts, torch.float32, "verts", 2)
    qq = _dev(q, torch.float64, "q", 2)
    if prepared is None:
        prepared = pft2d_batched_prepare(poly_off, qq.shape[0], q_off, options=options, device=v.device,
                                         stream=stream)
    off_d = poly_off if (isinstance(poly_off, torch.Tensor) and poly_off.is_cuda) else \
        _host_i64(poly_off).to(v.device)
    off_d = _dev(off_d, torch.int64, "poly_off")
    qo_d = None
    if q_off is not None:
        qo_d = q_off if (isinstance(q_off, torch.Tensor) and q_off.is_cuda) else _host_i64(q_off).to(v.device)
        qo_d = _dev(qo_d, torch.int64, "q_off")
    npoly, nq = off_d.numel() - 1, qq.shape[0]
    n_out = npoly * nq if q_off is None else nq
    if out is None:
        out = torch.empty(n_out, 2, dtype=torch.float64, device=v.device)
    st = _stream(stream, v.device)
    lib = load()
    check(lib.pft2d_polygons_batched(v.data_ptr(), v.shape[0], off_d.data_ptr(), npoly, qq.data_ptr(),
                                     None if qo_d is None else qo_d.data_ptr(), nq, out.data_ptr(),
                                     prepared.ws.data_ptr(), prepared.ws.numel(), ctypes.byref(prepared.plan), st),
          "pft2d_polygons_batched")
    if check_status:
        check(lib.pft_status(prepared.ws.data_ptr(), st), "pft2d_polygons_batched (device status)")
    return out.view(npoly, nq, 2) if q_off is None else out


def pft3d_batched_prepare(mesh_off, n_q, q_off=None, *, options=None, device=None, stream=None):
    """Schedule for a batch of closed triangle meshes (CSR over faces), as pft2d_batched_prepare."""
    torch = _torch()
    off_h = _host_i64(mesh_off)
    qo_h = None if q_off is None else _host_i64(q_off)
    device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    o = make_options(options)
    lib = load()
    n_meshes = off_h.numel() - 1
    n_faces = int(off_h[-1]) if n_meshes > 0 else 0
    qo_ptr = None if qo_h is None else qo_h.data_ptr()
    nb = lib.pft3d_batched_workspace_size(n_faces, off_h.data_ptr(), n_meshes, qo_ptr, int(n_q), ctypes.byref(o))
    if nb == 0:
        raise ValueError("pft3d_batched_workspace_size rejected the offsets, sizes or options")
    ws = torch.empty(int(nb), dtype=torch.uint8, device=device)
    plan = BatchedPlan()
    check(lib.pft3d_batched_prepare(off_h.data_ptr(), n_meshes, qo_ptr, int(n_q), ws.data_ptr(), ws.numel(),
                                    ctypes.byref(o), ctypes.byref(plan), _stream(stream, device)),
          "pft3d_batched_prepare")
    return BatchedPrepared(ws, plan, n_faces, n_meshes, int(n_q), q_off is None)


def pft3d_meshes_batched(verts, faces, mesh_off, q, q_off=None, *, prepared=None, options=None, out=None,
                         stream=None, check_status=False):
    """One FT_V per closed triangle mesh in one persistent launch; meshes share verts and the
    faces of mesh i are faces[mesh_off[i]:mesh_off[i+1]].  Result [n_meshes, n_q, 2] for a shared
    Q set, else [n_q, 2] with mesh i on q[q_off[i]:q_off[i+1]].  With ``prepared`` (from
    pft3d_batched_prepare) the call only launches kernels (CUDA-graph capturable)."""
    torch = _torch()
    v = _dev(verts, torch.float32, "verts", 3)
    f = _dev(faces, torch.int32, "faces", 3)
    qq = _dev(q, torch.float64, "q", 3)
    if prepared is None:
        prepared = pft3d_batched_prepare(mesh_off, qq.shape[0], q_off, options=options, device=v.device,
                                         stream=stream)
    off_d = mesh_off if (isinstance(mesh_off, torch.Tensor) and mesh_off.is_cuda) else \
        _host_i64(mesh_off).to(v.device)
    off_d = _dev(off_d, torch.int64, "mesh_off")
    qo_d = None
    if q_off is not None:
        qo_d = q_off if (isinstance(q_off, torch.Tensor) and q_off.is_cuda) else _host_i64(q_off).to(v.device)
        qo_d = _dev(qo_d, torch.int64, "q_off")
    nm, nq = off_d.numel() - 1, qq.shape[0]
    n_out = nm * nq if q_off is None else nq
    if out is None:
        out = torch.empty(n_out, 2, dtype=torch.float64, device=v.device)
    st = _stream(stream, v.device)
    lib = load()
    check(lib.pft3d_meshes_batched(v.data_ptr(), v.shape[0], f.data_ptr(), f.shape[0], off_d.data_ptr(), nm,
                                   qq.data_ptr(), None if qo_d is None else qo_d.data_ptr(), nq, out.data_ptr(),
                                   prepared.ws.data_ptr(), prepared.ws.numel(), ctypes.byref(prepared.plan), st),
          "pft3d_meshes_batched")
    if check_status:
        check(lib.pft_status(prepared.ws.data_ptr(), st), "pft3d_meshes_batched (device status)")
    return out.view(nm, nq, 2) if q_off is None else out


def pft3d_mesh(verts, faces, q, *, options=None, out=None, ws=None, stream=None, check_status=False):
    """FT_V(Q) of a closed outward triangle surface (Eq. 14, sign-corrected).  Returns float64 [n_q, 2]."""
    torch = _torch()
    v = _dev(verts, torch.float32, "verts", 3)
    f = _dev(faces, torch.int32, "faces", 3)
    qq = _dev(q, torch.float64, "q", 3)
    o = make_options(options)
    lib = load()
    nv, nf, nq = v.shape[0], f.shape[0], qq.shape[0]
    nb = lib.pft3d_workspace_size(nv, nf, nq, ctypes.byref(o))
    ws = _ws(nb, v.device, ws)
    out = torch.empty(nq, 2, dtype=torch.float64, device=v.device) if out is None else out
    st = _stream(stream, v.device)
    check(lib.pft3d_mesh(v.data_ptr(), nv, f.data_ptr(), nf, qq.data_ptr(), nq, out.data_ptr(), ws.data_ptr(),
                         ws.numel(), ctypes.byref(o), st), "pft3d_mesh")
    if check_status:
        check(lib.pft_status(ws.data_ptr(), st), "pft3d_mesh (device status)")
    return out


def pair_faces(faces):
    """Host helper (no GPU): reorder a triangle list [n, 3] so that faces 2k and 2k+1 share their first
    edge in opposite directions, for k < n_pairs, followed by the unpaired faces.  Returns
    (faces_out int32 [n, 3], n_pairs); pass n_pairs as the ``face_pairs`` option of pft3d_mesh."""
    import numpy as np
    f = np.ascontiguousarray(np.asarray(faces.detach().cpu() if hasattr(faces, "detach") else faces,
                                        dtype=np.int32).reshape(-1, 3))
    out = np.empty_like(f)
    n = ctypes.c_int64(0)
    check(load().pft3d_pair_faces(f.ctypes.data, f.shape[0], out.ctypes.data, ctypes.byref(n)),
          "pft3d_pair_faces")
    return out, int(n.value)


def q_order(q, q_per_thread=4, block_threads=128, *, stream=None):
    """The slot -> Q index map (int32 [n_q], on q's device) by which the main kernel visits the Q
    points under the default ``q_order`` option, for q [n_q, 2] or [n_q, 3] float64 on a GPU and the
    given launch shape: slot s holds Q point perm[s]."""
    torch = _torch()
    if not isinstance(q, torch.Tensor) or not q.is_cuda or q.dim() != 2 or q.shape[1] not in (2, 3):
        raise ValueError("q must be a CUDA tensor [n_q, 2] or [n_q, 3]")
    qq = _dev(q, torch.float64, "q")
    lib = load()
    nq = qq.shape[0]
    perm = torch.empty(nq, dtype=torch.int32, device=qq.device)
    ws = _ws(lib.pft_q_order_workspace_size(nq), qq.device, None)
    check(lib.pft_q_order(qq.data_ptr(), nq, qq.shape[1], q_per_thread, block_threads, perm.data_ptr(),
                          ws.data_ptr(), ws.numel(), _stream(stream, qq.device)), "pft_q_order")
    return perm


def pft3d_polymesh(verts, face_idx, face_off, q, *, options=None, out=None, ws=None, stream=None,
                   check_status=False):
    """FT_V(Q) of a closed surface of planar polygon faces in CSR form: face m is
    face_idx[face_off[m]:face_off[m+1]] (int32 indices, int64 offsets, counter-clockwise seen
    from outside).  Returns float64 [n_q, 2]."""
    torch = _torch()
    v = _dev(verts, torch.float32, "verts", 3)
    idx = _dev(face_idx, torch.int32, "face_idx").reshape(-1)
    off = _dev(face_off, torch.int64, "face_off").reshape(-1)
    qq = _dev(q, torch.float64, "q", 3)
    o = make_options(options)
    lib = load()
    nv, ni, nf, nq = v.shape[0], idx.shape[0], max(off.shape[0] - 1, 0), qq.shape[0]
    nb = lib.pft3d_polymesh_workspace_size(nv, ni, nf, nq, ctypes.byref(o))
    if nb == 0:
        raise PFTError(1, "pft3d_polymesh (each face needs at least 3 vertices)")
    ws = _ws(nb, v.device, ws)
    out = torch.empty(nq, 2, dtype=torch.float64, device=v.device) if out is None else out
    st = _stream(stream, v.device)
    check(lib.pft3d_polymesh(v.data_ptr(), nv, idx.data_ptr(), ni, off.data_ptr(), nf, qq.data_ptr(), nq,
                             out.data_ptr(), ws.data_ptr(), ws.numel(), ctypes.byref(o), st), "pft3d_polymesh")
    if check_status:
        check(lib.pft_status(ws.data_ptr(), st), "pft3d_polymesh (device status)")
    return out


def pft3d_mesh_noalloc(verts, faces, q, out, *, options=None, stream=None):
    """pft3d_mesh with the library's fixed 32 MiB device scratch instead of a workspace.

    For callers that must not allocate at call time (stream capture, host
    applications that own all device memory): ``out`` ([n_q, 2] float64, CUDA)
    is required, every tensor must already be contiguous (no copies are made),
    and nothing is allocated here or in the library.  Calls whose
    GPU work overlaps share the scratch and race; the first call on a device
    must come before any stream capture.
    """
    torch = _torch()
    for t, name in ((verts, "verts"), (faces, "faces"), (q, "q")):
        if isinstance(t, torch.Tensor) and not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous: pft3d_mesh_noalloc makes no copies")
    v = _dev(verts, torch.float32, "verts", 3)
    f = _dev(faces, torch.int32, "faces", 3)
    qq = _dev(q, torch.float64, "q", 3)
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64
            and out.is_contiguous() and out.shape == (qq.shape[0], 2)):
        raise ValueError("out must be a contiguous CUDA float64 tensor of shape [n_q, 2]")
    o = make_options(options)
    check(load().pft3d_mesh_noalloc(v.data_ptr(), v.shape[0], f.data_ptr(), f.shape[0], qq.data_ptr(),
                                    qq.shape[0], out.data_ptr(), ctypes.byref(o), _stream(stream, v.device)),
          "pft3d_mesh_noalloc")
    return out


def pft2d_polygons_backward(verts, q, grad_out, loop_off=None, *, options=None, out=None, ws=None,
                            stream=None, check_status=False):
    """dL/dverts [n_v, 2] float32 from grad_out [n_q, 2] = (dL/dRe F, dL/dIm F)."""
    torch = _torch()
    v = _dev(verts, torch.float32, "verts", 2)
    qq = _dev(q, torch.float64, "q", 2)
    g = _dev(grad_out, torch.float64, "grad_out", 2)
    if loop_off is None:
        loop_off = torch.tensor([0, v.shape[0]], dtype=torch.int64, device=v.device)
    off = _dev(loop_off.to(v.device), torch.int64, "loop_off")
    o = make_options(options)
    lib = load()
    nv, nl, nq = v.shape[0], off.numel() - 1, qq.shape[0]
    nb = lib.pft2d_backward_workspace_size(nv, nl, nq, ctypes.byref(o))
    ws = _ws(nb, v.device, ws)
    out = torch.empty(nv, 2, dtype=torch.float32, device=v.device) if out is None else out
    st = _stream(stream, v.device)
    check(lib.pft2d_polygons_backward(v.data_ptr(), nv, off.data_ptr(), nl, qq.data_ptr(), nq, g.data_ptr(),
                                      out.data_ptr(), ws.data_ptr(), ws.numel(), ctypes.byref(o), st),
          "pft2d_polygons_backward")
    if check_status:
        check(lib.pft_status(ws.data_ptr(), st), "pft2d_polygons_backward (device status)")
    return out


def pft3d_mesh_backward(verts, faces, q, grad_out, *, options=None, out=None, ws=None, stream=None,
                        check_status=False):
    """dL/dverts [n_v, 3] float32 from grad_out [n_q, 2] = (dL/dRe F, dL/dIm F)."""
    torch = _torch()
    v = _dev(verts, torch.float32, "verts", 3)
    f = _dev(faces, torch.int32, "faces", 3)
    qq = _dev(q, torch.float64, "q", 3)
    g = _dev(grad_out, torch.float64, "grad_out", 2)
    o = make_options(options)
    lib = load()
    nv, nf, nq = v.shape[0], f.shape[0], qq.shape[0]
    nb = lib.pft3d_backward_workspace_size(nv, nf, nq, ctypes.byref(o))
    ws = _ws(nb, v.device, ws)
    out = torch.empty(nv, 3, dtype=torch.float32, device=v.device) if out is None else out
    st = _stream(stream, v.device)
    check(lib.pft3d_mesh_backward(v.data_ptr(), nv, f.data_ptr(), nf, qq.data_ptr(), nq, g.data_ptr(),
                                  out.data_ptr(), ws.data_ptr(), ws.numel(), ctypes.byref(o), st),
          "pft3d_mesh_backward")
    if check_status:
        check(lib.pft_status(ws.data_ptr(), st), "pft3d_mesh_backward (device status)")
    return out


def pft3d_polymesh_backward(verts, face_idx, face_off, q, grad_out, *, options=None, out=None, ws=None,
                            stream=None, check_status=False):
    """dL/dverts [n_v, 3] float32 for pft3d_polymesh, from grad_out [n_q, 2] = (dL/dRe F, dL/dIm F)."""
    torch = _torch()
    v = _dev(verts, torch.float32, "verts", 3)
    idx = _dev(face_idx, torch.int32, "face_idx").reshape(-1)
    off = _dev(face_off, torch.int64, "face_off").reshape(-1)
    qq = _dev(q, torch.float64, "q", 3)
    g = _dev(grad_out, torch.float64, "grad_out", 2)
    o = make_options(options)
    lib = load()
    nv, ni, nf, nq = v.shape[0], idx.shape[0], max(off.shape[0] - 1, 0), qq.shape[0]
    nb = lib.pft3d_polymesh_backward_workspace_size(nv, ni, nf, nq, ctypes.byref(o))
    if nb == 0:
        raise PFTError(1, "pft3d_polymesh_backward (each face needs at least 3 vertices)")
    ws = _ws(nb, v.device, ws)
    out = torch.empty(nv, 3, dtype=torch.float32, device=v.device) if out is None else out
    st = _stream(stream, v.device)
    check(lib.pft3d_polymesh_backward(v.data_ptr(), nv, idx.data_ptr(), ni, off.data_ptr(), nf, qq.data_ptr(), nq,
                                      g.data_ptr(), out.data_ptr(), ws.data_ptr(), ws.numel(), ctypes.byref(o), st),
          "pft3d_polymesh_backward")
    if check_status:
        check(lib.pft_status(ws.data_ptr(), st), "pft3d_polymesh_backward (device status)")
    return out


def pft3d_mesh_qgrad(verts, faces, q, grad_out, *, options=None, out=None, ws=None, stream=None,
                     check_status=False):
    """dL/dQ [n_q, 3] float64 from grad_out [n_q, 2] = (dL/dRe F, dL/dIm F) (3D triangles)."""
    torch = _torch()
    v = _dev(verts, torch.float32, "verts", 3)
    f = _dev(faces, torch.int32, "faces", 3)
    qq = _dev(q, torch.float64, "q", 3)
    g = _dev(grad_out, torch.float64, "grad_out", 2)
    o = make_options(options)
    lib = load()
    nv, nf, nq = v.shape[0], f.shape[0], qq.shape[0]
    nb = lib.pft3d_qgrad_workspace_size(nv, nf, nq, ctypes.byref(o))
    ws = _ws(nb, v.device, ws)
    out = torch.empty(nq, 3, dtype=torch.float64, device=v.device) if out is None else out
    st = _stream(stream, v.device)
    check(lib.pft3d_mesh_qgrad(v.data_ptr(), nv, f.data_ptr(), nf, qq.data_ptr(), nq, g.data_ptr(), out.data_ptr(),
                               ws.data_ptr(), ws.numel(), ctypes.byref(o), st), "pft3d_mesh_qgrad")
    if check_status:
        check(lib.pft_status(ws.data_ptr(), st), "pft3d_mesh_qgrad (device status)")
    return out


def pft2d_polygons_qgrad(verts, q, grad_out, loop_off=None, *, options=None, out=None, ws=None, stream=None,
                         check_status=False):
    """dL/dQ [n_q, 2] float64 from grad_out [n_q, 2] = (dL/dRe F, dL/dIm F) (2D loops)."""
    torch = _torch()
    v = _dev(verts, torch.float32, "verts", 2)
    qq = _dev(q, torch.float64, "q", 2)
    g = _dev(grad_out, torch.float64, "grad_out", 2)
    if loop_off is None:
        loop_off = torch.tensor([0, v.shape[0]], dtype=torch.int64, device=v.device)
    off = _dev(loop_off.to(v.device), torch.int64, "loop_off")
    o = make_options(options)
    lib = load()
    nv, nl, nq = v.shape[0], off.numel() - 1, qq.shape[0]
    nb = lib.pft2d_qgrad_workspace_size(nv, nl, nq, ctypes.byref(o))
    ws = _ws(nb, v.device, ws)
    out = torch.empty(nq, 2, dtype=torch.float64, device=v.device) if out is None else out
    st = _stream(stream, v.device)
    check(lib.pft2d_polygons_qgrad(v.data_ptr(), nv, off.data_ptr(), nl, qq.data_ptr(), nq, g.data_ptr(),
                                   out.data_ptr(), ws.data_ptr(), ws.numel(), ctypes.byref(o), st),
          "pft2d_polygons_qgrad")
    if check_status:
        check(lib.pft_status(ws.data_ptr(), st), "pft2d_polygons_qgrad (device status)")
    return out


def pft2d_polygons_batched_backward(verts, poly_off, q, grad_out, q_off=None, *, options=None, out=None, ws=None,
                                    stream=None, check_status=False):
    """dL/dverts [n_v, 2] float32 for a batch of polygons, from grad_out = (dL/dRe F_i(Q), dL/dIm F_i(Q)):
    [n_polys, n_q, 2] on a shared Q set (q_off None), or [n_q, 2] with polygon i on q[q_off[i]:q_off[i+1]]."""
    torch = _torch()
    v = _dev(verts, torch.float32, "verts", 2)
    off = poly_off if (isinstance(poly_off, torch.Tensor) and poly_off.is_cuda) else _host_i64(poly_off).to(v.device)
    off = _dev(off, torch.int64, "poly_off").reshape(-1)
    qq = _dev(q, torch.float64, "q", 2)
    np_, nq = off.shape[0] - 1, qq.shape[0]
    qo = None
    if q_off is not None:
        qo = q_off if (isinstance(q_off, torch.Tensor) and q_off.is_cuda) else _host_i64(q_off).to(v.device)
        qo = _dev(qo, torch.int64, "q_off").reshape(-1)
    g = _dev(grad_out, torch.float64, "grad_out").reshape(nq if qo is not None else np_ * nq, 2)
    o = make_options(options)
    lib = load()
    nb = lib.pft2d_batched_backward_workspace_size(v.shape[0], np_, nq, int(qo is not None), ctypes.byref(o))
    ws = _ws(nb, v.device, ws)
    out = torch.empty(v.shape[0], 2, dtype=torch.float32, device=v.device) if out is None else out
    st = _stream(stream, v.device)
    check(lib.pft2d_polygons_batched_backward(v.data_ptr(), v.shape[0], off.data_ptr(), np_, qq.data_ptr(),
                                              None if qo is None else qo.data_ptr(), nq, g.data_ptr(),
                                              out.data_ptr(), ws.data_ptr(), ws.numel(), ctypes.byref(o), st),
          "pft2d_polygons_batched_backward")
    if check_status:
        check(lib.pft_status(ws.data_ptr(), st), "pft2d_polygons_batched_backward (device status)")
    return out


def pft3d_meshes_batched_backward(verts, faces, mesh_off, q, grad_out, q_off=None, *, options=None, out=None,
                                  ws=None, stream=None, check_status=False):
    """dL/dverts [n_v, 3] float32 for a batch of closed meshes (faces of mesh i: faces[mesh_off[i]:
    mesh_off[i+1]]), from grad_out = (dL/dRe F_i(Q), dL/dIm F_i(Q)): [n_meshes, n_q, 2] on a shared Q
    set (q_off None), or [n_q, 2] with mesh i on q[q_off[i]:q_off[i+1]]."""
    torch = _torch()
    v = _dev(verts, torch.float32, "verts", 3)
    f = _dev(faces, torch.int32, "faces", 3)
    off = mesh_off if (isinstance(mesh_off, torch.Tensor) and mesh_off.is_cuda) else _host_i64(mesh_off).to(v.device)
    off = _dev(off, torch.int64, "mesh_off").reshape(-1)
    qq = _dev(q, torch.float64, "q", 3)
    nm, nq = off.shape[0] - 1, qq.shape[0]
    qo = None
    if q_off is not None:
        qo = q_off if (isinstance(q_off, torch.Tensor) and q_off.is_cuda) else _host_i64(q_off).to(v.device)
        qo = _dev(qo, torch.int64, "q_off").reshape(-1)
    g = _dev(grad_out, torch.float64, "grad_out").reshape(nq if qo is not None else nm * nq, 2)
    o = make_options(options)
    lib = load()
    nb = lib.pft3d_batched_backward_workspace_size(v.shape[0], f.shape[0], nm, nq, int(qo is not None),
                                                   ctypes.byref(o))
    ws = _ws(nb, v.device, ws)
    out = torch.empty(v.shape[0], 3, dtype=torch.float32, device=v.device) if out is None else out
    st = _stream(stream, v.device)
    check(lib.pft3d_meshes_batched_backward(v.data_ptr(), v.shape[0], f.data_ptr(), f.shape[0], off.data_ptr(), nm,
                                            qq.data_ptr(), None if qo is None else qo.data_ptr(), nq, g.data_ptr(),
                                            out.data_ptr(), ws.data_ptr(), ws.numel(), ctypes.byref(o), st),
          "pft3d_meshes_batched_backward")
    if check_status:
        check(lib.pft_status(ws.data_ptr(), st), "pft3d_meshes_batched_backward (device status)")
    return out


def pft_status(ws, stream=None) -> int:
    """Device-detected status of the last call on this workspace (synchronises the stream)."""
    return int(load().pft_status(ws.data_ptr(), _stream(stream, ws.device)))


def launch_count() -> int:
    """Kernel launches enqueued by the most recent library call on this thread."""
    return int(load().pft_last_launch_count())


def version() -> int:
    return int(load().pft_version())


# ----------------------------------------------------------------------------
# Differentiable wrappers.
# ----------------------------------------------------------------------------

def _autograd():
    torch = _torch()

    class _FT2D(torch.autograd.Function):
        @staticmethod
        def forward(ctx, verts, q, loop_off, options):
            ctx.save_for_backward(verts, q, loop_off)
            ctx.options = options
            return pft2d_polygons(verts.detach(), q.detach(), loop_off, options=options)

        @staticmethod
        def backward(ctx, g):
            verts, q, loop_off = ctx.saved_tensors
            g = g.contiguous()
            gv = pft2d_polygons_backward(verts.detach(), q.detach(), g, loop_off, options=ctx.options) \
                if ctx.needs_input_grad[0] else None
            gq = pft2d_polygons_qgrad(verts.detach(), q.detach(), g, loop_off, options=ctx.options) \
                if ctx.needs_input_grad[1] else None
            return gv, gq, None, None

    class _FT3D(torch.autograd.Function):
        @staticmethod
        def forward(ctx, verts, faces, q, options):
            ctx.save_for_backward(verts, faces, q)
            ctx.options = options
            return pft3d_mesh(verts.detach(), faces, q.detach(), options=options)

        @staticmethod
        def backward(ctx, g):
            verts, faces, q = ctx.saved_tensors
            g = g.contiguous()
            gv = pft3d_mesh_backward(verts.detach(), faces, q, g, options=ctx.options) \
                if ctx.needs_input_grad[0] else None
            gq = pft3d_mesh_qgrad(verts.detach(), faces, q.detach(), g, options=ctx.options) \
                if ctx.needs_input_grad[2] else None
            return gv, None, gq, None

    class _FT3DPoly(torch.autograd.Function):
        @staticmethod
        def forward(ctx, verts, face_idx, face_off, q, options):
            ctx.save_for_backward(verts, face_idx, face_off, q)
            ctx.options = options
            return pft3d_polymesh(verts.detach(), face_idx, face_off, q, options=options)

        @staticmethod
        def backward(ctx, g):
            verts, face_idx, face_off, q = ctx.saved_tensors
            gv = pft3d_polymesh_backward(verts.detach(), face_idx, face_off, q, g.contiguous(), options=ctx.options)
            return gv, None, None, None, None

    class _FT2DBatched(torch.autograd.Function):
        @staticmethod
        def forward(ctx, verts, poly_off, q, q_off, options):
            ctx.save_for_backward(verts, poly_off, q, q_off)
            ctx.precision = make_options(options).precision
            return pft2d_polygons_batched(verts.detach(), poly_off, q, q_off, options=options)

        @staticmethod
        def backward(ctx, g):
            verts, poly_off, q, q_off = ctx.saved_tensors
            # the forward's precision goes to the adjoint, which refuses FP64 (it has an FP32 path
            # only); the forward's launch shape does not apply to it
            gv = pft2d_polygons_batched_backward(verts.detach(), poly_off, q, g.contiguous(), q_off,
                                                 options={"precision": ctx.precision})
            return gv, None, None, None, None

    class _FT3DBatched(torch.autograd.Function):
        @staticmethod
        def forward(ctx, verts, faces, mesh_off, q, q_off, options):
            ctx.save_for_backward(verts, faces, mesh_off, q, q_off)
            ctx.precision = make_options(options).precision
            ctx.tau = make_options(options).face_series_tau
            return pft3d_meshes_batched(verts.detach(), faces, mesh_off, q, q_off, options=options)

        @staticmethod
        def backward(ctx, g):
            verts, faces, mesh_off, q, q_off = ctx.saved_tensors
            gv = pft3d_meshes_batched_backward(verts.detach(), faces, mesh_off, q, g.contiguous(), q_off,
                                               options={"precision": ctx.precision, "face_series_tau": ctx.tau})
            return gv, None, None, None, None, None

    return _FT2D, _FT3D, _FT3DPoly, _FT2DBatched, _FT3DBatched


_FNS = None


def ft2d(verts, q, loop_off=None, options=None):
    """Differentiable FT_A(Q) as complex128 [n_q]; gradients w.r.t. verts and q via the adjoint kernels."""
    global _FNS
    torch = _torch()
    _FNS = _FNS or _autograd()
    if loop_off is None:
        loop_off = torch.tensor([0, verts.shape[0]], dtype=torch.int64, device=verts.device)
    return torch.view_as_complex(_FNS[0].apply(verts, q, loop_off, options))


def ft3d(verts, faces, q, options=None):
    """Differentiable FT_V(Q) as complex128 [n_q]; gradients w.r.t. verts and q via the adjoint kernels."""
    global _FNS
    torch = _torch()
    _FNS = _FNS or _autograd()
    return torch.view_as_complex(_FNS[1].apply(verts, faces, q, options))


def ft2d_batched(verts, poly_off, q, options=None, q_off=None):
    """Differentiable FT_A of each polygon of a batch, complex128 [n_polys, n_q] on a shared Q set, or
    [n_q] with polygon i on q[q_off[i]:q_off[i+1]];
    grad w.r.t. verts via the batched adjoint, which runs in FP32 with compensated sums.  ``options``
    set the forward call (launch shape, precision); a gradient of an FP64 forward is refused (raised
    here when ``verts`` requires grad) rather than silently computed in FP32."""
    global _FNS
    torch = _torch()
    _FNS = _FNS or _autograd()
    if (make_options(options).precision == PFT_FP64 and torch.is_grad_enabled()
            and isinstance(verts, torch.Tensor) and verts.requires_grad):
        raise ValueError("ft2d_batched: the batched adjoint has no FP64 path; use precision='fp32' "
                         "for a differentiable batch, or detach verts")
    off = poly_off if (isinstance(poly_off, torch.Tensor) and poly_off.is_cuda) else \
        _host_i64(poly_off).to(verts.device)
    qo = None
    if q_off is not None:
        qo = q_off if (isinstance(q_off, torch.Tensor) and q_off.is_cuda) else _host_i64(q_off).to(verts.device)
    return torch.view_as_complex(_FNS[3].apply(verts, off, q, qo, options))


def ft3d_batched(verts, faces, mesh_off, q, options=None, q_off=None):
    """Differentiable FT_V of each closed mesh of a batch, complex128 [n_meshes, n_q] on a shared Q set,
    or [n_q] with mesh i on q[q_off[i]:q_off[i+1]]; grad w.r.t. verts via the batched adjoint (FP32 with
    compensated sums: a gradient of an FP64 forward is refused)."""
    global _FNS
    torch = _torch()
    _FNS = _FNS or _autograd()
    if (make_options(options).precision == PFT_FP64 and torch.is_grad_enabled()
            and isinstance(verts, torch.Tensor) and verts.requires_grad):
        raise ValueError("ft3d_batched: the batched adjoint has no FP64 path; use precision='fp32' "
                         "for a differentiable batch, or detach verts")
    off = mesh_off if (isinstance(mesh_off, torch.Tensor) and mesh_off.is_cuda) else \
        _host_i64(mesh_off).to(verts.device)
    qo = None
    if q_off is not None:
        qo = q_off if (isinstance(q_off, torch.Tensor) and q_off.is_cuda) else _host_i64(q_off).to(verts.device)
    return torch.view_as_complex(_FNS[4].apply(verts, faces, off, q, qo, options))


def ft3d_poly(verts, face_idx, face_off, q, options=None):
    """Differentiable FT_V(Q) of a planar-polygon-face surface as complex128 [n_q]; grad w.r.t. verts
    via the adjoint kernel."""
    global _FNS
    torch = _torch()
    _FNS = _FNS or _autograd()
    return torch.view_as_complex(_FNS[2].apply(verts, face_idx, face_off, q, options))
