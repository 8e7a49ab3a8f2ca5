"""Launch-shape autotuner for the forward kernels (Q points per thread, threads per block).

For a shape class it times every candidate configuration with CUDA events on
the caller's device, keeps the fastest, and caches the choice in a JSON file
keyed by (GPU name, path, size bucket), so later calls with similar sizes pay
nothing.  Results do not depend on the choice beyond rounding (the summation
order over segments/faces is fixed by the chunking, not by the launch shape).

Cache file: $PFT_TUNE_CACHE, else ~/.cache/pft/tune.json.
"""
from __future__ import annotations

import json
import math
import os
import threading

CANDIDATES_FP32 = [(1, 128), (2, 128), (4, 128), (8, 128), (1, 256), (2, 256), (4, 256), (8, 256)]
CANDIDATES_FP64 = [(1, 128), (2, 128), (1, 256), (2, 256)]
# the batched calls also run one block of 512 threads per SM (4 Q points per thread)
CANDIDATES_BATCHED_FP32 = CANDIDATES_FP32 + [(4, 512)]

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("PFT_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "pft", "tune.json")


def _load_cache(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, key, value):
    with _lock:
        data = _load_cache(path)
        data[key] = value
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def bucket(*sizes) -> str:
    """Size class: each size rounded to its power of two."""
    return "x".join(str(int(round(math.log2(max(1, int(s)))))) for s in sizes)


def make_key(device_name: str, kind: str, precision: str, *sizes) -> str:
    return f"{device_name}|{kind}|{precision}|{bucket(*sizes)}"


def pick(timings: dict) -> tuple:
    """Fastest candidate; ties go to the first listed (deterministic)."""
    best = None
    for cand, ms in timings.items():
        if ms is None:
            continue
        if best is None or ms < timings[best]:
            best = cand
    if best is None:
        raise RuntimeError("no autotune candidate ran")
    return best


def event_timer(fn, reps: int = 3, warmup: int = 1) -> float:
    """Median milliseconds of fn() over reps runs, timed with CUDA events on the current stream."""
    import torch
    for _ in range(warmup):
        fn()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    return sorted(times)[len(times) // 2]


def tune(key: str, run_for, candidates, timer=event_timer, use_cache: bool = True, path: str | None = None):
    """Return the best (q_per_thread, block_threads) for `key`.

    run_for(cand) returns a zero-argument callable that enqueues one call with that
    configuration (or raises if the configuration is unsupported).
    """
    path = path or cache_path()
    if use_cache:
        hit = _load_cache(path).get(key)
        if hit:
            return tuple(hit["best"])
    timings = {}
    for cand in candidates:
        try:
            timings[tuple(cand)] = timer(run_for(tuple(cand)))
        except Exception:   # an unsupported shape for this path: skip it
            timings[tuple(cand)] = None
    best = pick(timings)
    if use_cache:
        _store(path, key, {"best": list(best),
                           "ms": {f"{c[0]}x{c[1]}": t for c, t in timings.items() if t is not None}})
    return best


def _device_name(t):
    import torch
    return torch.cuda.get_device_name(t.device)


def tune_mesh3d(verts, faces, q, precision: str = "fp32", sample: int = 65536, **kw):
    """Best launch shape for pft3d_mesh on this mesh, timed on an evenly strided sample of Q."""
    import paper_2104_08309_gb300 as pft
    step = max(1, q.shape[0] // sample)
    qs = q[::step].contiguous()
    cands = CANDIDATES_FP64 if precision == "fp64" else CANDIDATES_FP32
    key = make_key(_device_name(verts), "mesh3d", precision, faces.shape[0], q.shape[0])

    def run_for(c):
        opts = {"precision": precision, "q_per_thread": c[0], "block_threads": c[1]}
        return lambda: pft.pft3d_mesh(verts, faces, qs, options=opts)
    r, nt = tune(key, run_for, cands, **kw)
    return {"precision": precision, "q_per_thread": r, "block_threads": nt}


def tune_batched2d(verts, poly_off, q, q_off=None, precision: str = "fp32", **kw):
    """Best launch shape for pft2d_polygons_batched (each candidate with its own prepared schedule)."""
    import paper_2104_08309_gb300 as pft
    cands = CANDIDATES_FP64 if precision == "fp64" else CANDIDATES_BATCHED_FP32
    n_polys = len(poly_off) - 1
    key = make_key(_device_name(verts), "batched2d", precision, n_polys, verts.shape[0], q.shape[0])

    def run_for(c):
        opts = {"precision": precision, "q_per_thread": c[0], "block_threads": c[1]}
        prep = pft.pft2d_batched_prepare(poly_off, q.shape[0], q_off, options=opts, device=verts.device)
        return lambda: pft.pft2d_polygons_batched(verts, poly_off, q, q_off, prepared=prep)
    r, nt = tune(key, run_for, cands, **kw)
    return {"precision": precision, "q_per_thread": r, "block_threads": nt}
