#!/usr/bin/env python
"""Benchmark of the direct polyhedron Fourier transform on one or more GB300s.

Workload (one step): FT_V(Q) of an icosphere of subdivision 8 (1,310,720
triangles, vertices moved radially by 1 + 0.05 U[-1,1), seed 5) on a 128^3 Q
grid over [-60, 60)^3 -- 2.75e12 (Q, triangle) pairs -- through the C ABI
(pft3d_mesh, FP32 arithmetic with compensated sums and an FP64 finish).

Prints one JSON line: G pair-evaluations/s, the main kernel's roofline
fraction against the FP32-lane / SFU limit, the end-to-end rate with host
buffers, and the FP64 CPU oracle's rate on a bounded sample of the same
workload.  ``--impl reference`` times that oracle alone (the reference arm).

Multi-GPU (torchrun): every rank transforms its own perturbed mesh (seed
5 + rank) on the full grid; there is no collective on the data path (weak
scaling); the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G (Q,segment) pair-evals/s and % FP32/SFU roofline at stated error vs FP64"
UNIT = "Gpair/s"
WORKLOAD = "icosphere8_perturbed_q128cubed"

# Algorithmic per-pair instruction counts of the 3D FP32 face term (face_common,
# face_series* / face_edge, face_finish in pft_pairs.cuh): FP32-pipe operations
# (add/mul/fma/compare/select, the SFU argument scaling) and SFU operations (sin,
# cos, reciprocal), per branch.  Each series form costs 25 ops outside the series
# (projections with P and T 16, branch tests 2, finish 7) plus its own: T^2 1 and
# one FMA per coefficient beyond the first of each polynomial in P, and the nesting in T^2.
OPS = {
    "series_k7": {"fp32": 33, "sfu": 2},      # face-integral series through k = 7 (P < 1/4)
    "series_k9": {"fp32": 37, "sfu": 2},      # through k = 9 (P < 1)
    "series_k11": {"fp32": 41, "sfu": 2},     # through k = 11 (P < 9/4)
    "series_k13": {"fp32": 46, "sfu": 2},     # through k = 13 (P < 4)
    "series_k17": {"fp32": 58, "sfu": 2},     # through k = 17 (P < 9)
    "edge_sum": {"fp32": 92, "sfu": 7},       # edge sum of Eq. 14, polynomial sinc
    # a face of a pair whose two faces both take the edge sum (face_pairs option): the second face
    # skips the shared edge's u^2, Chebyshev sinc and range test (8), so each face costs 88 on average
    "edge_sum_shared": {"fp32": 88, "sfu": 7},
}
# An edge of the edge sum with |Q.d/2| > pi: sin(u)/u on the SFU (sinc_large: the turn reduction 4, the
# SFU argument scaling 1, the product with 1/u 1; sin and 1/u on the SFU) on top of the polynomial.
OPS_EDGE_SFU_SINC = {"fp32": 6, "sfu": 2}
SERIES_BOUNDS = [("series_k7", 0.25), ("series_k9", 1.0), ("series_k11", 2.25),
                 ("series_k13", 4.0)]         # P bounds of the forms below k = 17 (kP* in pft_pairs.cuh)
# 2D segment term (Pol2F32::tile): projections 6, u^2 1, Chebyshev sinc 6, range test 1, the
# SFU argument scaling 1, w*S 1, accumulation 2; beyond |u| > pi the SFU sinc adds the turn
# reduction and 1/u (6 FP32-pipe + 2 SFU).
OPS2D = {
    "poly_sinc": {"fp32": 18, "sfu": 2},
    "sfu_sinc": {"fp32": 24, "sfu": 4},
}
# 2D pair adjoint (seg_adj in pft_bwd.cu: the term recomputed and differentiated, four record
# adjoints updated): 21 written, sinc_d's polynomial and derivative 14, range test 1, the sincos
# argument scaling 1, with 2 SFU operations; beyond |u| > pi sinc_d adds the turn reduction, sin,
# cos and 1/u and the two quotients (8 FP32-pipe + 3 SFU).
OPS2D_ADJ = {
    "poly_sinc": {"fp32": 37, "sfu": 2},
    "sfu_sinc": {"fp32": 45, "sfu": 5},
}
# Per-pair operation counts of the 3D pair adjoint (face_adj_t in pft_bwd.cu, forward recomputed
# and differentiated in reverse mode), as a part every pair pays plus one part per branch; a warp
# whose lanes take two branches issues both.  Common to every branch: the projections (face_common,
# 15), the branch selection (one warp reduction of |P|, four compares and the predicate logic, 10),
# the argument scaling of sincos(mu) (1) and its 2 SFU operations, the weights W = e^{i mu} Z and
# the adjoints of s and mu (15), and the 12 updates of the record (vertex adjoint, RecAdj) or, for
# the Q-gradient (QAdj), the 12 updates of Q plus the 2 adds of the pair's own term.  Per branch:
# the series forms' forward part and derivatives in P and T (k <= 7, 9, 11, 17: 17 / 26 / 34 / 70)
# plus their adjoint (10); the edge sum's forward part (38, three sinc_d on the polynomial path of
# 15, two sincos scalings, the 1/|X|^2 test and select: 87, with 5 SFU operations) plus its adjoint
# (62) and the X-adjoint terms (12 record updates, or 6 for Q).  Products of two literals are
# folded by the compiler and not counted; the SFU sinc beyond |u| > pi is the rare branch.
OPS_ADJ = {"common": {"fp32": 53, "sfu": 2},
           "short": {"fp32": 27, "sfu": 0}, "k9": {"fp32": 36, "sfu": 0}, "long": {"fp32": 44, "sfu": 0},
           "xlong": {"fp32": 80, "sfu": 0}, "edge": {"fp32": 161, "sfu": 5}}
OPS_QADJ = {"common": {"fp32": 57, "sfu": 2},
            "short": {"fp32": 27, "sfu": 0}, "k9": {"fp32": 36, "sfu": 0}, "long": {"fp32": 44, "sfu": 0},
            "xlong": {"fp32": 80, "sfu": 0}, "edge": {"fp32": 155, "sfu": 5}}
FP32_LANES, SFU_LANES = 128, 16       # per SM per clock
# A fixed per-pair count of the triangle term taken as the edge sum of Eq. 14 with a polynomial sinc
# (projections, three edges' phase/sinc/term, face factor): the basis of frac_vs_survey_count.
SURVEY_COUNT = {"fp32": 82, "sfu": 7}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target length of the CPU-oracle sample")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle leg")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default="c5",
                   help="c5: the benchmark workload; c5small: same mesh family at subdivision 6 on 64^3 Q "
                        "(for profiling captures)")
    p.add_argument("--q-per-thread", type=int, default=4)
    p.add_argument("--block-threads", type=int, default=128)
    p.add_argument("--tau", type=float, default=0.0, help="face_series_tau (0 = library default)")
    p.add_argument("--no-extra", action="store_true", help="skip the secondary paths (batched 2D, adjoint)")
    p.add_argument("--only", choices=["batched", "adjoint", "polymesh", "batched3d", "voxels"], default=None,
                   help="run one secondary path alone and print its result (for profiler captures)")
    return p.parse_args()


def bench_out_dir():
    """Where the bench leaves its side files (clock samples, the autotuner's cache): $PFT_BENCH_OUT,
    else a folder in the system's temporary directory."""
    import tempfile
    d = os.environ.get("PFT_BENCH_OUT") or os.path.join(tempfile.gettempdir(), "pft_bench")
    os.makedirs(d, exist_ok=True)
    return d


def replica_seed(rank):
    """Seed of the mesh rank `rank` transforms: every rank an independent problem of the same size."""
    return 5 + rank


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over all ranks (one all-reduce; identity at N = 1)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(x) for x in values]
    t = torch.tensor([float(x) for x in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_rate(world, pairs_per_rank, ms):
    """G pairs/s of the whole job: all ranks' pairs over the slowest rank's time."""
    return world * pairs_per_rank / (ms / 1e3) / 1e9


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), ws


WORKLOADS = {
    "c5": (WORKLOAD, 1),
    # the same mesh on every 4th (qx, qy) column of the same grid (1/16 of the Q
    # points, same spacing along qz): for profiler captures of the main kernel
    "c5small": ("icosphere8_perturbed_q128cubed_every16th_column", 4),
    "c5tiny": ("icosphere8_perturbed_q128cubed_every64th_column", 8),
}


def workload(rank, name="c5"):
    from paper_2104_08309_gb300 import synth
    _, stride = WORKLOADS[name]
    v, f = synth.perturbed_icosphere(8, seed=replica_seed(rank), amp=0.05)
    q = synth.q_grid_3d(128, 60.0)
    if stride > 1:
        q = np.ascontiguousarray(q.reshape(128, 128, 128, 3)[::stride, ::stride].reshape(-1, 3))
    return v, f, q


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"sm_max_mhz": 2070.0}, "fallback"


def _warp_sample(v, f, q, r, nt, n_warps, seed):
    """A seeded sample of (face, warp) pairs as the kernel forms them: for one face, a warp holds the
    Q indices base + k*nt + 32*w + lane (k < r, lane < 32).  Returns the faces and the Q of each warp."""
    rng = np.random.default_rng(seed)
    fi = rng.integers(0, f.shape[0], n_warps)
    per_block = r * nt
    base = per_block * rng.integers(0, max(1, q.shape[0] // per_block), n_warps)
    w = rng.integers(0, nt // 32, n_warps)
    idx = (base[:, None, None] + np.arange(r)[None, :, None] * nt + 32 * w[:, None, None]
           + np.arange(32)[None, None, :]).reshape(n_warps, -1)
    idx = np.minimum(idx, q.shape[0] - 1)
    return fi, q[idx]                                    # [w], [w, r*32, 3]


def _corner_phases(v, f, faces, qq):
    p = v.astype(np.float64)[f[faces]]                   # [w, 3, 3]
    g = p.mean(axis=1)
    return np.einsum("wlj,wj->wl", qq, p[:, 0] - g), np.einsum("wlj,wj->wl", qq, p[:, 1] - g)


def _edge_rule(v, f, q, tau, r, nt, n_warps, seed, n_pairs):
    fi, qq = _warp_sample(v, f, q, r, nt, n_warps, seed)

    def warp_pmax(faces):
        a0, a1 = _corner_phases(v, f, faces, qq)
        return (a0 * a0 + a0 * a1 + a1 * a1).max(axis=1).astype(np.float32)

    pmax = warp_pmax(fi)
    p_hi = np.float32(0.25 * tau * tau)
    left = pmax < p_hi                                   # warps that take a series form
    shared = np.zeros(n_warps, dtype=bool)
    if n_pairs > 0:
        partner = np.where(fi < 2 * n_pairs, fi ^ 1, fi)
        shared = (fi < 2 * n_pairs) & ~left & (warp_pmax(partner) >= p_hi)
    return fi, qq, pmax, p_hi, left, shared


def branch_mix(v, f, q, tau=6.0, r=2, nt=128, n_warps=4096, seed=0, n_pairs=0):
    """Fractions of (Q, face) pairs the kernel evaluates with each branch.

    Mirrors the kernel's rule on a seeded sample (`_warp_sample`): if every Q of a warp has
    P < p_hi = tau^2/4 they all take the first series form whose bound b has
    p_hi <= b or every P < b (k = 17 when none has); otherwise the edge sum (the
    few pairs below tau_lo^2/4 that the edge branch redoes with the series are
    counted as edge).  Thresholds are compared in float32, as the kernel does.  With n_pairs > 0
    (faces 2k, 2k+1 paired, k < n_pairs) a paired face whose partner takes the edge sum in the same
    warp as well is counted as edge_sum_shared.
    """
    _, _, pmax, p_hi, left, shared = _edge_rule(v, f, q, tau, r, nt, n_warps, seed, n_pairs)
    out = {"edge_sum": float(np.mean(~left & ~shared)), "edge_sum_shared": float(np.mean(shared))}
    for name, b in SERIES_BOUNDS:
        take = left & ((p_hi <= np.float32(b)) | (pmax < np.float32(b)))
        out[name] = float(np.mean(take))
        left &= ~take
    out["series_k17"] = float(np.mean(left))
    return {k: out[k] for k in OPS}


def edge_sfu_sinc(v, f, q, tau=6.0, r=2, nt=128, n_warps=4096, seed=0, n_pairs=0):
    """Edges per pair (over all pairs) whose sinc the edge sum takes on the SFU: in a warp on the edge
    sum, edge l of a pair with u_l^2 > pi^2 in float32, u = ((a1 - a0)/2, (-a0 - 2 a1)/2, (2 a0 + a1)/2)
    (face_edge).  The shared first edge of a pair whose faces both take the edge sum is evaluated once,
    by the first face, for both: half an edge per face, as edge_sum_shared averages its saving.  Each
    costs OPS_EDGE_SFU_SINC on top of the polynomial sinc every edge pays."""
    fi, qq, _, _, left, shared = _edge_rule(v, f, q, tau, r, nt, n_warps, seed, n_pairs)
    a0, a1 = _corner_phases(v, f, fi, qq)
    u = np.stack([(a1 - a0) / 2, (-a0 - 2 * a1) / 2, (2 * a0 + a1) / 2], axis=-1).astype(np.float32)
    big = (u * u) > np.float32(np.pi ** 2)                # [w, r*32, 3]
    per_pair = np.where(shared[:, None], big[:, :, 1:].sum(axis=-1) + 0.5 * big[:, :, 0], big.sum(axis=-1))
    return float(np.mean(np.where((~left)[:, None], per_pair, 0)))


def kernel_order(pft, q, qd, r, nt, n_items):
    """q in the order the main kernel visits it (the q_order option's default): the library orders
    the Q points when there are at least two blocks' worth of them and 2^30 pairs or more, and
    pft.q_order returns that order (slot -> Q index)."""
    if q.shape[0] >= 2 * r * nt and float(q.shape[0]) * float(n_items) >= 2.0 ** 30:
        return q[pft.q_order(qd, r, nt).cpu().numpy()]
    return q


def adjoint_branch_mix(v, f, q, tau=6.0, lanes="faces", n_warps=4096, seed=0):
    """The pair adjoint's branch rule on a seeded sample of warps, and the per-pair cost it implies.

    lanes="faces" (k_bwd: a warp holds 32 consecutive faces and takes one Q record at a time) or
    "q" (k_qgrad: 32 consecutive Q points, one face at a time).  Per lane, with P in float32 and
    wmax the warp's largest P: short when every P < 1/4 (tau > 1; else every P < tau^2/4) or its
    own P < tau_lo^2/4; the k <= 9 form when not short and every P < 1 (and < tau^2/4); long when
    neither and every P < 9/4 (and < tau^2/4); extra-long when none of these but every P < tau^2/4;
    else the edge sum.  Returns the fraction of lanes in
    each branch, the fraction of warps issuing each, and the mean count of issued operations per
    pair (a warp pays the common part once and the part of every branch one of its lanes takes)."""
    rng = np.random.default_rng(seed)
    v64 = v.astype(np.float64)
    if lanes == "faces":
        fi = 32 * rng.integers(0, max(1, f.shape[0] // 32), n_warps)[:, None] + np.arange(32)[None, :]
        fi = np.minimum(fi, f.shape[0] - 1)
        qq = np.broadcast_to(q[rng.integers(0, q.shape[0], n_warps)][:, None, :], (n_warps, 32, 3))
    else:
        qi = 32 * rng.integers(0, max(1, q.shape[0] // 32), n_warps)[:, None] + np.arange(32)[None, :]
        qq = q[np.minimum(qi, q.shape[0] - 1)]
        fi = np.broadcast_to(rng.integers(0, f.shape[0], n_warps)[:, None], (n_warps, 32))
    p = v64[f[fi]]                                        # [w, 32, 3, 3]
    g = p.mean(axis=2)
    a0 = np.einsum("wlj,wlj->wl", qq, p[:, :, 0] - g)
    a1 = np.einsum("wlj,wlj->wl", qq, p[:, :, 1] - g)
    P = (a0 * a0 + a0 * a1 + a1 * a1).astype(np.float32)
    wmax = P.max(axis=1)[:, None]
    hi, lo = np.float32(0.25 * tau * tau), np.float32(0.25 * min(tau, 0.05) ** 2)
    all_hi = wmax < hi
    shorts = ((wmax < np.float32(0.25)) if tau > 1 else all_hi) | (P < lo)
    k9 = ~shorts & all_hi & (wmax < np.float32(1.0))
    longs = ~shorts & ~k9 & all_hi & ((wmax < np.float32(2.25)) if tau > 3 else True)
    series = shorts | all_hi
    br = {"short": shorts, "k9": k9, "long": longs, "xlong": series & ~shorts & ~k9 & ~longs, "edge": ~series}
    lane = {k: float(m.mean()) for k, m in br.items()}
    warp = {k: float(m.any(axis=1).mean()) for k, m in br.items()}
    return lane, warp


def adjoint_ops(warp_fracs, table):
    """Mean issued FP32-pipe and SFU operations per pair for the branch-issue fractions of warps."""
    return {k: table["common"][k] + sum(warp_fracs[b] * table[b][k] for b in warp_fracs) for k in ("fp32", "sfu")}


def sfu_sinc_fraction(verts, poly_off, q, n=1 << 16, seed=0):
    """Fraction of (segment, Q) pairs of a batched 2D problem with |Q.D/2| > pi (the SFU sinc),
    on a seeded uniform sample of the pairs (every polygon uses the same Q set)."""
    rng = np.random.default_rng(seed)
    seg = rng.integers(0, verts.shape[0], n)
    poly = np.searchsorted(poly_off, seg, side="right") - 1
    nxt = np.where(seg + 1 == poly_off[poly + 1], poly_off[poly], seg + 1)
    d = verts[nxt].astype(np.float64) - verts[seg]
    qq = q[rng.integers(0, q.shape[0], n)]
    u = 0.5 * np.abs(np.einsum("ij,ij->i", qq, d))
    return float(np.mean(u > np.pi))


def bound_cycles(ops, paired):
    """SM cycles per pair at the limit, and the operations per pair that bind.  An SM has 128
    FP32 lanes and 16 SFU lanes per clock and issues 128 thread-instructions per clock: one per
    scalar FP32 or SFU operation, one per paired FP32 instruction (two operations, each on its
    own lane).  Scalar code is issue-bound at (fp32 + sfu) / 128.  In the paired kernels more
    than 2 sfu of the fp32 operations issue in pairs, so their issue count stays below fp32 and
    the FP32 lanes bind at fp32 / 128.  Either way the SFU lanes bound at sfu / 16."""
    lanes = ops["fp32"] if paired else ops["fp32"] + ops["sfu"]
    return max(lanes / FP32_LANES, ops["sfu"] / SFU_LANES), lanes


def roofline2d(pairs, t_s, f_sfu, n_sm, clk_mhz, table=None, paired=True):
    """FP32-lane (paired) or issue-slot (scalar) / SFU bound of the 2D segment term (or, with
    table=OPS2D_ADJ, of its adjoint) for a given SFU-sinc fraction."""
    table = OPS2D if table is None else table
    mix = {"poly_sinc": 1.0 - f_sfu, "sfu_sinc": f_sfu}
    ops = {k: sum(mix[b] * table[b][k] for b in table) for k in ("fp32", "sfu")}
    cyc, lanes = bound_cycles(ops, paired)
    peak_pairs = n_sm * clk_mhz * 1e6 / cyc
    return {"bound": "alu" if lanes / FP32_LANES >= ops["sfu"] / SFU_LANES else "sfu",
            "ops_per_pair": ops, "sfu_sinc_fraction": f_sfu, "peak_gpair_s": peak_pairs / 1e9,
            "frac": pairs / t_s / peak_pairs,
            "peak_basis": "128 FP32 lanes" if paired else "128 FP32/SFU issue slots"}


def roofline(pairs, t_main_s, mix, n_sm, clk_mhz, paired=True, sfu_edges=0.0):
    """3D face term: (ops per pair, binding ops per pair, achieved and peak binding ops/s).
    sfu_edges: edges per pair whose sinc the edge sum takes on the SFU (`edge_sfu_sinc`)."""
    ops = {k: sum(mix[b] * OPS[b][k] for b in OPS) + sfu_edges * OPS_EDGE_SFU_SINC[k] for k in ("fp32", "sfu")}
    cyc, lanes = bound_cycles(ops, paired)                       # SM cycles per pair at the limit
    peak_ops = n_sm * clk_mhz * 1e6 * lanes / cyc                # binding ops/s at the limit
    achieved = lanes * pairs / t_main_s
    return ops, lanes, achieved, peak_ops


def survey_count_frac(pairs, t_s, n_sm, clk_mhz):
    """Main-kernel pair rate over the peak pair rate of SURVEY_COUNT's fixed per-pair count."""
    cyc = max(SURVEY_COUNT["fp32"] / FP32_LANES, SURVEY_COUNT["sfu"] / SFU_LANES)
    return pairs / t_s / (n_sm * clk_mhz * 1e6 / cyc)


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid, self.proc, self.path = uuid, None, None

    def start(self):
        try:
            out = bench_out_dir()
            os.makedirs(out, exist_ok=True)
            self.path = os.path.join(out, f"clocks_{os.getpid()}.csv")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.uuid}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = [r.split(", ") for r in open(self.path).read().strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "samples": len(rows), "reasons": reasons}


def err_stats(got, ref, measure):
    """max / p99 / median of |got - ref| / |measure| over the points (complex arrays)."""
    e = np.abs(np.asarray(got) - np.asarray(ref)) / abs(measure)
    return {"max": float(np.max(e)), "p99": float(np.percentile(e, 99)), "median": float(np.median(e))}


def cpu_baseline(v, f, q, sub, chunk=1024):
    """FP64 oracle (as it stands) on every host core, on the seeded 4,096-point Q subsample over all
    faces.  The first chunk of 1,024 points is the timed CPU sample (about 15 s on 16 cores); the
    remaining points are computed untimed, for the error figures over the whole subsample."""
    import oracle
    threads = os.cpu_count() or 1
    parts, dt = [], None
    for k in range(0, sub.size, chunk):
        t0 = time.perf_counter()
        parts.append(oracle.ft3d(v, f, q[sub[k:k + chunk]], threads=threads))
        if dt is None:
            dt = time.perf_counter() - t0
    n = min(chunk, sub.size)
    rate = n * f.shape[0] / dt / 1e9
    return {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n} of the {sub.size} seeded Q points of the 128^3 grid x all {f.shape[0]} triangles "
                      f"({dt:.1f} s timed); the other {sub.size - n} computed untimed for the error figures"}, \
        np.concatenate(parts)


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    v, f, q = workload(0)
    import oracle
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(11)
    t0 = time.perf_counter()
    oracle.ft3d(v, f, q[rng.integers(0, q.shape[0], threads)], threads=threads)
    per_q = (time.perf_counter() - t0) / threads
    n = max(threads, int(threads * round(6.0 / max(per_q * threads, 1e-6))))   # ~6 s per step
    times = []
    for s in range(args.warmup + args.steps):
        idx = rng.choice(q.shape[0], n, replace=False)
        t0 = time.perf_counter()
        oracle.ft3d(v, f, q[idx], threads=threads)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    value = n * f.shape[0] / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "faces": int(f.shape[0]), "q_points": int(q.shape[0]),
                       "step": f"{n} seeded Q points x all triangles (bounded sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{n} Q points per step x {f.shape[0]} triangles"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def bench_batched(dev, warmup, steps):
    """Secondary path: 4,096 star polygons (8..4,096 vertices) on a shared 64^2 grid, one prepared
    schedule replayed from a CUDA graph; each replay is one full batched transform."""
    import torch
    import paper_2104_08309_gb300 as pft
    from paper_2104_08309_gb300 import synth
    w = synth.workload_c3()
    vd, qd = torch.from_numpy(w.verts).to(dev), torch.from_numpy(w.q).to(dev)
    offd = torch.from_numpy(w.poly_off).to(dev)
    from paper_2104_08309_gb300 import autotune
    tuned = autotune.tune_batched2d(vd, w.poly_off, qd,
                                    path=os.path.join(bench_out_dir(), "tune_cache.json"))
    prep = pft.pft2d_batched_prepare(w.poly_off, w.q.shape[0], options=tuned, device=dev)
    out = torch.empty(w.poly_off.size - 1, w.q.shape[0], 2, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        pft.pft2d_polygons_batched(vd, offd, qd, prepared=prep, out=out)
    torch.cuda.current_stream(dev).wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pft.pft2d_polygons_batched(vd, offd, qd, prepared=prep, out=out)
    launches = pft.load().pft_batched_last_launch_count()
    for _ in range(max(3, warmup)):
        g.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for a, b in ev:
        flush.zero_()
        a.record()
        g.replay()
        b.record()
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    pairs = float(w.verts.shape[0]) * float(w.q.shape[0])
    status = pft.pft_status(prep.ws)
    pk, pk_kind = peaks()
    rl = roofline2d(pairs, ms / 1e3, sfu_sinc_fraction(w.verts, w.poly_off, w.q),
                    torch.cuda.get_device_properties(dev).multi_processor_count, float(pk.get("sm_max_mhz", 2070.0)),
                    paired=tuned["q_per_thread"] % 2 == 0)
    rl["note"] = (f"whole {int(launches)}-launch call timed; the finish of the 16.8M outputs (2/|Q|^2, "
                  "e^{iQ.c}) "
                  "is outside the per-pair count")
    # the plain FP64 GPU path on the same batch (one call), and the FP32 result's deviation from it
    p64 = pft.pft2d_batched_prepare(w.poly_off, w.q.shape[0], options={"precision": "fp64"}, device=dev)
    o64 = pft.pft2d_polygons_batched(vd, offd, qd, prepared=p64)
    torch.cuda.synchronize()
    flush.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    pft.pft2d_polygons_batched(vd, offd, qd, prepared=p64, out=o64)
    b.record()
    b.synchronize()
    q0 = int(np.flatnonzero(np.all(w.q == 0, axis=1))[0])
    area = o64[:, q0, 0].abs()
    dev32 = ((out - o64).abs().amax(dim=(1, 2)) / area).max().item()
    fp64 = {"value": pairs / (a.elapsed_time(b) / 1e3) / 1e9, "unit": UNIT, "ms": a.elapsed_time(b),
            "fp32_vs_fp64_max_abs_over_area": dev32}
    del o64
    # the batched adjoint (vertex gradients of every polygon for seeded weights on the same grid)
    gb = torch.randn(w.poly_off.size - 1, w.q.shape[0], 2, dtype=torch.float64, device=dev,
                     generator=torch.Generator(device=dev).manual_seed(7))
    for _ in range(2):
        pft.pft2d_polygons_batched_backward(vd, offd, qd, gb)
    tb = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        pft.pft2d_polygons_batched_backward(vd, offd, qd, gb)
        b.record()
        b.synchronize()
        tb.append(a.elapsed_time(b))
    launches_b = int(pft.load().pft_backward_last_launch_count())
    tk = []   # the pair kernel k_bbwd alone: caller events the library records around it
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        b.record()
        pft.pft2d_polygons_batched_backward(vd, offd, qd, gb, options={"main_start_event": a.cuda_event,
                                                                       "main_stop_event": b.cuda_event})
        torch.cuda.synchronize()
        tk.append(a.elapsed_time(b))
    rlb = roofline2d(pairs, float(np.mean(tk)) / 1e3, rl["sfu_sinc_fraction"],
                     torch.cuda.get_device_properties(dev).multi_processor_count, float(pk.get("sm_max_mhz", 2070.0)),
                     table=OPS2D_ADJ)
    rlb.update({"kernel": "k_bbwd", "kernel_ms": float(np.mean(tk))})
    backward = {"value": pairs / (float(np.mean(tb)) / 1e3) / 1e9, "unit": UNIT + " (adjoint call)",
                "ms": float(np.mean(tb)), "launches": launches_b, "roofline": rlb}
    del gb
    return {"value": pairs / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms, "pairs_per_step": pairs,
            "roofline": rl,
            "polygons": int(w.poly_off.size - 1), "segments": int(w.verts.shape[0]), "q_points": int(w.q.shape[0]),
            "launches_per_step": int(launches), "cuda_graph": True, "device_status": int(status),
            "launch": {"q_per_thread": tuned["q_per_thread"], "block_threads": tuned["block_threads"],
                       "chosen_by": "autotune"}, "fp64_gpu": fp64, "backward": backward,
            "l2": "flushed between steps"}


def bench_batched3d(dev, warmup, steps):
    """Secondary path: 1,024 separate closed meshes (perturbed icospheres of levels 1-4: 80 to 5,120
    faces, 1.68M faces in all) on a shared 32^3 grid, one prepared schedule replayed from a CUDA
    graph; each replay is one full batched transform."""
    import torch
    import paper_2104_08309_gb300 as pft
    from paper_2104_08309_gb300 import synth
    v, f, off = synth.mesh_batch(1024, seed=21)
    q = synth.q_grid_3d(32, 30.0)
    vd, fd, qd, offd = (torch.from_numpy(a).to(dev) for a in (v, f, q, off))
    r, nt = 4, 512                           # the default launch shape on this shared Q set
    prep = pft.pft3d_batched_prepare(off, q.shape[0], options={"q_per_thread": r, "block_threads": nt},
                                     device=dev)
    out = torch.empty(off.size - 1, q.shape[0], 2, dtype=torch.float64, device=dev)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        pft.pft3d_meshes_batched(vd, fd, offd, qd, prepared=prep, out=out)
    torch.cuda.current_stream(dev).wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pft.pft3d_meshes_batched(vd, fd, offd, qd, prepared=prep, out=out)
    launches = pft.load().pft_batched_last_launch_count()
    for _ in range(max(3, warmup)):
        g.replay()
    torch.cuda.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ts = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.replay()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ms = float(np.mean(ts))
    pairs = float(f.shape[0]) * float(q.shape[0])
    pk, _ = peaks()
    qk = kernel_order(pft, q, qd, r, nt, f.shape[0])
    mix = branch_mix(v, f, qk, tau=6.0, r=r, nt=nt)
    sfu_e = edge_sfu_sinc(v, f, qk, tau=6.0, r=r, nt=nt)
    _, _, ach, peak = roofline(pairs, ms / 1e3, mix, torch.cuda.get_device_properties(dev).multi_processor_count,
                               float(pk.get("sm_max_mhz", 2070.0)), sfu_edges=sfu_e)
    status = int(pft.pft_status(prep.ws))
    del g                                    # the CUDA graph
    # the batched adjoint: vertex gradients of every mesh for seeded weights on the same grid
    gb = torch.randn(off.size - 1, q.shape[0], 2, dtype=torch.float64, device=dev,
                     generator=torch.Generator(device=dev).manual_seed(9))
    for _ in range(2):
        pft.pft3d_meshes_batched_backward(vd, fd, offd, qd, gb)
    tb = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        pft.pft3d_meshes_batched_backward(vd, fd, offd, qd, gb)
        b.record()
        b.synchronize()
        tb.append(a.elapsed_time(b))
    backward = {"value": pairs / (float(np.mean(tb)) / 1e3) / 1e9, "unit": UNIT + " (adjoint call)",
                "ms": float(np.mean(tb)), "launches": int(pft.load().pft_backward_last_launch_count())}
    del gb
    return {"value": pairs / (ms / 1e3) / 1e9, "unit": UNIT + " (Q, triangle)", "ms_per_step": ms,
            "pairs_per_step": pairs, "meshes": int(off.size - 1), "faces": int(f.shape[0]),
            "q_points": int(q.shape[0]), "launch_shape": [r, nt], "launches_per_step": int(launches),
            "cuda_graph": True,
            "device_status": status, "roofline_frac": ach / peak, "branch_fractions": mix,
            "edge_sfu_sinc_per_pair": sfu_e,
            "backward": backward,
            "note": "whole batched call timed (prep, pair kernel, multi-chunk finish, small-|Q| pass)",
            "l2": "flushed between steps"}


def bench_fp64(pft, vd, fd, qd, sub, dev):
    """The plain FP64 GPU path on the same mesh, on the seeded 4,096-point Q subsample (FP64 runs at a
    small fraction of the FP32 rate on this part); returns its rate and its result there."""
    import torch
    qs = qd[torch.from_numpy(sub).to(dev)].contiguous()
    o64 = {"precision": "fp64"}
    pft.pft3d_mesh(vd, fd, qs, options=o64)          # warm-up
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    r64 = pft.pft3d_mesh(vd, fd, qs, options=o64)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b)
    pairs = float(fd.shape[0]) * float(sub.size)
    r64 = r64.cpu().numpy()
    return {"value": pairs / (ms / 1e3) / 1e9, "unit": UNIT, "ms": ms,
            "sample": f"{sub.size} seeded Q points (the oracle's subsample)"}, r64[:, 0] + 1j * r64[:, 1]


def halving_triangles(idx, off):
    """The library's split of planar polygon faces into triangles (recursive halving, pre-order),
    on the host: only for the branch-mix sample of the roofline."""
    tris = []
    for m in range(off.size - 1):
        f = idx[off[m]:off[m + 1]]
        stack = [(0, f.size - 1)]
        while stack:
            i, j = stack.pop()
            if j - i < 2:
                continue
            k = (i + j) // 2
            tris.append((f[i], f[k], f[j]))
            stack += [(k, j), (i, k)]
    return np.array(tris, dtype=np.int32)


def bench_polymesh(dev, warmup, steps):
    """Secondary path: a prism over a 65,536-vertex non-convex star (two 65,536-gon caps and
    65,536 side quadrilaterals = 262,140 triangles) on a 64^3 grid through pft3d_polymesh; also
    its largest deviation from the 2D path times the extrusion factor (e^{iQz h} - 1)/(iQz)."""
    import torch
    import paper_2104_08309_gb300 as pft
    from paper_2104_08309_gb300 import synth
    star = synth.star_polygon(65536, seed=11).astype(np.float32)
    h = 0.75
    v, idx, off = synth.extruded_polygon(star, h)
    q = synth.q_grid_3d(64, 30.0)
    vd, idd, od, qd = (torch.from_numpy(a).to(dev) for a in (v, idx, off, q))
    out = torch.empty(q.shape[0], 2, dtype=torch.float64, device=dev)
    for _ in range(max(3, warmup)):
        pft.pft3d_polymesh(vd, idd, od, qd, out=out)
    torch.cuda.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ts = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        pft.pft3d_polymesh(vd, idd, od, qd, out=out)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ms = float(np.mean(ts))
    launches = int(pft.launch_count())
    n_tris = int(idx.size - 2 * (off.size - 1))
    pairs = float(n_tris) * float(q.shape[0])
    got = out.cpu().numpy()
    got = got[:, 0] + 1j * got[:, 1]
    f2 = pft.pft2d_polygons(torch.from_numpy(star).to(dev), torch.from_numpy(np.ascontiguousarray(q[:, :2])).to(dev))
    f2 = f2.cpu().numpy()
    x = 0.5 * q[:, 2] * h
    ref = (f2[:, 0] + 1j * f2[:, 1]) * h * np.sinc(x / np.pi) * np.exp(1j * x)
    vol = abs(got[int(np.flatnonzero(np.all(q == 0, axis=1))[0])])
    pk, _ = peaks()
    tris, qk = halving_triangles(idx, off), kernel_order(pft, q, qd, 4, 128, n_tris)
    mix = branch_mix(v, tris, qk, tau=6.0, r=4, nt=128)
    sfu_e = edge_sfu_sinc(v, tris, qk, tau=6.0, r=4, nt=128)
    _, _, ach, peak = roofline(pairs, ms / 1e3, mix, torch.cuda.get_device_properties(dev).multi_processor_count,
                               float(pk.get("sm_max_mhz", 2070.0)), sfu_edges=sfu_e)
    return {"value": pairs / (ms / 1e3) / 1e9, "unit": UNIT + " (Q, triangle)", "ms_per_call": ms,
            "faces": int(off.size - 1), "triangles": n_tris, "q_points": int(q.shape[0]), "pairs_per_call": pairs,
            "launches_per_call": launches, "roofline_frac": ach / peak, "branch_fractions": mix,
            "edge_sfu_sinc_per_pair": sfu_e,
            "vs_2d_path_times_extrusion_max_abs_over_volume": float(np.max(np.abs(got - ref)) / vol),
            "l2": "flushed between calls"}


def bench_adjoint(dev, warmup, steps):
    """Secondary path: vertex gradient of sum_Q (|F|^2 - I)^2 for 16 icospheres (81,920 triangles) on
    a 32^3 grid; a step is one forward plus one adjoint call (the loss weights in between on torch)."""
    import torch
    import paper_2104_08309_gb300 as pft
    from paper_2104_08309_gb300 import synth
    w = synth.workload_c4()
    vd, fd, qd = (torch.from_numpy(a).to(dev) for a in (w.verts, w.faces, w.q))
    vt = torch.from_numpy(w.verts_target).to(dev)
    Ft = pft.pft3d_mesh(vt, fd, qd)
    target = (Ft[:, 0] ** 2 + Ft[:, 1] ** 2)

    def step():
        F = pft.pft3d_mesh(vd, fd, qd)
        r = F[:, 0] ** 2 + F[:, 1] ** 2 - target
        g = 4.0 * r[:, None] * F
        return pft.pft3d_mesh_backward(vd, fd, qd, g)

    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    eb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for (a, b), (c, d) in zip(ev, eb):
        flush.zero_()
        a.record()
        F = pft.pft3d_mesh(vd, fd, qd)
        r = F[:, 0] ** 2 + F[:, 1] ** 2 - target
        g = 4.0 * r[:, None] * F
        c.record()
        grad = pft.pft3d_mesh_backward(vd, fd, qd, g)
        d.record()
        b.record()
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    ms_b = float(np.mean([c.elapsed_time(d) for c, d in eb]))
    pairs = float(w.faces.shape[0]) * float(w.q.shape[0])
    launches_adj = int(pft.load().pft_backward_last_launch_count())

    def kernel_ms(fn):
        """The call's pair kernel alone: caller events the library records around it."""
        ts = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            b.record()
            fn({"main_start_event": a.cuda_event, "main_stop_event": b.cuda_event})
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts))

    ms_kbwd = kernel_ms(lambda o: pft.pft3d_mesh_backward(vd, fd, qd, g, options=o))
    # the Q-gradient of the same loss (one call per step, same weights)
    for _ in range(3):
        pft.pft3d_mesh_qgrad(vd, fd, qd, g)
    torch.cuda.synchronize()
    tq = []
    for _ in range(steps):
        flush.zero_()
        c, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c.record()
        pft.pft3d_mesh_qgrad(vd, fd, qd, g)
        d.record()
        d.synchronize()
        tq.append(c.elapsed_time(d))
    ms_q = float(np.mean(tq))
    launches_q = int(pft.load().pft_backward_last_launch_count())
    ms_kq = kernel_ms(lambda o: pft.pft3d_mesh_qgrad(vd, fd, qd, g, options=o))
    pk, pk_kind = peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk = float(pk.get("sm_max_mhz", 2070.0))

    def rl(kernel, ms_k, lanes, table):
        # k_qgrad holds one Q point per thread, in the library's order (q_order's default)
        qm = kernel_order(pft, w.q, qd, 1, 128, w.faces.shape[0]) if lanes == "q" else w.q
        lane, warp = adjoint_branch_mix(w.verts, w.faces, qm, lanes=lanes)
        ops = adjoint_ops(warp, table)
        issue = ops["fp32"] + ops["sfu"]
        cyc = max(issue / FP32_LANES, ops["sfu"] / SFU_LANES)
        peak = n_sm * clk * 1e6 * issue / cyc
        return {"bound": "alu", "kernel": kernel, "kernel_ms": ms_k, "achieved": issue * pairs / (ms_k / 1e3) / 1e12,
                "peak": peak / 1e12, "unit": "Tops/s", "frac": issue * pairs / (ms_k / 1e3) / peak,
                "ops_per_pair": ops, "branch_lanes": lane, "branch_warps": warp,
                "peak_basis": f"{n_sm} SMs x 128 issue slots x {clk:.0f} MHz ({pk_kind} max SM clock)"}

    return {"value": pairs / (ms_b / 1e3) / 1e9, "unit": UNIT + " (adjoint call)", "ms_adjoint": ms_b,
            "roofline": rl("k_bwd<3,12>", ms_kbwd, "faces", OPS_ADJ),
            "qgrad": {"value": pairs / (ms_q / 1e3) / 1e9, "unit": UNIT + " (Q-gradient call)", "ms": ms_q,
                      "launches": launches_q, "roofline": rl("k_qgrad", ms_kq, "q", OPS_QADJ)},
            "ms_forward_plus_adjoint": ms, "pairs_per_call": pairs, "faces": int(w.faces.shape[0]),
            "q_points": int(w.q.shape[0]), "finite": bool(torch.isfinite(grad).all().item()),
            "launches_adjoint": launches_adj}


def bench_sphere_voxels(dev):
    """Sec. 4.3's comparison along Q_x = 0 .. 60 through the GPU path: the unit sphere voxelised with
    cube side d = 0.2 (the closed surface of the 552 cubes, pft3d_polymesh) and icospheres of
    subdivision 2 and 5 (pft3d_mesh), each against the sphere's closed form (Eq. 23); a table at
    a few Q_x and where the voxel transform's deviation peaks beyond Q_x = 15."""
    import torch
    import paper_2104_08309_gb300 as pft
    from paper_2104_08309_gb300 import synth
    d = 0.2
    qx = np.arange(0, 241) * 0.25
    q = np.stack([qx, 0 * qx, 0 * qx], axis=1)
    qd = torch.from_numpy(q).to(dev)
    with np.errstate(invalid="ignore", divide="ignore"):
        exact = np.where(qx == 0, 4 * np.pi / 3, 4 * np.pi * (np.sin(qx) - qx * np.cos(qx)) / qx ** 3)

    def c(out):
        o = out.cpu().numpy()
        return o[:, 0] + 1j * o[:, 1]

    occ = synth.voxel_ball(10, 1.0, d)
    v, idx, off = synth.voxel_surface(occ, d)
    vox = c(pft.pft3d_polymesh(torch.from_numpy(v).to(dev), torch.from_numpy(idx).to(dev),
                               torch.from_numpy(off).to(dev), qd, check_status=True))
    ico = {}
    for level in (2, 5):
        vi, fi = synth.icosphere(level)
        ico[level] = c(pft.pft3d_mesh(torch.from_numpy(vi).to(dev), torch.from_numpy(fi).to(dev), qd,
                                      check_status=True))
    far = qx >= 15.0
    dev_vox = np.abs(vox - exact)
    pick = [0, 20, 40, 80, 100, 112, 117, 120, 126, 140, 160, 200, 240]
    return {"workload": "unit sphere: 552 cubes of side 0.2 (voxels) vs icospheres of subdivision 2 (320 "
                        "triangles) and 5 (20,480), Q along x from 0 to 60",
            "voxel_cubes": int(occ.sum()), "two_pi_over_d": 2 * np.pi / d,
            "voxel_peak_deviation_qx": float(qx[far][np.argmax(dev_vox[far])]),
            "max_deviation_qx_ge_15": {"voxels": float(np.max(dev_vox[far])),
                                       "icosphere2": float(np.max(np.abs(ico[2] - exact)[far])),
                                       "icosphere5": float(np.max(np.abs(ico[5] - exact)[far]))},
            "table": {"qx": [float(qx[i]) for i in pick], "sphere_eq23": [float(exact[i]) for i in pick],
                      "voxels": [float(vox[i].real) for i in pick],
                      "icosphere2": [float(ico[2][i].real) for i in pick],
                      "icosphere5": [float(ico[5][i].real) for i in pick]}}


KERNEL_SOURCES = ("pft_fwd.cu", "pft_pairs.cuh", "pft_common.cuh", "pft_kernels.cuh", "pft_api.cu")


def kernel_source_hash():
    """First 16 hex digits of the SHA-256 of the main kernel's sources and of the launch planner
    (in a fixed order): the DRAM traffic of a launch depends on both."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2104_08309_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def synth_c5_sub(q):
    from paper_2104_08309_gb300 import synth
    return synth.c5_subsample_indices(q)


def traffic_from_profile():
    """DRAM bytes per main-kernel launch from the committed ncu summary, if it was taken on
    these kernel sources (None once the kernel has changed since the counters were taken)."""
    path = os.path.join(ROOT, "profiles", "k_fwd_dram_icosphere8_q128cubed.txt")
    try:
        kv = dict(l.split(":", 1) for l in open(path).read().splitlines() if ":" in l)
        if kv.get("source_sha256_16", "").strip() == kernel_source_hash():
            return float(kv["dram_bytes_per_launch_full_size"])
    except (OSError, KeyError, ValueError):
        pass
    return None


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        import torch
        dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
        torch.cuda.set_device(dev)
        from paper_2104_08309_gb300 import build as pbuild
        pbuild.build()
        fn = {"batched": bench_batched, "adjoint": bench_adjoint, "polymesh": bench_polymesh,
              "batched3d": bench_batched3d, "voxels": lambda d, w, s: bench_sphere_voxels(d)}[args.only]
        print(json.dumps({"path": args.only, **fn(dev, args.warmup, args.steps)}))
        return 0
    import torch
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import paper_2104_08309_gb300 as pft
    from paper_2104_08309_gb300 import build as pbuild
    pbuild.build()

    v, f, q = workload(rank, args.workload)
    pairs = float(f.shape[0]) * float(q.shape[0])
    vd, fd, qd = (torch.from_numpy(a).to(dev) for a in (v, f, q))
    lib = pft.load()
    e_main = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    e_step = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    for a, b in e_main:
        a.record()
        b.record()
    tune = {"q_per_thread": args.q_per_thread, "block_threads": args.block_threads,
            "face_series_tau": args.tau}
    opts = pft.make_options(tune)
    nbytes = lib.pft3d_workspace_size(v.shape[0], f.shape[0], q.shape[0], ctypes.byref(opts))
    # the paired variant's launch plan (another kernel, other occupancy) may want a larger workspace
    paired_opts = pft.make_options({**tune, "face_pairs": f.shape[0] // 2})
    nbytes = max(nbytes, lib.pft3d_workspace_size(v.shape[0], f.shape[0], q.shape[0], ctypes.byref(paired_opts)))
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = torch.empty(q.shape[0], 2, dtype=torch.float64, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)    # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def step(o, faces_dev=None):
        faces_dev = fd if faces_dev is None else faces_dev
        rc = lib.pft3d_mesh(vd.data_ptr(), v.shape[0], faces_dev.data_ptr(), f.shape[0], qd.data_ptr(), q.shape[0],
                            out.data_ptr(), ws.data_ptr(), nbytes, ctypes.byref(o), stream.cuda_stream)
        if rc:
            raise RuntimeError(f"pft3d_mesh failed: {pft.status_string(rc)}")
        return lib.pft_last_launch_count()

    for _ in range(args.warmup):
        step(opts)
    torch.cuda.synchronize()
    if pft.pft_status(ws) != 0:
        raise RuntimeError("device status after warm-up: " + pft.status_string(pft.pft_status(ws)))

    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    clocks = ClockSampler(uuid if uuid.startswith("GPU-") else "GPU-" + uuid)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches = 0
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()                                   # L2 flushed between steps (outside the step events)
        o = pft.make_options({**tune, "main_start_event": e_main[k][0].cuda_event,
                              "main_stop_event": e_main[k][1].cuda_event})
        e_step[k][0].record(stream)
        launches += step(o)
        e_step[k][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms_step = float(np.mean([a.elapsed_time(b) for a, b in e_step]))
    ms_main = float(np.mean([a.elapsed_time(b) for a, b in e_main]))
    ms_step, ms_main = max_over_ranks([ms_step, ms_main], dev)
    status = pft.pft_status(ws)

    # end to end: pinned host buffers, H2D of the inputs and D2H of the result inside the timed region
    hv, hf, hq = (torch.from_numpy(a).pin_memory() for a in (v, f, q))
    hout = torch.empty(q.shape[0], 2, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(max(1, args.e2e_steps)):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        vd.copy_(hv, non_blocking=True)
        fd.copy_(hf, non_blocking=True)
        qd.copy_(hq, non_blocking=True)
        step(opts)
        hout.copy_(out, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_t = float(np.mean(e2e_ms))
    e2e_t = max_over_ranks([e2e_t], dev)[0]

    # variants: the same workload with face_series_tau = 3 (no extra-long series) and 1 (short
    # series only, edge sum wherever the in-face phase spread reaches 1); one warm-up and one
    # timed call each
    variants, variant_out = [], []
    out_main = out.clone()          # result of the benchmarked configuration (checked against the oracle)
    f_pairs, n_pairs = None, 0
    if not args.no_extra and world == 1:
        # the faces reordered into pairs that share an edge (host helper), for the paired variant
        t_pair = time.perf_counter()
        f_pairs, n_pairs = pft.pair_faces(f)
        t_pair = time.perf_counter() - t_pair
        fd_pairs = torch.from_numpy(f_pairs).to(dev)
        for vt, paired in ((3.0, False), (1.0, False), (1.0, True)):
            ov = dict(tune, face_series_tau=vt, face_pairs=n_pairs if paired else 0)
            faces_dev = fd_pairs if paired else fd
            step(pft.make_options(ov), faces_dev)
            flush.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record()
            eb.record()
            a.record(stream)
            step(pft.make_options({**ov, "main_start_event": ea.cuda_event, "main_stop_event": eb.cuda_event}),
                 faces_dev)
            b.record(stream)
            b.synchronize()
            vr = {"face_series_tau": vt, "value": pairs / (a.elapsed_time(b) / 1e3) / 1e9, "unit": UNIT,
                  "ms_per_step": a.elapsed_time(b), "main_kernel_ms": ea.elapsed_time(eb),
                  "device_status": int(pft.pft_status(ws))}
            if paired:
                vr["face_pairs"] = {"pairs": n_pairs, "faces_paired": 2 * n_pairs / f.shape[0],
                                    "host_pairing_s": t_pair}
            variants.append(vr)
            variant_out.append(out.clone())

    if rank == 0:
        pk, pk_kind = peaks()
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        clk_max = float(pk.get("sm_max_mhz", 2070.0))
        qk = kernel_order(pft, q, qd, args.q_per_thread, args.block_threads, f.shape[0])
        mix = branch_mix(v, f, qk, tau=args.tau or 6.0, r=args.q_per_thread, nt=args.block_threads)
        sfu_e = edge_sfu_sinc(v, f, qk, tau=args.tau or 6.0, r=args.q_per_thread, nt=args.block_threads)
        paired = args.q_per_thread % 2 == 0        # even R: Q points in paired FP32 registers
        ops, lanes, achieved, peak_ops = roofline(pairs, ms_main / 1e3, mix, n_sm, clk_max, paired, sfu_e)
        for variant in variants:
            if "face_pairs" in variant:
                vkw = dict(tau=variant["face_series_tau"], r=args.q_per_thread, nt=args.block_threads,
                           n_pairs=n_pairs)
                vf = f_pairs
            else:
                vkw = dict(tau=variant["face_series_tau"], r=args.q_per_thread, nt=args.block_threads)
                vf = f
            vmix = branch_mix(v, vf, qk, **vkw)
            v_sfu = edge_sfu_sinc(v, vf, qk, **vkw)
            _, _, v_ach, v_peak = roofline(pairs, variant["main_kernel_ms"] / 1e3, vmix, n_sm, clk_max, paired,
                                           v_sfu)
            variant["branch_fractions"] = vmix
            variant["edge_sfu_sinc_per_pair"] = v_sfu
            variant["roofline_frac"] = v_ach / v_peak
        value = whole_job_rate(world, pairs, ms_step)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][0], "faces": int(f.shape[0]),
                       "q_points": int(q.shape[0]), "pairs_per_step": pairs,
                       "launch": {"q_per_thread": args.q_per_thread, "block_threads": args.block_threads,
                                  "face_series_tau": opts.face_series_tau or 6.0}, "edge_terms_per_step": 3 * pairs,
                       "l2": "flushed between steps (512 MB write outside the step events)",
                       "parallelism": f"independent replicas x{world}" if world > 1 else "single GPU",
                       "wall_s_timed_region": t_wall, "device_status": int(status)},
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                         "unit": "Tops/s", "frac": achieved / peak_ops,
                         "traffic": traffic_from_profile(),
                         "kernel": f"k_fwd<Pol3F32,{args.q_per_thread},{args.block_threads}>",
                         "main_kernel_ms": ms_main,
                         "peak_basis": (f"{n_sm} SMs x 128 FP32 lanes x {clk_max:.0f} MHz ({pk_kind} max SM "
                                        "clock); paired FP32 instructions keep issue below the FP32 lanes, so "
                                        "achieved counts FP32-pipe operations" if paired else
                                        f"{n_sm} SMs x 128 FP32/SFU issue slots x {clk_max:.0f} MHz "
                                        f"({pk_kind} max SM clock)"),
                         "ops_per_pair": {"fp32": ops["fp32"], "sfu": ops["sfu"]},
                         "branch_fractions": mix, "edge_sfu_sinc_per_pair": sfu_e},
            "clocks": clk,
            "gpu_launches": launches,
            "e2e": {"value": whole_job_rate(world, pairs, e2e_t), "unit": UNIT,
                    "h2d_bytes_per_step": int(v.nbytes + f.nbytes + q.nbytes),
                    "d2h_bytes_per_step": int(q.shape[0] * 16)},
        }
        if clk and clk.get("sm_mhz"):
            line["roofline"]["frac_at_measured_clock"] = achieved / (peak_ops * clk["sm_mhz"] / clk_max)
        # the same main-kernel rate against the fixed per-triangle count of the edge sum (82 FP32-pipe +
        # 7 SFU operations), which ignores that most warps take the cheaper series of the face integral
        line["roofline"]["frac_vs_survey_count"] = survey_count_frac(pairs, ms_main / 1e3, n_sm, clk_max)
        line["roofline"]["survey_count_basis"] = (f"{SURVEY_COUNT['fp32']} FP32-pipe + {SURVEY_COUNT['sfu']} SFU "
                                                  "ops per (Q, triangle) for every pair, bound max(fp32/128, "
                                                  "sfu/16) SM cycles per pair")
        sub = synth_c5_sub(q) if args.workload == "c5" else None
        got32 = out_main.cpu().numpy()
        got32 = got32[:, 0] + 1j * got32[:, 1]
        f64 = None
        if not args.no_extra and world == 1 and sub is not None:
            fp64, f64 = bench_fp64(pft, vd, fd, qd, sub, dev)
            line["fp64_gpu"] = fp64
        if not args.no_cpu and world == 1 and sub is not None:
            cb, ref = cpu_baseline(v, f, q, sub)
            iz = int(np.flatnonzero(np.all(q[sub] == 0, axis=1))[0])
            vol = float(np.real(ref[iz]))
            parity = {"sample": f"{sub.size} seeded Q points incl. Q = 0, all triangles",
                      "measure": "|F - F_oracle| / V (V = F_oracle(0), the volume)",
                      "fp32": err_stats(got32[sub], ref, vol)}
            if f64 is not None:
                parity["fp64_gpu"] = err_stats(f64, ref, vol)
                parity["fp32_vs_fp64_gpu"] = err_stats(got32[sub], f64, vol)
            cb["max_abs_err_vs_oracle_over_volume"] = parity["fp32"]["max"]
            line["cpu_baseline"] = cb
            line["parity_vs_oracle"] = parity
            for variant, vo in zip(variants, variant_out):
                gv = vo.cpu().numpy()[sub]
                variant["max_abs_err_vs_oracle_over_volume"] = float(
                    np.max(np.abs(gv[:, 0] + 1j * gv[:, 1] - ref)) / vol)
        if variants:
            line["variants"] = variants
        if not args.no_extra and world == 1:
            line["other_paths"] = {"batched2d_4096stars_q64x64": bench_batched(dev, args.warmup, args.steps),
                                   "adjoint3d_union16icospheres4_q32cubed": bench_adjoint(dev, args.warmup,
                                                                                          args.steps),
                                   "polymesh3d_star65536prism_q64cubed": bench_polymesh(dev, args.warmup,
                                                                                        args.steps),
                                   "batched3d_1024meshes_q32cubed": bench_batched3d(dev, args.warmup, args.steps),
                                   "sphere_vs_voxels_qx": bench_sphere_voxels(dev)}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
