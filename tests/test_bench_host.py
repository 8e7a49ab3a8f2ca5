"""Host-side pieces of bench.py: the branch-mix mirror of the kernel's rule and
the roofline arithmetic (no GPU needed)."""
import numpy as np
import pytest

import bench
from paper_2104_08309_gb300 import synth


@pytest.fixture(scope="module")
def mesh():
    v, f = synth.perturbed_icosphere(4, seed=2, amp=0.05)
    return v, f


def test_branch_fractions_partition_the_pairs(mesh):
    v, f = mesh
    q = synth.q_grid_3d(32, 60.0)
    for tau in (0.5, 1.0, 2.0, 3.0, 4.5, 6.0):
        m = bench.branch_mix(v, f, q, tau=tau, n_warps=512)
        assert set(m) == set(bench.OPS)
        assert abs(sum(m.values()) - 1.0) < 1e-12
        # no form beyond the one whose bound covers p_hi = tau^2/4
        for name, b in bench.SERIES_BOUNDS:
            if 0.25 * tau * tau <= b:
                later = [k for k in list(bench.OPS)[list(bench.OPS).index(name) + 1:] if k.startswith("series")]
                assert all(m[k] == 0.0 for k in later), (tau, name)
                break
    lo = bench.branch_mix(v, f, q, tau=1.0, n_warps=512)
    hi = bench.branch_mix(v, f, q, tau=3.0, n_warps=512)
    # the same seeded sample: raising tau only moves warps from the edge sum into the series,
    # and warps with every P < 1/4 keep the k <= 7 form
    assert hi["edge_sum"] <= lo["edge_sum"]
    assert hi["series_k7"] == lo["series_k7"]


def test_branch_rule_on_hand_made_phases():
    """One face, Q points along its normal (all phases 0 -> the k <= 7 form) and in its plane
    at |Q| where P falls into each form's interval, or above tau^2/4 (edge sum)."""
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    f = np.array([[0, 1, 2]], np.int32)
    along = np.tile([[0.0, 0.0, 5.0]], (256, 1))
    m = bench.branch_mix(v, f, along, tau=3.0, r=2, nt=128, n_warps=16)
    assert m["series_k7"] == 1.0
    # a0 = Q.(p0 - g) with g = (1/3, 1/3, 0): Q = (k, 0, 0) gives a = (-k/3, 2k/3, -k/3), P = k^2/3
    mix = lambda k, tau: bench.branch_mix(v, f, np.tile([[k, 0.0, 0.0]], (256, 1)), tau=tau, r=2, nt=128,
                                          n_warps=16)
    for k, form in ((0.75, "series_k7"), (1.5, "series_k9"), (2.25, "series_k11"), (3.0, "series_k13"),
                    (4.0, "series_k17"), (5.0, "series_k17")):   # P = 0.1875, 0.75, 1.6875, 3, 5.33, 8.33
        assert mix(k, 6.0)[form] == 1.0, (k, form)
    assert mix(1.5, 1.0)["edge_sum"] == 1.0
    assert mix(1.5, 3.0)["series_k9"] == 1.0
    assert mix(4.0, 3.0)["edge_sum"] == 1.0


def test_roofline_arithmetic():
    mix = {b: 1.0 / len(bench.OPS) for b in bench.OPS}
    want = {k: sum(bench.OPS[b][k] for b in bench.OPS) / len(bench.OPS) for k in ("fp32", "sfu")}
    # scalar code: issue-bound, every FP32 and SFU operation takes one of 128 slots per SM clock
    ops, issue, achieved, peak = bench.roofline(1e12, 1.0, mix, 152, 2070.0, paired=False)
    assert ops == pytest.approx(want)
    assert issue == pytest.approx(want["fp32"] + want["sfu"])
    assert achieved == pytest.approx(issue * 1e12)
    assert peak == pytest.approx(152 * 128 * 2070e6)
    # paired code: the 128 FP32 lanes bind, and only FP32-pipe operations count against them
    ops, lanes, achieved_p, peak_p = bench.roofline(1e12, 1.0, mix, 152, 2070.0, paired=True)
    assert lanes == pytest.approx(want["fp32"])
    assert achieved_p == pytest.approx(want["fp32"] * 1e12)
    assert peak_p == pytest.approx(152 * 128 * 2070e6)
    # the pair rate at the limit: 128 / fp32 pairs per SM clock, against 128 / (fp32 + sfu)
    assert achieved_p / peak_p < achieved / peak


def test_sfu_sinc_fraction_on_a_square():
    """Unit square (sides along x and y), Q = (1, 0) and (10, 0): only the two x-directed sides at
    |Q| = 10 have |Q.D/2| = 5 > pi, i.e. a quarter of the (segment, Q) pairs."""
    v = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float32)
    off = np.array([0, 4])
    q = np.array([[1.0, 0.0], [10.0, 0.0]])
    assert bench.sfu_sinc_fraction(v, off, q) == pytest.approx(0.25, abs=0.01)
    # two polygons: the second (a tiny triangle) never needs the SFU sinc
    v2 = np.concatenate([v, 0.01 * np.array([[0, 0], [1, 0], [0, 1]], np.float32)])
    off2 = np.array([0, 4, 7])
    assert bench.sfu_sinc_fraction(v2, off2, q) == pytest.approx(0.25 * 4 / 7, abs=0.01)


def test_roofline2d_bounds():
    r0 = bench.roofline2d(1e12, 1.0, 0.0, 152, 2070.0, paired=False)
    assert r0["bound"] == "alu"
    assert r0["peak_gpair_s"] == pytest.approx(152 * 2070e6 * 128 / 20 / 1e9)
    r1 = bench.roofline2d(1e12, 1.0, 1.0, 152, 2070.0, paired=False)
    assert r1["bound"] == "sfu"                      # 4 SFU results / 16 lanes > 28 issue slots / 128
    assert r1["peak_gpair_s"] == pytest.approx(152 * 2070e6 * 16 / 4 / 1e9)
    p0 = bench.roofline2d(1e12, 1.0, 0.0, 152, 2070.0, paired=True)
    assert p0["bound"] == "alu"                      # 18 FP32 ops / 128 lanes > 2 SFU / 16
    assert p0["peak_gpair_s"] == pytest.approx(152 * 2070e6 * 128 / 18 / 1e9)
    p1 = bench.roofline2d(1e12, 1.0, 1.0, 152, 2070.0, paired=True)
    assert p1["bound"] == "sfu" and p1["peak_gpair_s"] == pytest.approx(r1["peak_gpair_s"])


def test_traffic_figure_only_for_the_profiled_sources(monkeypatch):
    """roofline.traffic comes from the committed ncu summary while the kernel sources hash to the value
    recorded there, and is None as soon as they differ."""
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    path = bench.os.path.join(bench.ROOT, "profiles", "k_fwd_dram_icosphere8_q128cubed.txt")
    kv = dict(l.split(":", 1) for l in open(path).read().splitlines() if ":" in l)
    recorded = kv["source_sha256_16"].strip()
    t = bench.traffic_from_profile()
    if recorded == h:
        assert t == float(kv["dram_bytes_per_launch_full_size"])
        assert t == float(kv["dram_bytes_read"]) + float(kv["dram_bytes_write"])
    else:
        assert t is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.traffic_from_profile() is None


def _fn_body(name):
    import os
    import re
    text = open(os.path.join(bench.ROOT, "paper_2104_08309_gb300", "csrc", "pft_pairs.cuh")).read()
    i = text.index(name)
    body = text[text.index("{", i) + 1:text.index("\n}\n", i)]
    return re.sub(r"//[^\n]*", "", body)


def _arith_ops(body):
    """FP32-pipe operations written in a device function body: each fmaf, each binary * + -
    between operands, and each call of the scalar-or-packed helpers vfma / vmul / vadd (one
    operation per Q point; unary minus, also as vneg, folds into the FMA or multiply, so it is
    not counted)."""
    import re
    n = body.count("fmaf(") + body.count("vfma(") + body.count("vmul(") + body.count("vadd(")
    n += len(re.findall(r"[\w\)\]] \* [\w\(-]", body))
    n += len(re.findall(r"[\w\)\]] [+-] [\w\(]", body))
    return n


def test_ops_table_matches_the_source():
    """bench.OPS is the roofline's per-pair operation count: each series form's entry is the 25
    operations outside the series plus the arithmetic written in its function, and the 16
    projection operations (mu, a0, a1, s, then s1, p1, P, T) are those of face_common_pt."""
    assert _arith_ops(_fn_body("void face_common_pt(")) == 16
    # the finish: 6 written here plus the argument scaling inside __sincosf = the 7 of the count
    assert _arith_ops(_fn_body("void face_finish(")) == 6
    forms = {"series_k7": "void face_series(", "series_k9": "void face_series_k9(",
             "series_k11": "void face_series_long(", "series_k13": "void face_series_k13(",
             "series_k17": "void face_series_xlong("}
    for key, fn in forms.items():
        assert bench.OPS[key]["fp32"] == 25 + _arith_ops(_fn_body(fn)), key
        assert bench.OPS[key]["sfu"] == 2


def test_survey_count_fraction_and_error_stats():
    # 82 FP32-pipe ops per pair on 128 lanes bound the SFU's 7/16: 0.640625 SM cycles per pair
    n_sm, clk = 152, 2070.0
    peak = n_sm * clk * 1e6 / (82 / 128)
    assert abs(bench.survey_count_frac(peak * 2.0, 2.0, n_sm, clk) - 1.0) < 1e-12
    assert abs(bench.survey_count_frac(peak * 0.5, 1.0, n_sm, clk) - 0.5) < 1e-12
    got = np.array([1.0, 2.0, 3.0 + 1j, 4.0]) + 0j
    ref = np.array([1.0, 2.5, 3.0, 1.0]) + 0j
    st = bench.err_stats(got, ref, -2.0)      # |errors| / 2 = 0, 0.25, 0.5, 1.5
    assert st["max"] == 1.5 and st["median"] == 0.375
    assert abs(st["p99"] - (0.5 + 0.97 * 1.0)) < 1e-12


def _bwd_body(start, stop=None, struct=False):
    """Text of pft_bwd.cu from `start` to `stop` (or to the end of the function / struct), comments
    removed."""
    import os
    import re
    text = open(os.path.join(bench.ROOT, "paper_2104_08309_gb300", "csrc", "pft_bwd.cu")).read()
    text = re.sub(r"//[^\n]*", "", text)
    i = text.index(start)
    j = text.index(stop, i) if stop else text.index("\n};\n" if struct else "\n}\n", i)
    return text[i:j]


def _ops_no_literal_products(body):
    """FP32-pipe operations a device-code body executes: each fmaf and each call of the packed
    helpers vfma / vmul / vadd, and each binary * + - whose operands are not both numeric literals
    (those products are folded by the compiler; a chain a * b * c counts two); the body of each
    `for (int l = 0; l < 3; ++l)` loop counts three times (the loops are unrolled)."""
    import re
    lit = r"(?<![\w.])\d+\.?\d*(?:e[-+]?\d+)?f?(?![\w.])"

    def flat(text):
        n = sum(text.count(f + "(") for f in ("fmaf", "vfma", "vmul", "vadd"))
        b = re.sub(lit, "LIT", text)
        for m in re.finditer(r"(?<=[\w\.\)\]]) ([*+-]) (?=-?[\w\.\(])", b):
            left = re.search(r"([\w\.]+|\))$", b[:m.start()])
            right = re.match(r"-?([\w\.]+|\()", b[m.end():])
            if not (left and right and left.group(1) == "LIT" and right.group(1) == "LIT"):
                n += 1
        return n

    n = flat(body)
    head = "for (int l = 0; l < 3; ++l)"
    k = body.find(head)
    while k >= 0:
        a = k + len(head)
        rest = body[a:].lstrip()
        if rest.startswith("{"):
            depth, e = 0, a + body[a:].index("{")
            for e in range(e, len(body)):
                depth += {"{": 1, "}": -1}.get(body[e], 0)
                if depth == 0:
                    break
            loop = body[a:e + 1]
        else:
            loop = body[a:body.index(";", a) + 1]
        n += 2 * flat(loop)
        k = body.find(head, a)
    return n


def test_adjoint_ops_table_matches_the_source():
    """bench.OPS_ADJ / OPS_QADJ: each branch part is the arithmetic that branch of face_adj_t and
    its adjoint execute; the edge part adds three sinc_d on their polynomial path (with the range
    test; the SFU form beyond |u| > pi is the rare branch) and the record or Q updates of the X
    adjoint; the common part adds face_common, the 10 branch-selection operations, the sincos
    scaling, the code after the branches and the 12 record or Q updates."""
    c = _ops_no_literal_products
    fwd = {"short": c(_bwd_body("if (shorts) {", "} else if (k9s) {")),
           "k9": c(_bwd_body("} else if (k9s) {", "} else if (longs) {")),
           "long": c(_bwd_body("} else if (longs) {", "} else if (series) {")),
           "xlong": c(_bwd_body("} else if (series) {", "} else {\n    const float nx"))}
    series_adj = c(_bwd_body("if (series) {\n    const float Pb", "} else {\n    const float Sr"))
    edge_fwd = c(_bwd_body("} else {\n    const float nx", "const float Wr"))
    edge_adj = c(_bwd_body("} else {\n    const float Sr", "out.common("))
    post = c(_bwd_body("const float Wr", "float a0b, a1b;"))
    sinc_d = c(_bwd_body("void sinc_d(", "constexpr int kE")) + 1   # polynomial path + range test
    rec_edge = c(_bwd_body("void edge(float b0b", "__device__ __forceinline__ void common"))
    q_edge = c(_bwd_body("void edge(float, float", "__device__ __forceinline__ void common"))
    assert (rec_edge, q_edge) == (12, 6)
    # hand counts: the short series' 17, the edge sum's forward 38 and adjoint 62, sinc_d's 14 + 1
    assert (fwd["short"], edge_fwd, edge_adj, sinc_d) == (17, 38, 62, 15)
    assert _arith_ops(_fn_body("void face_common(")) == 15
    for key in ("short", "k9", "long", "xlong"):
        assert bench.OPS_ADJ[key]["fp32"] == fwd[key] + series_adj, key
        assert bench.OPS_QADJ[key]["fp32"] == fwd[key] + series_adj, key
    # two sincos argument scalings and the 1/|X|^2 test and select are not written as arithmetic
    assert bench.OPS_ADJ["edge"]["fp32"] == edge_fwd + 3 * sinc_d + 2 + 2 + edge_adj + rec_edge
    assert bench.OPS_QADJ["edge"]["fp32"] == edge_fwd + 3 * sinc_d + 2 + 2 + edge_adj + q_edge
    # common: projections 15, branch selection 10, sincos(mu) scaling 1, the code after the branches
    # (whose two products -s W feed only the Q-gradient's own term), 12 updates (+2 adds for QAdj)
    assert bench.OPS_ADJ["common"]["fp32"] == 15 + 10 + 1 + (post - 2) + 12
    assert bench.OPS_QADJ["common"]["fp32"] == 15 + 10 + 1 + post + 2 + 12
    assert bench.OPS_ADJ["edge"]["sfu"] == 5 and bench.OPS_ADJ["common"]["sfu"] == 2


def test_2d_adjoint_ops_match_the_source():
    """bench.OPS2D_ADJ: seg_adj's arithmetic plus sinc_d's polynomial path, its range test and the
    sincos argument scaling; the SFU sinc adds sinc_d's quotients and the turn reduction (rint,
    subtract, scale) with the sincos argument scaling."""
    c = _ops_no_literal_products
    seg = c(_bwd_body("void seg_adj("))
    poly = c(_bwd_body("void sinc_d(", "constexpr int kE"))
    large = c(_bwd_body("constexpr int kE", "void seg_adj("))
    assert (seg, poly, large) == (21, 14, 4)
    assert bench.OPS2D_ADJ["poly_sinc"] == {"fp32": seg + poly + 1 + 1, "sfu": 2}
    assert bench.OPS2D_ADJ["sfu_sinc"] == {"fp32": seg + poly + 1 + 1 + large + 3 + 1, "sfu": 2 + 3}


def test_adjoint_branch_mix_partitions_the_lanes(mesh):
    v, f = mesh
    q = synth.q_grid_3d(24, 40.0)
    for lanes in ("faces", "q"):
        for tau in (0.5, 1.0, 3.0, 6.0):
            lane, warp = bench.adjoint_branch_mix(v, f, q, tau=tau, lanes=lanes, n_warps=256)
            assert abs(sum(lane.values()) - 1.0) < 1e-12
            assert all(warp[k] >= lane[k] for k in lane)
            ops = bench.adjoint_ops(warp, bench.OPS_ADJ)
            assert bench.OPS_ADJ["common"]["fp32"] < ops["fp32"] <= sum(x["fp32"] for x in bench.OPS_ADJ.values())
            if tau <= 3.0:
                assert lane["xlong"] == 0.0


def test_branch_mix_with_pairs_splits_the_edge_sums(mesh):
    """Pairing moves edge-sum units into edge_sum_shared and leaves every other fraction as it was."""
    import paper_2104_08309_gb300 as pft
    v, f = mesh
    fp, n = pft.pair_faces(f)
    q = synth.q_grid_3d(32, 60.0)
    plain = bench.branch_mix(v, fp, q, tau=1.0, n_warps=512)
    paired = bench.branch_mix(v, fp, q, tau=1.0, n_warps=512, n_pairs=n)
    assert plain["edge_sum_shared"] == 0.0
    assert abs(paired["edge_sum"] + paired["edge_sum_shared"] - plain["edge_sum"]) < 1e-12
    assert paired["edge_sum_shared"] > 0.5 * plain["edge_sum"]
    for k in plain:
        if not k.startswith("edge"):
            assert paired[k] == plain[k]


def test_edge_sfu_sinc_count():
    """bench.edge_sfu_sinc counts the edges whose sinc the edge sum takes on the SFU.  A triangle
    (0,0,0), (L,0,0), (0,e,0) at Q = (k,0,0) has edge phases u = kL/2, -kL/2, 0 and P = (kL)^2/3:
    kL = 6.5 puts it on the edge sum (P > 9) with two edges past pi; kL = 4 takes a series form
    (P < 9, nothing counted), and at tau = 1 the edge sum with both |u| = 2 < pi."""
    L, e = 1.0, 1e-3
    v = np.array([[0, 0, 0], [L, 0, 0], [0, e, 0]], dtype=np.float32)
    f = np.array([[0, 1, 2]], dtype=np.int32)
    count = lambda kl, tau: bench.edge_sfu_sinc(v, f, np.tile([[kl / L, 0.0, 0.0]], (256, 1)), tau=tau, r=2,
                                                nt=128, n_warps=16)
    assert count(6.5, 6.0) == 2.0
    assert count(4.0, 6.0) == 0.0
    assert count(4.0, 1.0) == 0.0
    assert count(6.5, 1.0) == 2.0
    # a pair sharing its first edge (faces 0 and 1, both on the edge sum): that edge counts half per face
    v2 = np.array([[0, 0, 0], [L, 0, 0], [0, e, 0], [0, -e, 0]], dtype=np.float32)
    f2 = np.array([[0, 1, 2], [1, 0, 3]], dtype=np.int32)
    q2 = np.tile([[6.5 / L, 0.0, 0.0]], (256, 1))
    assert bench.edge_sfu_sinc(v2, f2, q2, tau=6.0, r=2, nt=128, n_warps=64, n_pairs=1) == 1.5
    assert bench.edge_sfu_sinc(v2, f2, q2, tau=6.0, r=2, nt=128, n_warps=64) == 2.0
    # the per-edge price is the 2D SFU sinc's extra over the polynomial one (the same sinc_large code)
    assert bench.OPS_EDGE_SFU_SINC == {k: bench.OPS2D["sfu_sinc"][k] - bench.OPS2D["poly_sinc"][k]
                                       for k in ("fp32", "sfu")}
