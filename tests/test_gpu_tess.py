"""Tessellation parity: CUDA path (through the C ABI) against the FP64 oracle.

Bar: exact rib counts per link and exact tags on every link the oracle does not
flag as fragile for the precision in use; vertices within the conditioning-aware
bound of tests/_parity.py; cumulative arc length within 1e-5 relative (absolute
1e-5 px below s = 1 px)."""
import math

import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W
from tests._parity import compare_tess, gpu_tessellate

pytestmark = pytest.mark.gpu

PLAIN, MIXED = 0, 1
# angle error of the FP32 kernel's angle pipeline (atan2f, psi accumulation,
# sincosf), rad, for its diagnostic bound; None: the contract bar (mixed)
EPS_ANG = {PLAIN: 4e-6, MIXED: None}
FRAG = {PLAIN: oracle.FRAGILE32, MIXED: oracle.FRAGILE64}


def _check(batch, prec, s_rel=1e-5, max_fragile_frac=2e-3):
    o = oracle.tessellate(batch)
    g = gpu_tessellate(batch, prec)
    assert g["status"] == 0, g["status"]
    stats, fails = compare_tess(o, g, batch, FRAG[prec], EPS_ANG[prec], s_rel=s_rel)
    print(batch.name, "prec", prec, stats)
    assert not fails, fails
    assert stats["count_mismatch_fragile"] <= max(2, max_fragile_frac * stats["links"])
    return o, g, stats


@pytest.mark.parametrize("prec", [PLAIN, MIXED])
def test_c1_plain_small(prec):
    _check(W.c1_plain_small(), prec)


@pytest.mark.parametrize("prec", [PLAIN, MIXED])
def test_c2_batching_subset(prec):
    _check(W.c2_batching(n_paths=300, seed=W.SEED_BASE + 2), prec)


def test_c5_shape_subset():
    _check(W.c5_differentiation(n_paths=64), MIXED)


def _edge_batches():
    L, Q, C, K = W.LINE, W.QUAD, W.CUBIC, W.CONIC
    out = {}
    out["cusp"] = W.single(C, [[0, 0], [100, 100], [0, 100], [100, 0]], width=6, dtheta_deg=4)
    out["loop"] = W.single(C, [[0, 0], [150, 100], [-50, 100], [100, 0]], width=6, dtheta_deg=1)
    out["serpentine2"] = W.single(C, [[86, 54], [30, 42], [3, 12], [67, 65]], width=3, dtheta_deg=1)
    out["quad"] = W.single(Q, [[0, 0], [50, 80], [50, 80], [100, 0]], width=5)
    out["conics"] = W.single([K, K, K], [[[0, 0], [50, 50], [50, 50], [100, 0]],
                                         [[100, 0], [150, -50], [150, -50], [200, 0]],
                                         [[200, 0], [250, 60], [250, 60], [300, 0]]],
                             w=[0.7, 3.0, -0.5], width=4, dtheta_deg=1)
    # external ellipses (-1 < w < 0, the complementary arcs), and w = 0 (the chord)
    R = 60.0
    ext = [[[R, 0], [R, R], [R, R], [0, R]], [[0, R], [-40, 90], [-40, 90], [-80, 20]],
           [[-80, 20], [-60, -30], [-60, -30], [-20, -40]],
           [[-20, -40], [10, -10], [10, -10], [30, -60]], [[30, -60], [60, -20], [60, -20], [90, -50]]]
    out["external_conics"] = W.single([K] * 5, ext, w=[-math.cos(math.pi / 4), -0.05, -0.5, -0.95, 0.0],
                                      width=5, join=W.JOIN_ROUND, cap=W.CAP_ROUND, dtheta_deg=1)
    out["coincident"] = W.single([C, C, Q], [[[0, 0], [0, 0], [40, 30], [60, 0]],
                                             [[60, 0], [80, 10], [90, 0], [90, 0]],
                                             [[90, 0], [90, 0], [90, 0], [120, 40]]], width=4)
    out["collinear_backtrack"] = W.single(C, [[0, 0], [30, 0], [-10, 0], [10, 0]], width=4)
    out["zero_length_mid"] = W.single([L, C, L], [[[0, 0], [0, 0], [10, 0], [10, 0]],
                                                  [[10, 0], [10, 0], [10, 0], [10, 0]],
                                                  [[10, 0], [10, 0], [10, 10], [10, 10]]],
                                      width=2, join=W.JOIN_BEVEL)
    ang = [30, 90, 150, -45, -120, 179, 180]
    for style in (W.JOIN_BEVEL, W.JOIN_MITER, W.JOIN_MITER_TRUNCATE, W.JOIN_ROUND, W.JOIN_TRIANGLE,
                  W.JOIN_NONE):
        pts, x, y, h = [], 0.0, 0.0, 0.0
        for a in ang:
            nx, ny = x + 20 * math.cos(h), y + 20 * math.sin(h)
            pts.append([[x, y], [x, y], [nx, ny], [nx, ny]])
            x, y, h = nx, ny, h + math.radians(a)
        out[f"joins_{style}"] = W.single([L] * len(pts), pts, width=6, join=style, miter=2.0)
    for cap in (W.CAP_BUTT, W.CAP_SQUARE, W.CAP_ROUND, W.CAP_TRIANGLE):
        out[f"cap_{cap}"] = W.single(C, [[0, 0], [30, 40], [60, -40], [90, 0]], width=8, cap=cap)
    closed = [[[0, 0], [0, 0], [40, 0], [40, 0]], [[40, 0], [60, 20], [60, 20], [40, 40]],
              [[40, 40], [40, 40], [0, 40], [0, 40]], [[0, 40], [0, 40], [0, 0], [0, 0]]]
    out["closed"] = W.single([L, Q, L, L], closed, width=4, join=W.JOIN_ROUND, closed=1)
    return out


EDGES = _edge_batches()


@pytest.mark.parametrize("name", sorted(EDGES))
@pytest.mark.parametrize("prec", [PLAIN, MIXED])
def test_edge_cases(name, prec):
    if name == "collinear_backtrack" and prec == PLAIN:
        pytest.skip("exact collinearity is not decidable in FP32 differences")
    _check(EDGES[name], prec)


def test_external_parabola_and_hyperbola_are_rejected():
    """w_B <= -1: the curve passes through infinity; the link is an error (status
    PS_ERR_INVALID) and emits nothing, and the oracle refuses the batch."""
    import paper_2007_00308_gb300 as ps
    b = W.single([W.LINE, W.CONIC], [[[0, 0], [0, 0], [50, 0], [50, 0]],
                                     [[50, 0], [100, 60], [100, 60], [150, 0]]],
                 w=[1.0, -1.5], width=4)
    with pytest.raises(oracle.OracleError):
        oracle.tessellate(b)
    for prec in (PLAIN, MIXED):
        g = gpu_tessellate(b, prec)
        assert g["status"] == ps.PS_ERR_INVALID
        assert np.diff(g["link_rib_off"])[3] == 0  # the conic's link


def test_empty_and_degenerate_paths():
    L = W.LINE
    pts = np.array([[[0, 0], [0, 0], [0, 0], [0, 0]], [[5, 5], [5, 5], [5, 5], [5, 5]],
                    [[0, 0], [0, 0], [10, 0], [10, 0]]], np.float32)
    b = W.make_batch("degenerate", [L, L, L], pts, [1, 1, 1], [0, 2, 1], 2.0, W.JOIN_ROUND,
                     W.CAP_ROUND)
    for prec in (PLAIN, MIXED):
        o = oracle.tessellate(b)
        g = gpu_tessellate(b, prec)
        assert g["R"] == len(o["s"])
        assert np.array_equal(np.diff(g["link_rib_off"]), o["link_nrib"])
        assert np.array_equal(g["path_rib_off"], o["path_rib_off"])


def test_c3_large_path_full():
    _check(W.c3_large_path(), MIXED)


def test_c4_precision_subset_mixed_beats_fp32():
    b = W.c4_precision(n=4000)
    o = oracle.tessellate(b)
    res = {}
    for prec in (PLAIN, MIXED):
        g = gpu_tessellate(b, prec)
        stats, fails = compare_tess(o, g, b, FRAG[prec], EPS_ANG[prec])
        res[prec] = stats
        print("c4 prec", prec, stats)
    assert res[MIXED]["count_mismatch_nonfragile"] == 0
    assert res[MIXED]["vertex_ratio_max"] <= 1.0 and res[MIXED]["s_ratio_max"] <= 1.0
    assert res[MIXED]["count_mismatch_nonfragile"] + res[MIXED]["count_mismatch_fragile"] <= \
        res[PLAIN]["count_mismatch_nonfragile"] + res[PLAIN]["count_mismatch_fragile"]


def test_capacity_overflow_is_reported():
    import torch
    import paper_2007_00308_gb300 as ps
    b = W.c1_plain_small()
    ctx = ps.Context()
    db = ps.DeviceBatch(b)
    out = ps.TessOutput(db.n_link, db.n_path, 100, arclength=True)
    ps.ps_tessellate_strokes(ctx, db, out, ps.PS_PREC_FP32, ps.PS_TESS_ARCLENGTH)
    torch.cuda.synchronize()
    assert ctx.status() == ps.PS_ERR_CAPACITY
    assert int(out.n_rib.item()) == len(oracle.tessellate(b)["s"])
    with pytest.raises(ps.PolarStrokeError):
        ps.ps_tessellate_strokes(ctx, db, out, 7, ps.PS_TESS_ARCLENGTH)
    with pytest.raises(ps.PolarStrokeError):
        ps.ps_tessellate_strokes(ctx, db, out, 0, ps.PS_TESS_ARCLENGTH, dtheta=0.0)


def test_standalone_arclength_matches_fused():
    import torch
    import paper_2007_00308_gb300 as ps
    b = W.c1_plain_small()
    g = gpu_tessellate(b, MIXED)
    out, ctx = g["out"], g["ctx"]
    s2 = torch.empty_like(out.s)
    pl2 = torch.empty_like(out.path_len)
    ps.ps_arclength_scan(ctx, out.rib, out.tag, out.n_rib, out.capacity, s2, pl2, b.n_path)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    s2 = s2[:g["R"]].cpu().numpy().astype(np.float64)
    o = oracle.tessellate(b)
    # midpoints of FP32 ribs carry ~ulp(coordinate) error per rib; it telescopes
    tol = 1e-5 * np.maximum(o["s"], 1.0) + 4e-4
    assert np.all(np.abs(s2 - o["s"]) <= tol), np.abs(s2 - o["s"]).max()
