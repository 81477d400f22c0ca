"""Raster and dash parity.  Coverage must be bit-exact against the oracle's raster
of the GPU's own vertices; dashing of the GPU's ribs must give the same pieces as
the oracle's dasher on the same ribs."""
import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W
from tests._parity import gpu_tessellate

pytestmark = pytest.mark.gpu


def gpu_raster(g, batch, W_, H_, exact=False):
    import torch
    import paper_2007_00308_gb300 as ps
    canvas = torch.zeros((H_, W_), dtype=torch.int16, device="cuda")
    covered = torch.zeros(batch.n_path, dtype=torch.int64, device="cuda")
    out = g["out"]
    ps.ps_rasterize_coverage(g["ctx"], out.rib, out.tag, out.n_rib, out.capacity, batch.n_path,
                             W_, H_, canvas, covered, exact=exact)
    torch.cuda.synchronize()
    st = g["ctx"].status()
    return canvas.cpu().numpy().view(np.uint16), covered.cpu().numpy().view(np.uint64), st


def _raster_case(name):
    if name == "c1":
        return W.c1_plain_small()
    if name == "c2_small":
        return W.c2_batching(n_paths=120, canvas=512)
    if name == "c5_small":
        return W.c5_differentiation(n_paths=16)
    if name == "bow_ties":
        # wide strokes around tight bends: inner sides fold into bow-tie quads
        pts = [[[20, 100], [220, 20], [-60, 20], [150, 100]],
               [[150, 100], [300, 200], [100, 200], [250, 120]],
               [[250, 120], [330, 60], [330, 60], [380, 130]]]
        return W.single([W.CUBIC, W.CUBIC, W.QUAD], pts, width=46, join=W.JOIN_MITER,
                        cap=W.CAP_BUTT, dtheta_deg=4.0, canvas=(420, 260))
    if name == "crowded":
        # 300 paths on four tiles: more paths per tile than the coverage kernel
        # keeps in shared memory at once (further passes over the tile)
        return W.c2_batching(n_paths=300, canvas=32, mean_segs=3.0, max_segs=6)
    if name == "long_quads":
        # quads with edges over 1024 px (the int64 path of the exact mode)
        pts = [[[10, 30], [10, 30], [1500, 200], [1500, 200]],
               [[1500, 200], [1500, 200], [40, 420], [40, 420]]]
        return W.single([W.LINE, W.LINE], pts, width=9, join=W.JOIN_BEVEL, cap=W.CAP_SQUARE,
                        dtheta_deg=2.0, canvas=(1536, 448))
    raise KeyError(name)


@pytest.mark.parametrize("exact", [False, True])
@pytest.mark.parametrize("name", ["c1", "c2_small", "c5_small", "bow_ties", "long_quads",
                                  "crowded"])
def test_coverage_bit_exact_on_gpu_vertices(name, exact):
    b = _raster_case(name)
    Wd, Ht = b.canvas
    g = gpu_tessellate(b, 1)
    can, cov, st = gpu_raster(g, b, Wd, Ht, exact=exact)
    assert st == 0
    ocan, ocov = oracle.raster(g["rib"], g["tag"], Wd, Ht, b.n_path, exact=exact)
    diff = can != ocan
    assert not diff.any(), f"{diff.sum()} pixels differ"
    assert np.array_equal(cov, ocov)
    assert cov.sum() > 0


def test_dash_matches_oracle_on_gpu_ribs():
    import torch
    import paper_2007_00308_gb300 as ps
    b = W.c3_large_path(n_seg=400)
    g = gpu_tessellate(b, 1)
    out, ctx = g["out"], g["ctx"]
    pattern, offset = b.dash
    od = oracle.dash(g["rib"], g["s"], g["tag"], pattern, offset)
    cap = len(od["s"]) + 16
    orib = torch.empty((cap, 4), dtype=torch.float32, device="cuda")
    os_ = torch.empty(cap, dtype=torch.float32, device="cuda")
    otag = torch.empty(cap, dtype=torch.int32, device="cuda")
    osrc = torch.empty(cap, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    ps.ps_dash(ctx, out.rib, out.s, out.tag, out.n_rib, out.capacity, pattern, offset, orib, os_,
               otag, osrc, n, cap)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    m = int(n.item())
    assert m == len(od["s"])
    # the piece list of each tile is ordered; compare as sets keyed by (src, s)
    gs = os_[:m].cpu().numpy()
    gsrc = osrc[:m].cpu().numpy()
    gk = np.lexsort((gs, gsrc))
    ok_ = np.lexsort((od["s"].astype(np.float32), od["src"]))
    assert np.array_equal(gsrc[gk], od["src"][ok_])
    assert np.array_equal(gs[gk], od["s"].astype(np.float32)[ok_])
    grib = orib[:m].cpu().numpy()
    assert np.array_equal(grib[gk], od["rib"].astype(np.float32)[ok_])
    assert np.array_equal(otag[:m].cpu().numpy().view(np.uint32)[gk], od["tag"][ok_])
    # and the dashed stream rasterizes identically on both sides
    can = torch.zeros((512, 512), dtype=torch.int16, device="cuda")
    cov = torch.zeros(1, dtype=torch.int64, device="cuda")
    ps.ps_rasterize_coverage(ctx, orib, otag, n, cap, 1, 512, 512, can, cov)
    torch.cuda.synchronize()
    ocan, ocov = oracle.raster(grib.astype(np.float64), otag[:m].cpu().numpy().view(np.uint32), 512,
                               512, 1)
    assert np.array_equal(can.cpu().numpy().view(np.uint16), ocan)
    assert int(cov.item()) == int(ocov[0])


@pytest.mark.parametrize("cap", [W.CAP_ROUND, W.CAP_SQUARE, W.CAP_TRIANGLE])
def test_capped_dash_matches_oracle_on_gpu_ribs(cap):
    """Capped dash ends: same order, pieces bit-identical, cap ribs within the
    vertex bound (FP32 sincos about the same boundary ribs), tags and s exact."""
    import torch
    import paper_2007_00308_gb300 as ps
    from tests._parity import ulp32
    b = W.c3_large_path(n_seg=400)
    b.path_cap[:] = cap
    g = gpu_tessellate(b, 1)
    out, ctx = g["out"], g["ctx"]
    pattern, offset = b.dash
    od = oracle.dash_capped(g["rib"], g["s"], g["tag"], pattern, offset, b.path_cap, b.dtheta)
    m = len(od["s"])
    cap_ = m + 16
    orib = torch.empty((cap_, 4), dtype=torch.float32, device="cuda")
    os_ = torch.empty(cap_, dtype=torch.float32, device="cuda")
    otag = torch.empty(cap_, dtype=torch.int32, device="cuda")
    osrc = torch.empty(cap_, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    pc = torch.from_numpy(b.path_cap.astype(np.uint8)).cuda()
    ps.ps_dash_capped(ctx, out.rib, out.s, out.tag, out.n_rib, out.capacity, pattern, offset, pc,
                      b.dtheta, orib, os_, otag, osrc, n, cap_)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert int(n.item()) == m
    gtag = otag[:m].cpu().numpy().view(np.uint32)
    assert np.array_equal(gtag, od["tag"])
    assert np.array_equal(osrc[:m].cpu().numpy(), od["src"])
    assert np.array_equal(os_[:m].cpu().numpy(), od["s"].astype(np.float32))
    grib = orib[:m].cpu().numpy().astype(np.float64)
    piece = ((gtag >> 1) & 1) == 1
    assert np.array_equal(grib[piece], od["rib"].astype(np.float32)[piece].astype(np.float64))
    capr = ~piece
    assert capr.sum() > 0 or cap == W.CAP_BUTT
    err = np.abs(grib[capr] - od["rib"][capr])
    tol = 1e-4 + 4 * ulp32(np.abs(od["rib"][capr]))
    assert (err <= tol).all(), float((err / tol).max())
    # and the capped dashes rasterize identically on both sides
    can = torch.zeros((512, 512), dtype=torch.int16, device="cuda")
    cov = torch.zeros(1, dtype=torch.int64, device="cuda")
    ps.ps_rasterize_coverage(ctx, orib, otag, n, cap_, 1, 512, 512, can, cov)
    torch.cuda.synchronize()
    ocan, ocov = oracle.raster(grib, gtag, 512, 512, 1)
    assert np.array_equal(can.cpu().numpy().view(np.uint16), ocan)
    assert int(cov.item()) == int(ocov[0])


@pytest.mark.parametrize("n_paths", [1000, 1100])
def test_tile_path_limit(n_paths):
    """One 16x16 tile met by n_paths distinct paths: up to 1,024 the coverage
    kernel takes them in passes of 96 (every per-path count bit-exact against the
    oracle's raster of the GPU's vertices); beyond that it records
    PS_ERR_CAPACITY instead of dropping paths silently."""
    import torch
    import paper_2007_00308_gb300 as ps
    rng = np.random.default_rng(n_paths)
    a = rng.uniform(1.0, 6.0, (n_paths, 2))
    d = rng.uniform(10.0, 15.0, (n_paths, 2))
    pts = np.zeros((n_paths, 4, 2))
    pts[:, 0], pts[:, 1], pts[:, 2], pts[:, 3] = a, a, d, d
    pts = np.round(pts * 64) / 64
    b = W.make_batch("tile_limit", [W.LINE] * n_paths, pts, [1.0] * n_paths, [1] * n_paths,
                     rng.uniform(0.5, 2.0, n_paths), W.JOIN_ROUND, W.CAP_BUTT, canvas=(16, 16))
    g = gpu_tessellate(b, 1)
    ctx, out = g["ctx"], g["out"]
    canvas = torch.zeros((16, 16), dtype=torch.int16, device="cuda")
    covered = torch.zeros(n_paths, dtype=torch.int64, device="cuda")
    ps.ps_rasterize_coverage(ctx, out.rib, out.tag, out.n_rib, out.capacity, n_paths, 16, 16,
                             canvas, covered)
    torch.cuda.synchronize()
    st = ctx.status()
    if n_paths <= 1024:
        assert st == ps.PS_OK
        ocan, ocov = oracle.raster(g["rib"], g["tag"], 16, 16, n_paths)
        assert np.array_equal(canvas.cpu().numpy().view(np.uint16), ocan)
        assert np.array_equal(covered.cpu().numpy().view(np.uint64), ocov)
    else:
        assert st == ps.PS_ERR_CAPACITY
