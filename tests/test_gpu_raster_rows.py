"""The raster split of one batch over ranks by canvas rows, on one GPU with the
ranks taken one after another (paper_2007_00308_gb300/shard.py):

- windows of pixel rows (ps_rasterize_coverage_rows) that tile the canvas give
  the whole canvas's masks row for row, and per-path sample counts that sum to
  the whole canvas's;
- a batch cut into link ranges (ps_tessellate_links), each range's quads routed
  to the owners of the rows they reach (ps_route_quads), each owner covering its
  rows from the blocks addressed to it, gives the canvas and the per-path
  counts of ps_rasterize_coverage on the whole batch, bit for bit.
Both coverage rules (two triangles, crossing)."""
import numpy as np
import pytest

from paper_2007_00308_gb300 import shard
from paper_2007_00308_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _case(name):
    if name == "c1":
        return W.c1_plain_small()
    if name == "c2_200":
        return W.c2_batching(n_paths=200, seed=W.SEED_BASE + 2)
    return W.c3_large_path(n_seg=400)


def _whole(ps, ctx, db, b, exact):
    import torch
    out = ps.tessellate(ctx, db, ps.PS_PREC_MIXED, arclength=False)
    Wd, Ht = b.canvas
    canvas = torch.zeros((Ht, Wd), dtype=torch.int16, device="cuda")
    cov = torch.zeros(b.n_path, dtype=torch.int64, device="cuda")
    ps.ps_rasterize_coverage(ctx, out.rib, out.tag, out.n_rib, out.capacity, b.n_path, Wd, Ht,
                             canvas, cov, exact=exact)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    return out, canvas.cpu().numpy(), cov.cpu().numpy()


@pytest.mark.parametrize("exact", [False, True])
@pytest.mark.parametrize("name,G", [("c1", 3), ("c2_200", 4)])
def test_row_windows_tile_the_canvas(name, G, exact):
    import torch
    import paper_2007_00308_gb300 as ps
    b = _case(name)
    ctx = ps.Context()
    db = ps.DeviceBatch(b)
    out, canvas, cov = _whole(ps, ctx, db, b, exact)
    Wd, Ht = b.canvas
    for bounds in (shard.raster_rows(Ht, G), np.array([0, 16, 48, Ht], np.int32)):
        total = np.zeros(b.n_path, np.int64)
        for d in range(len(bounds) - 1):
            y0, h = int(bounds[d]), int(bounds[d + 1] - bounds[d])
            if h == 0:
                continue
            cw = torch.zeros((h, Wd), dtype=torch.int16, device="cuda")
            cv = torch.zeros(b.n_path, dtype=torch.int64, device="cuda")
            ps.ps_rasterize_coverage_rows(ctx, out.rib, out.tag, out.n_rib, out.capacity, b.n_path,
                                          Wd, y0, h, cw, cv, exact=exact)
            torch.cuda.synchronize()
            assert ctx.status() == 0
            assert np.array_equal(cw.cpu().numpy(), canvas[y0:y0 + h])
            total += cv.cpu().numpy()
        assert np.array_equal(total, cov)


@pytest.mark.parametrize("exact", [False, True])
@pytest.mark.parametrize("name,G", [("c1", 2), ("c2_200", 3), ("c3", 4)])
def test_routed_link_ranges_cover_like_the_whole_batch(name, G, exact):
    import torch
    import paper_2007_00308_gb300 as ps
    b = _case(name)
    ctx = ps.Context()
    db = ps.DeviceBatch(b)
    whole, canvas, cov = _whole(ps, ctx, db, b, exact)
    Wd, Ht = b.canvas
    lbounds = shard.split_links(shard.link_rib_estimates(b), G)
    rbounds = shard.raster_rows(Ht, G)
    woff = whole.link_rib_off.cpu().numpy().astype(np.int64)
    # every range routes its quads; block d of range r goes to rank d
    blocks = [[None] * G for _ in range(G)]
    n_quads = 0
    for r in range(G):
        l0, l1 = int(lbounds[r]), int(lbounds[r + 1])
        cap = max(int(woff[l1] - woff[l0]), 1)
        out = ps.TessOutput(l1 - l0, db.n_path, cap, arclength=False)
        ps.ps_tessellate_links(ctx, db, out, l0, l1, ps.PS_PREC_MIXED, 0)
        qr, qt, cnt = shard.route(ps, ctx, out.rib, out.tag, out.n_rib, out.capacity, Wd, Ht,
                                  rbounds)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        cnt = cnt.cpu().numpy()
        n_quads += int(cnt.sum())
        o = np.concatenate([[0], np.cumsum(cnt)])
        for d in range(G):
            blocks[r][d] = (qr[o[d]:o[d + 1]], qt[o[d]:o[d + 1]])
    assert n_quads > 0
    got = np.zeros_like(canvas)
    total = np.zeros(b.n_path, np.int64)
    for d in range(G):
        y0, h = int(rbounds[d]), int(rbounds[d + 1] - rbounds[d])
        if h == 0:
            continue
        qr = torch.cat([blocks[r][d][0] for r in range(G)])
        qt = torch.cat([blocks[r][d][1] for r in range(G)])
        n = qr.shape[0]
        rib = qr.reshape(2 * n, 4).contiguous() if n else torch.zeros((2, 4), device="cuda")
        tag = qt.reshape(2 * n).contiguous() if n else torch.ones(2, dtype=torch.int32,
                                                                  device="cuda")
        n_rib = torch.tensor([2 * n], dtype=torch.int64, device="cuda")
        cw = torch.zeros((h, Wd), dtype=torch.int16, device="cuda")
        cv = torch.zeros(b.n_path, dtype=torch.int64, device="cuda")
        ps.ps_rasterize_coverage_rows(ctx, rib, tag, n_rib, rib.shape[0], b.n_path, Wd, y0, h, cw,
                                      cv, exact=exact)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        got[y0:y0 + h] = cw.cpu().numpy()
        total += cv.cpu().numpy()
    print(f"{name} G={G} exact={exact}: {n_quads} routed quads, "
          f"{int(np.count_nonzero(canvas))} covered pixels")
    assert np.array_equal(got, canvas)
    assert np.array_equal(total, cov)


def test_route_arguments_are_checked():
    import torch
    import paper_2007_00308_gb300 as ps
    b = W.c1_plain_small()
    ctx = ps.Context()
    out = ps.tessellate(ctx, ps.DeviceBatch(b), ps.PS_PREC_MIXED, arclength=False)
    Wd, Ht = b.canvas
    rb = torch.tensor([0, 256, Ht], dtype=torch.int32, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    off = torch.zeros(3, dtype=torch.int64, device="cuda")
    qr = torch.zeros((4, 8), device="cuda")
    with pytest.raises(ps.PolarStrokeError):  # outputs without room, or room without outputs
        ps.ps_route_quads(ctx, out.rib, out.tag, out.n_rib, out.capacity, Wd, Ht, rb, qr, None, 4,
                          cnt, off)
    cw = torch.zeros((16, Wd), dtype=torch.int16, device="cuda")
    cv = torch.zeros(b.n_path, dtype=torch.int64, device="cuda")
    for y0 in (-16, 8):  # negative or not a multiple of the tile size
        with pytest.raises(ps.PolarStrokeError):
            ps.ps_rasterize_coverage_rows(ctx, out.rib, out.tag, out.n_rib, out.capacity, b.n_path,
                                          Wd, y0, 16, cw, cv)


def test_route_edge_cases():
    """An empty window receives nothing; a quad reaching every window goes to all
    of them; quads outside the canvas go nowhere; the counting call and the
    writing call agree."""
    import torch
    import paper_2007_00308_gb300 as ps
    # one long vertical stroke through the whole canvas, one stroke outside it
    b = W.single([W.LINE, W.LINE], [[[100, 5], [100, 5], [100, 250], [100, 250]],
                                    [[100, 250], [100, 250], [400, 400], [400, 400]]],
                 width=6, join=W.JOIN_BEVEL, cap=W.CAP_BUTT, dtheta_deg=2.0, canvas=(256, 256))
    ctx = ps.Context()
    db = ps.DeviceBatch(b)
    out = ps.tessellate(ctx, db, ps.PS_PREC_MIXED, arclength=False)
    Wd, Ht = b.canvas
    bounds = np.array([0, 0, 64, 128, 128, Ht], np.int32)  # windows 0 and 3 are empty
    qr, qt, cnt = shard.route(ps, ctx, out.rib, out.tag, out.n_rib, out.capacity, Wd, Ht, bounds)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    cnt = cnt.cpu().numpy()
    assert cnt[0] == 0 and cnt[3] == 0
    assert cnt[1] > 0 and cnt[2] > 0 and cnt[4] > 0
    # every routed pair is one quad: link start on the first rib, not on the second
    t = qt.cpu().numpy().view(np.uint32)
    assert np.all(t[:, 0] & 1) and not np.any(t[:, 1] & 1)
    # the windows give the whole canvas
    canvas = torch.zeros((Ht, Wd), dtype=torch.int16, device="cuda")
    cov = torch.zeros(b.n_path, dtype=torch.int64, device="cuda")
    ps.ps_rasterize_coverage(ctx, out.rib, out.tag, out.n_rib, out.capacity, b.n_path, Wd, Ht,
                             canvas, cov)
    o = np.concatenate([[0], np.cumsum(cnt)])
    got = torch.zeros_like(canvas)
    total = torch.zeros_like(cov)
    for d in range(len(bounds) - 1):
        y0, h = int(bounds[d]), int(bounds[d + 1] - bounds[d])
        if h == 0:
            continue
        n = int(cnt[d])
        rib = qr[o[d]:o[d + 1]].reshape(2 * n, 4).contiguous()
        tag = qt[o[d]:o[d + 1]].reshape(2 * n).contiguous()
        n_rib = torch.tensor([2 * n], dtype=torch.int64, device="cuda")
        cw = torch.zeros((h, Wd), dtype=torch.int16, device="cuda")
        cv = torch.zeros_like(cov)
        ps.ps_rasterize_coverage_rows(ctx, rib, tag, n_rib, 2 * n, b.n_path, Wd, y0, h, cw, cv)
        got[y0:y0 + h] = cw
        total += cv
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert torch.equal(got, canvas) and torch.equal(total, cov)
