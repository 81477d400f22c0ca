"""Empty inputs through every call of the path: a batch with no paths at all,
and a rib stream of length zero through arc length, dashing (plain and capped),
and both coverage rules; each must agree with the oracle's result for the same
empty input (no ribs, zero offsets, an empty dash, a blank canvas)."""
import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_batch_without_paths():
    import torch
    import paper_2007_00308_gb300 as ps
    b = W.make_batch("empty", [], np.zeros((0, 4, 2)), [], [], 2.0, W.JOIN_ROUND, W.CAP_ROUND)
    o = oracle.tessellate(b)
    assert len(o["s"]) == 0
    ctx = ps.Context()
    db = ps.DeviceBatch(b)
    for prec in (ps.PS_PREC_FP32, ps.PS_PREC_MIXED):
        out = ps.tessellate(ctx, db, prec, arclength=True, want_t=True)
        torch.cuda.synchronize()
        assert ctx.status() == ps.PS_OK
        assert int(out.n_rib.item()) == 0
        assert out.link_rib_off.cpu().tolist() == o["link_rib_off"].tolist() == [0]
        assert out.path_rib_off.cpu().tolist() == o["path_rib_off"].tolist() == [0]
        out2 = ps.TessOutput(0, 0, 0, arclength=True)
        out2.n_rib.fill_(7)
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert ps.ps_tessellate_strokes_noalloc(db, out2, status, prec,
                                                ps.PS_TESS_ARCLENGTH) == ps.PS_OK
        torch.cuda.synchronize()
        assert int(out2.n_rib.item()) == 0 and int(status.item()) == 0
    # the adjoint and the uniform comparison of an empty batch are no-ops
    e = torch.empty(0, device="cuda")
    ps.ps_tessellate_backward(ctx, db, out, e, e, e, e)
    ps.ps_uniform_tessellate(ctx, db, out, e)
    # segments without paths are refused
    bad = W.make_batch("bad", [W.LINE], np.zeros((1, 4, 2)), [1.0], [], 2.0, W.JOIN_ROUND,
                       W.CAP_ROUND)
    with pytest.raises(ps.PolarStrokeError):
        ps.ps_tessellate_strokes(ctx, ps.DeviceBatch(bad), ps.TessOutput(2, 0, 1))


@pytest.mark.parametrize("exact", [False, True])
def test_rib_stream_of_length_zero(exact):
    import torch
    import paper_2007_00308_gb300 as ps
    ctx = ps.Context()
    rib = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    tag = torch.zeros(4, dtype=torch.int32, device="cuda")
    s = torch.zeros(4, dtype=torch.float32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    plen = torch.full((2,), 5.0, dtype=torch.float32, device="cuda")
    ps.ps_arclength_scan(ctx, rib, tag, n, 4, s, plen, 2)
    torch.cuda.synchronize()
    assert plen.cpu().tolist() == [0.0, 0.0]
    o_rib = torch.zeros((8, 4), dtype=torch.float32, device="cuda")
    o_s = torch.zeros(8, dtype=torch.float32, device="cuda")
    o_tag = torch.zeros(8, dtype=torch.int32, device="cuda")
    o_src = torch.zeros(8, dtype=torch.int32, device="cuda")
    n_out = torch.full((1,), 9, dtype=torch.int64, device="cuda")
    od = oracle.dash(np.zeros((0, 4)), np.zeros(0), np.zeros(0, np.uint32), [3.0, 1.0], 0.5)
    ps.ps_dash(ctx, rib, s, tag, n, 4, [3.0, 1.0], 0.5, o_rib, o_s, o_tag, o_src, n_out, 8)
    torch.cuda.synchronize()
    assert int(n_out.item()) == len(od["s"]) == 0
    n_out.fill_(9)
    pc = torch.full((2,), W.CAP_ROUND, dtype=torch.uint8, device="cuda")
    ps.ps_dash_capped(ctx, rib, s, tag, n, 4, [3.0, 1.0], 0.5, pc, 0.05, o_rib, o_s, o_tag,
                      o_src, n_out, 8)
    torch.cuda.synchronize()
    assert int(n_out.item()) == 0
    canvas = torch.full((40, 40), -1, dtype=torch.int16, device="cuda")
    covered = torch.full((2,), 3, dtype=torch.int64, device="cuda")
    ps.ps_rasterize_coverage(ctx, rib, tag, n, 4, 2, 40, 40, canvas, covered, exact=exact)
    torch.cuda.synchronize()
    ocan, ocov = oracle.raster(np.zeros((0, 4)), np.zeros(0, np.uint32), 40, 40, 2)
    assert np.array_equal(canvas.cpu().numpy().view(np.uint16), ocan)
    assert covered.cpu().tolist() == ocov.astype(np.int64).tolist() == [0, 0]
    assert ctx.status() == ps.PS_OK
