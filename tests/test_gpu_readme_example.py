"""The usage example of the README, run as written, against the oracle: the
same rib count, and the same coverage (the GPU's vertices rasterized by the
oracle)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_readme_example():
    import torch
    import oracle
    import paper_2007_00308_gb300 as ps
    from paper_2007_00308_gb300 import workloads as W

    batch = W.single([W.CUBIC], [[[10, 10], [60, 120], [140, -40], [200, 60]]],
                     width=12, join=W.JOIN_ROUND, cap=W.CAP_ROUND, dtheta_deg=2.0,
                     canvas=(256, 256))
    ctx = ps.Context()
    db = ps.DeviceBatch(batch)
    out = ps.tessellate(ctx, db, ps.PS_PREC_MIXED)
    canvas = torch.zeros((256, 256), dtype=torch.int16, device="cuda")
    covered = torch.zeros(batch.n_path, dtype=torch.int64, device="cuda")
    ps.ps_rasterize_coverage(ctx, out.rib, out.tag, out.n_rib, out.capacity, batch.n_path,
                             256, 256, canvas, covered)
    assert ctx.status() == 0
    o = oracle.tessellate(batch)
    R = int(out.n_rib.item())
    assert R == len(o["s"])
    rib = out.rib[:R].cpu().numpy().astype(np.float64)
    tag = out.tag[:R].cpu().numpy().view(np.uint32)
    ocan, ocov = oracle.raster(rib, tag, 256, 256, 1)
    assert np.array_equal(canvas.cpu().numpy().view(np.uint16), ocan)
    assert int(covered.item()) == int(ocov[0])
