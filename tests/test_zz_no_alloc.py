"""The allocation-free tessellation entry point.

ps_tessellate_strokes_noalloc serves callers that cannot allocate device memory
when they stroke (for example where another allocator owns the device's memory
budget, or where an allocation must not block or fail partway through): it
takes its workspace from a fixed array inside the library instead of a context.  This test calls it
through the C ABI twice in a row and checks each result against the regular
entry point's, with the tolerances the other parity tests use; it also checks
that a problem larger than the fixed workspace is refused before any launch.
It lives in its own file, collected last, so that a stop at the first failure
has already run every other test."""
import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W
from tests._parity import compare_tess

pytestmark = pytest.mark.gpu


def _regular(ps, ctx, db, prec):
    out = ps.tessellate(ctx, db, prec, arclength=True, want_t=True)
    return out


def _as_dict(out, status=0):
    R = int(out.n_rib.item())
    return dict(R=R, rib=out.rib[:R].cpu().numpy().astype(np.float64),
                tag=out.tag[:R].cpu().numpy().view(np.uint32),
                s=out.s[:R].cpu().numpy().astype(np.float64),
                t=out.t[:R].cpu().numpy().astype(np.float64),
                link_rib_off=out.link_rib_off.cpu().numpy().astype(np.int64),
                path_rib_off=out.path_rib_off.cpu().numpy().astype(np.int64),
                path_len=out.path_len.cpu().numpy().astype(np.float64), status=status)


@pytest.mark.parametrize("name", ["c1", "c2_small"])
@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_regular_entry_point_twice(name, prec):
    import torch
    import paper_2007_00308_gb300 as ps
    b = W.c1_plain_small() if name == "c1" else W.c2_batching(n_paths=150)
    ctx = ps.Context()
    db = ps.DeviceBatch(b)
    ref_out = _regular(ps, ctx, db, prec)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    ref = _as_dict(ref_out)
    o = oracle.tessellate(b)
    for call in range(2):
        out = ps.TessOutput(db.n_link, db.n_path, ref["R"], arclength=True, want_t=True)
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        rc = ps.ps_tessellate_strokes_noalloc(db, out, status, prec, ps.PS_TESS_ARCLENGTH)
        assert rc == 0, ps.error_string(rc)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        g = _as_dict(out)
        # same counts, offsets and tags as the regular entry point
        assert g["R"] == ref["R"]
        assert np.array_equal(g["link_rib_off"], ref["link_rib_off"])
        assert np.array_equal(g["path_rib_off"], ref["path_rib_off"])
        assert np.array_equal(g["tag"], ref["tag"])
        # floating outputs within the parity tolerances, judged against the oracle
        frag = oracle.FRAGILE32 if prec == 0 else oracle.FRAGILE64
        eps = None if prec == 1 else 4e-6  # the contract bar in mixed precision
        st_ref, f_ref = compare_tess(o, ref, b, frag, eps)
        st_new, f_new = compare_tess(o, g, b, frag, eps)
        assert f_new == f_ref == []
        assert np.abs(g["rib"] - ref["rib"]).max() <= 1e-4
        assert np.abs(g["s"] - ref["s"]).max() <= 1e-5 * max(1.0, float(np.abs(ref["s"]).max()))


def test_noalloc_refuses_problems_beyond_its_workspace():
    import paper_2007_00308_gb300 as ps
    b = W.c5_differentiation(n_paths=400)  # 2*12800 + 400 links > 16384
    db = ps.DeviceBatch(b)
    out = ps.TessOutput(db.n_link, db.n_path, 16, arclength=True)
    import torch
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = ps.ps_tessellate_strokes_noalloc(db, out, status, 0, ps.PS_TESS_ARCLENGTH)
    assert rc == ps.PS_ERR_CAPACITY
