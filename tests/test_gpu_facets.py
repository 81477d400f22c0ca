"""Uniform parametric ribs and facet statistics on the GPU against the oracle
(Sec. 8.1): the uniform ribs of every segment equal the oracle's at the GPU's
own polar counts within the vertex bound, and the per-link facet statistics of
both tessellations equal the oracle's facet angles of the same FP32 ribs."""
import math

import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W
from tests._parity import gpu_tessellate, ulp32

pytestmark = pytest.mark.gpu

SLACK = 1e-5


def _runs(link_off, tag):
    seg = (tag >> 1) & 1
    for l in range(len(link_off) - 1):
        a, b = int(link_off[l]), int(link_off[l + 1])
        if b - a >= 2 and seg[a]:
            yield l, a, b


def test_uniform_ribs_and_facet_stats_match_the_oracle():
    import torch
    import paper_2007_00308_gb300 as ps
    b = W.facet_comparison(n_paths=300)
    g = gpu_tessellate(b, ps.PS_PREC_MIXED)
    assert g["status"] == 0
    ctx, out = g["ctx"], g["out"]
    db = ps.DeviceBatch(b)
    uni = torch.empty_like(out.rib)
    ps.ps_uniform_tessellate(ctx, db, out, uni)
    n_link = len(g["link_rib_off"]) - 1
    st_p = torch.empty((n_link, 4), dtype=torch.float32, device="cuda")
    st_u = torch.empty_like(st_p)
    ps.ps_facet_stats(ctx, out.rib, out.tag, out.link_rib_off, out.n_rib, out.capacity, st_p, SLACK)
    ps.ps_facet_stats(ctx, uni, out.tag, out.link_rib_off, out.n_rib, out.capacity, st_u, SLACK)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    R = g["R"]
    urib = uni[:R].cpu().numpy().astype(np.float64)
    sp, su = st_p.cpu().numpy().astype(np.float64), st_u.cpu().numpy().astype(np.float64)
    worst, mism, total = 0.0, 0, 0
    for l, a, e in _runs(g["link_rib_off"], g["tag"]):
        p = (l - 1) // 3  # one segment per path: links cap, seg, cap
        seg_pts = b.seg_pts[p].astype(np.float64)
        ref = oracle.uniform_ribs(W.CUBIC, seg_pts, 1.0, e - a - 1, float(b.path_width[p]))
        err = np.abs(urib[a:e] - ref)
        tol = 2e-4 + 4 * ulp32(np.abs(ref))
        worst = max(worst, float((err / tol).max()))
        for st, rib in ((sp, g["rib"][a:e]), (su, urib[a:e])):
            ang, ordn = oracle.facet_angles(rib, slack=SLACK)
            v = ang[ordn]
            total += 1
            if int(st[l, 3]) != len(v):
                mism += 1
                continue
            if len(v):
                assert st[l, 0] == pytest.approx(v.max(), abs=2e-5)
                assert st[l, 1] == pytest.approx(v.sum(), rel=1e-4, abs=1e-4)
    assert worst <= 1.0, worst
    assert mism <= max(2, 0.01 * total), (mism, total)


def test_polar_beats_uniform_at_equal_counts():
    """The paper's finding on the comparison batch (q = 4 deg): polar stroking's
    ordinary facets stay below 2q, and its largest facet and spread are smaller
    than uniform tessellation's with the same quads."""
    import torch
    import paper_2007_00308_gb300 as ps
    b = W.facet_comparison(n_paths=2000)
    g = gpu_tessellate(b, ps.PS_PREC_MIXED, want_t=False)
    ctx, out = g["ctx"], g["out"]
    db = ps.DeviceBatch(b)
    uni = torch.empty_like(out.rib)
    ps.ps_uniform_tessellate(ctx, db, out, uni)
    n_link = len(g["link_rib_off"]) - 1
    st_p = torch.empty((n_link, 4), dtype=torch.float32, device="cuda")
    st_u = torch.empty_like(st_p)
    ps.ps_facet_stats(ctx, out.rib, out.tag, out.link_rib_off, out.n_rib, out.capacity, st_p, SLACK)
    ps.ps_facet_stats(ctx, uni, out.tag, out.link_rib_off, out.n_rib, out.capacity, st_u, SLACK)
    torch.cuda.synchronize()
    sp, su = st_p.cpu().numpy().astype(np.float64), st_u.cpu().numpy().astype(np.float64)
    q = b.dtheta
    assert sp[:, 0].max() < 2 * q
    n_p, n_u = sp[:, 3].sum(), su[:, 3].sum()
    m_p, m_u = sp[:, 1].sum() / n_p, su[:, 1].sum() / n_u
    sd_p = math.sqrt(sp[:, 2].sum() / n_p - m_p ** 2)
    sd_u = math.sqrt(su[:, 2].sum() / n_u - m_u ** 2)
    print(f"polar max {math.degrees(sp[:, 0].max()):.2f} mean {math.degrees(m_p):.2f} "
          f"sd {math.degrees(sd_p):.2f} | uniform max {math.degrees(su[:, 0].max()):.2f} "
          f"mean {math.degrees(m_u):.2f} sd {math.degrees(sd_u):.2f}")
    assert sp[:, 0].max() < su[:, 0].max()
    assert sd_p < sd_u
