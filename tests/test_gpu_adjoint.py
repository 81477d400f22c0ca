"""Adjoint parity: gradients of L = sum(G_rib . rib) + sum(G_s . s) with respect
to control points and widths, from the library's adjoint kernel, against FP64
central differences (h = 1e-4) of the oracle at frozen step counts."""
import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fd_gradients(b, G_rib, G_s, h=1e-4):
    base_pts = b.seg_pts.astype(np.float64).copy()
    base_w = b.path_width.astype(np.float64).copy()
    o0 = oracle.tessellate(b, seg_pts64=base_pts, width64=base_w)
    counts = o0["link_nrib"]

    def L(pts, w):
        o = oracle.tessellate(b, seg_pts64=pts, width64=w)
        if not np.array_equal(o["link_nrib"], counts):
            return None
        return float((o["rib"] * G_rib).sum() + (o["s"] * G_s).sum())

    g_pts = np.full(base_pts.shape, np.nan)
    it = np.nditer(base_pts, flags=["multi_index"])
    for _ in it:
        idx = it.multi_index
        p1, p2 = base_pts.copy(), base_pts.copy()
        p1[idx] += h
        p2[idx] -= h
        a, c = L(p1, base_w), L(p2, base_w)
        if a is not None and c is not None:
            g_pts[idx] = (a - c) / (2 * h)
    g_w = np.full(base_w.shape, np.nan)
    for i in range(len(base_w)):
        w1, w2 = base_w.copy(), base_w.copy()
        w1[i] += h
        w2[i] -= h
        a, c = L(base_pts, w1), L(base_pts, w2)
        if a is not None and c is not None:
            g_w[i] = (a - c) / (2 * h)
    return g_pts, g_w, len(o0["s"])


@pytest.mark.parametrize("name", ["c5_pair", "mixed_forms"])
def test_adjoint_matches_fp64_central_differences(name):
    import torch
    import paper_2007_00308_gb300 as ps
    from paper_2007_00308_gb300.autograd import PolarStroke
    if name == "c5_pair":
        b = W.c5_differentiation(n_paths=2, n_seg=12)
    else:
        # no join here is tangent-continuous: a perturbation would make one appear
        pts = [[[10, 10], [40, 60], [80, -10], [120, 30]],
               [[120, 30], [150, 64], [150, 64], [170, 20]],
               [[170, 20], [190, 0], [190, 0], [220, 40]],
               [[220, 40], [220, 40], [260, 40], [260, 40]]]
        b = W.single([W.CUBIC, W.QUAD, W.CONIC, W.LINE], pts, w=[1, 1, 1.7, 1], width=6,
                     join=W.JOIN_ROUND, cap=W.CAP_SQUARE, dtheta_deg=2.0)
    dev = "cuda"
    pts_t = torch.tensor(b.seg_pts, dtype=torch.float32, device=dev, requires_grad=True)
    w_t = torch.tensor(b.path_width, dtype=torch.float32, device=dev, requires_grad=True)
    rib, s = PolarStroke.apply(pts_t, w_t, b, ps.PS_PREC_MIXED)
    R = rib.shape[0]
    rng = np.random.default_rng(7)
    G_rib = rng.standard_normal((R, 4))
    G_s = rng.standard_normal(R) * 0.1
    L = (rib * torch.tensor(G_rib, dtype=torch.float32, device=dev)).sum() + \
        (s * torch.tensor(G_s, dtype=torch.float32, device=dev)).sum()
    L.backward()
    g_gpu = pts_t.grad.cpu().numpy().astype(np.float64)
    gw_gpu = w_t.grad.cpu().numpy().astype(np.float64)
    g_fd, gw_fd, R_o = _fd_gradients(b, G_rib, G_s)
    assert R_o == R
    ok = ~np.isnan(g_fd)
    assert ok.mean() > 0.9
    # quadratic / conic middle point: gradient reported in the B slot, C unused
    for i, t in enumerate(b.seg_type):
        if t in (W.QUAD, W.CONIC):
            g_fd[i, 1] = np.nan_to_num(g_fd[i, 1]) + np.nan_to_num(g_fd[i, 2])
            g_fd[i, 2] = 0.0
    scale = np.abs(g_fd[ok]).max()
    err = np.abs(g_gpu - g_fd)[ok]
    rel = np.linalg.norm(err) / np.linalg.norm(g_fd[ok])
    print(name, "R", R, "grad rel l2 err", rel, "max abs err", err.max(), "scale", scale)
    assert rel < 2e-3
    assert err.max() < 2e-3 * scale + 1e-3 * np.abs(g_fd[ok]).max()
    okw = ~np.isnan(gw_fd)
    assert np.allclose(gw_gpu[okw], gw_fd[okw], rtol=2e-3, atol=1e-3 * np.abs(gw_fd[okw]).max())
