"""Adjoint parity: gradients of L = sum(G_rib . rib) + sum(G_s . s) with respect
to control points and widths, from the library's adjoint kernel, against FP64
central differences (h = 1e-4) of the oracle at frozen step counts: relative L2
error at most 1e-3, and per coordinate at most the larger of 1e-3 relative and
1e-4 of the largest gradient."""
import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# The bar (relative L2 over all compared coordinates, and per coordinate the
# larger of 1e-3 relative and this fraction of the path's largest gradient).
REL_L2 = 1e-3
ABS_FRAC = 1e-4


def _fd_multi(b, losses, h=1e-4):
    """FP64 central differences of the oracle at the unperturbed step counts for
    several losses L_k = sum(G_rib_k . rib) + sum(G_s_k . s) at once.  Returns
    ([(g_pts_k, g_w_k)], R, excluded): a coordinate whose perturbation changes a
    link's count (an interval boundary crossed) is NaN and counted in excluded."""
    base_pts = b.seg_pts.astype(np.float64).copy()
    base_w = b.path_width.astype(np.float64).copy()
    o0 = oracle.tessellate(b, seg_pts64=base_pts, width64=base_w)
    counts = o0["link_nrib"]

    def L(pts, w):
        o = oracle.tessellate(b, seg_pts64=pts, width64=w)
        if not np.array_equal(o["link_nrib"], counts):
            return None
        return [float((o["rib"] * Gr).sum() + (o["s"] * Gs).sum()) for Gr, Gs in losses]

    g_pts = [np.full(base_pts.shape, np.nan) for _ in losses]
    g_w = [np.full(base_w.shape, np.nan) for _ in losses]
    excluded = 0
    it = np.nditer(base_pts, flags=["multi_index"])
    for _ in it:
        idx = it.multi_index
        p1, p2 = base_pts.copy(), base_pts.copy()
        p1[idx] += h
        p2[idx] -= h
        a, c = L(p1, base_w), L(p2, base_w)
        if a is None or c is None:
            excluded += 1
            continue
        for k in range(len(losses)):
            g_pts[k][idx] = (a[k] - c[k]) / (2 * h)
    for i in range(len(base_w)):
        w1, w2 = base_w.copy(), base_w.copy()
        w1[i] += h
        w2[i] -= h
        a, c = L(base_pts, w1), L(base_pts, w2)
        if a is None or c is None:
            excluded += 1
            continue
        for k in range(len(losses)):
            g_w[k][i] = (a[k] - c[k]) / (2 * h)
    return list(zip(g_pts, g_w)), len(o0["s"]), excluded


def _fd_gradients(b, G_rib, G_s, h=1e-4):
    (res,), R, _ = _fd_multi(b, [(G_rib, G_s)], h)
    return res[0], res[1], R


def _fold_middle_points(b, g):
    """A quadratic's or conic's middle point gets its gradient in the B slot."""
    for i, t in enumerate(b.seg_type):
        if t in (W.QUAD, W.CONIC):
            g[i, 1] = np.nan_to_num(g[i, 1]) + np.nan_to_num(g[i, 2])
            g[i, 2] = 0.0


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
    _fold_middle_points(b, g_fd)
    scale = np.abs(g_fd[ok]).max()
    err = np.abs(g_gpu - g_fd)[ok]
    rel = np.linalg.norm(err) / np.linalg.norm(g_fd[ok])
    print(name, "R", R, "grad rel l2 err", rel, "max abs err", err.max(), "scale", scale)
    assert rel <= REL_L2
    assert np.all(err <= np.maximum(1e-3 * np.abs(g_fd[ok]), ABS_FRAC * scale))
    okw = ~np.isnan(gw_fd)
    assert np.allclose(gw_gpu[okw], gw_fd[okw], rtol=1e-3, atol=ABS_FRAC * np.abs(gw_fd[okw]).max())


def test_adjoint_c5_sampled_paths_at_full_size():
    """The c5 configuration at its full size (4,096 paths of 32 cubics): one
    forward and two backward passes on the GPU, with upstream gradients
    G_rib, G_s ~ N(0, 1) (all outputs) and G_s alone (the suffix sums of dL/ds on
    their own).  64 sampled paths are checked against FP64 central differences
    of the oracle on each path alone (paths are independent); coordinates whose
    perturbation crosses an interval boundary are excluded and counted."""
    import torch
    import paper_2007_00308_gb300 as ps
    from paper_2007_00308_gb300.autograd import PolarStroke
    b = W.c5_differentiation()
    dev = "cuda"
    pts_t = torch.tensor(b.seg_pts, dtype=torch.float32, device=dev, requires_grad=True)
    w_t = torch.tensor(b.path_width, dtype=torch.float32, device=dev, requires_grad=True)
    rib, s = PolarStroke.apply(pts_t, w_t, b, ps.PS_PREC_MIXED)
    R = rib.shape[0]
    rng = np.random.default_rng(11)
    G_rib = rng.standard_normal((R, 4))
    G_s = rng.standard_normal(R)
    G_s2 = rng.standard_normal(R)
    Gr_t = torch.tensor(G_rib, dtype=torch.float32, device=dev)
    L1 = (rib * Gr_t).sum() + (s * torch.tensor(G_s, dtype=torch.float32, device=dev)).sum()
    g1 = torch.autograd.grad(L1, [pts_t, w_t], retain_graph=True)
    L2 = (s * torch.tensor(G_s2, dtype=torch.float32, device=dev)).sum()
    g2 = torch.autograd.grad(L2, [pts_t, w_t])
    gpu = [(g[0].cpu().numpy().astype(np.float64), g[1].cpu().numpy().astype(np.float64))
           for g in (g1, g2)]
    # each path's rib range from the forward's own offsets
    ctx = ps.Context()
    out = ps.tessellate(ctx, ps.DeviceBatch(b), ps.PS_PREC_MIXED, arclength=True)
    torch.cuda.synchronize()
    poff = out.path_rib_off.cpu().numpy().astype(np.int64)
    assert int(poff[-1]) == R
    paths = np.sort(np.random.default_rng(12).choice(b.n_path, 64, replace=False))
    errs = [[], []]
    refs = [[], []]
    excluded = total = 0
    for p in paths:
        b1 = b.subset([p])
        a, e = int(poff[p]), int(poff[p + 1])
        losses = [(G_rib[a:e], G_s[a:e]), (np.zeros((e - a, 4)), G_s2[a:e])]
        fd, R1, ex = _fd_multi(b1, losses)
        assert R1 == e - a
        excluded += ex
        total += b1.seg_pts.size + 1
        segs = slice(int(b.path_seg_off[p]), int(b.path_seg_off[p + 1]))
        for k in range(2):
            g_fd, gw_fd = fd[k]
            ok = ~np.isnan(g_fd)
            g_gpu = gpu[k][0][segs]
            scale = np.abs(g_fd[ok]).max()
            err = np.abs(g_gpu - g_fd)[ok]
            assert np.all(err <= np.maximum(1e-3 * np.abs(g_fd[ok]), ABS_FRAC * scale)), \
                (k, p, float(err.max()), float(scale))
            errs[k].append(err)
            refs[k].append(g_fd[ok])
            if not np.isnan(gw_fd[0]):
                assert abs(gpu[k][1][p] - gw_fd[0]) <= max(1e-3 * abs(gw_fd[0]), ABS_FRAC * scale)
    for k, what in enumerate(("G_rib and G_s", "G_s alone")):
        e, r = np.concatenate(errs[k]), np.concatenate(refs[k])
        rel = np.linalg.norm(e) / np.linalg.norm(r)
        print(f"c5 full size, 64 sampled paths, upstream {what}: rel L2 {rel:.2e}, "
              f"max abs err {e.max():.3e} (max |grad| {np.abs(r).max():.3e}); "
              f"{excluded} of {total} coordinates excluded (interval boundary crossed)")
        assert rel <= REL_L2
    assert excluded <= 0.05 * total
