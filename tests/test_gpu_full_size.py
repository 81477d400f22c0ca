"""Parity at the benchmark's full sizes on sampled outputs.  The GPU runs the whole
configuration at once (the bench's sizes and launch parameters); the oracle, which
could not finish the whole of it in seconds, checks randomly sampled paths one by
one.  Paths are independent in tessellation, arc length (s restarts per path) and
per-path coverage (a path's covered samples are the union of its own quads), so a
sampled path's oracle result must match the GPU's at full size exactly as on a
small batch.  The canvas is checked through a property that holds at any size:
every sample a sampled path covers is set on the canvas."""
import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W
from tests._parity import compare_tess

pytestmark = pytest.mark.gpu

FRAG64 = oracle.FRAGILE64


def gpu_run(batch, emit_slabs=None, raster=False):
    import torch
    import paper_2007_00308_gb300 as ps
    ctx = ps.Context()
    if emit_slabs:
        ctx.set_tuning(ps.PS_TUNE_EMIT_SLABS, emit_slabs)
    db = ps.DeviceBatch(batch)
    out = ps.tessellate(ctx, db, ps.PS_PREC_MIXED, arclength=True, want_t=False)
    res = {}
    if raster:
        Wd, Ht = batch.canvas
        canvas = torch.zeros((Ht, Wd), dtype=torch.int16, device="cuda")
        covered = torch.zeros(batch.n_path, dtype=torch.int64, device="cuda")
        ps.ps_rasterize_coverage(ctx, out.rib, out.tag, out.n_rib, out.capacity, batch.n_path,
                                 Wd, Ht, canvas, covered)
        torch.cuda.synchronize()
        assert ctx.status() in (0, ps.PS_ERR_CAPACITY)
        if ctx.status() == ps.PS_ERR_CAPACITY:  # bins sized from the first pass's count
            ctx.reserve(n_tile=((Wd + 15) // 16) * ((Ht + 15) // 16),
                        n_pair=int(ps.ps_raster_stats(ctx)["pairs"] * 1.05) + 1024)
            ps.ps_rasterize_coverage(ctx, out.rib, out.tag, out.n_rib, out.capacity,
                                     batch.n_path, Wd, Ht, canvas, covered)
        res["canvas"] = canvas.cpu().numpy().view(np.uint16)
        res["covered"] = covered.cpu().numpy().view(np.uint64)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    R = int(out.n_rib.item())
    res.update(R=R, link_rib_off=out.link_rib_off.cpu().numpy().astype(np.int64),
               path_rib_off=out.path_rib_off.cpu().numpy().astype(np.int64),
               path_len=out.path_len.cpu().numpy().astype(np.float64), out=out)
    return res


def gather(batch, g, paths):
    """The GPU's output for the sampled paths, laid out as the oracle lays out the
    subset batch (path indices in the tags renumbered)."""
    out = g["out"]
    off = batch.path_seg_off.astype(np.int64)
    lo = g["link_rib_off"]
    link_n, ribs, tags, ss = [], [], [], []
    for i, p in enumerate(paths):
        l0, l1 = 2 * off[p] + p, 2 * off[p + 1] + p + 1
        link_n.append(np.diff(lo[l0:l1 + 1]))
        a, b = int(g["path_rib_off"][p]), int(g["path_rib_off"][p + 1])
        ribs.append(out.rib[a:b].cpu().numpy().astype(np.float64))
        t = out.tag[a:b].cpu().numpy().view(np.uint32)
        tags.append((t & np.uint32(3)) | np.uint32(i << 2))
        ss.append(out.s[a:b].cpu().numpy().astype(np.float64))
    link_off = np.zeros(sum(len(x) for x in link_n) + 1, np.int64)
    link_off[1:] = np.cumsum(np.concatenate(link_n))
    return dict(link_rib_off=link_off, rib=np.concatenate(ribs), tag=np.concatenate(tags),
                s=np.concatenate(ss), path_len=g["path_len"][paths])


def check_sampled(batch, g, n_sample, seed):
    rng = np.random.default_rng(seed)
    paths = np.sort(rng.choice(batch.n_path, n_sample, replace=False))
    sb = batch.subset(paths)
    o = oracle.tessellate(sb)
    gs = gather(batch, g, paths)
    stats, fails = compare_tess(o, gs, sb, FRAG64)
    print(batch.name, "full size, sampled", n_sample, stats)
    assert not fails, fails
    assert stats["count_mismatch_fragile"] <= max(2, 2e-3 * stats["links"])
    return paths, sb, gs


def test_c2_full_size_sampled_paths_and_coverage():
    """The bench configuration (10,000 paths, 2048^2) at the bench's tuned rib-task
    size; 150 sampled paths against the oracle, and their per-path covered samples
    bit-exact against the oracle's raster of the GPU's own vertices."""
    b = W.c2_batching()
    g = gpu_run(b, emit_slabs=32, raster=True)
    paths, sb, gs = check_sampled(b, g, 150, 1)
    Wd, Ht = b.canvas
    union = np.zeros((Ht, Wd), np.uint16)
    for i, p in enumerate(paths):
        sel = (gs["tag"] >> 2) == i
        rib, tag = gs["rib"][sel], gs["tag"][sel] & np.uint32(3)
        can, cov = oracle.raster(rib, tag, Wd, Ht, 1)
        assert int(cov[0]) == int(g["covered"][p]), (p, int(cov[0]), int(g["covered"][p]))
        union |= can
    # every sample a sampled path covers is set on the full canvas
    assert not (union & ~g["canvas"]).any()
    assert int(g["covered"].sum()) >= int(np.unpackbits(g["canvas"].view(np.uint8)).sum())


def test_c4_full_size_sampled_paths():
    """10^6 near-cusp / near-collinear cubics at coordinates up to 1e6 px."""
    b = W.c4_precision()
    g = gpu_run(b, emit_slabs=32)
    check_sampled(b, g, 400, 2)


def test_c5_full_size_sampled_paths():
    b = W.c5_differentiation()
    g = gpu_run(b, emit_slabs=32)
    check_sampled(b, g, 40, 3)
