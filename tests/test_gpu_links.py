"""Link-range tessellation on the GPU (ps_tessellate_links, ps_add_s_carry): a
batch cut into ranges by the partitioner of paper_2007_00308_gb300/shard.py and
tessellated range by range (as ranks would, here one after another on one GPU)
joins to the whole-batch call: counts, offsets, ribs and tags bit-identical, s
and path lengths within 1e-5 relative after the carries of the plan."""
import numpy as np
import pytest

from paper_2007_00308_gb300 import shard
from paper_2007_00308_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run_whole(ps, ctx, db, prec):
    import torch
    out = ps.tessellate(ctx, db, prec, arclength=True)
    torch.cuda.synchronize()
    R = int(out.n_rib.item())
    return dict(R=R, link_off=out.link_rib_off.cpu().numpy().astype(np.int64),
                rib=out.rib[:R].cpu().numpy(), tag=out.tag[:R].cpu().numpy().view(np.uint32),
                s=out.s[:R].cpu().numpy().astype(np.float64),
                path_len=out.path_len.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("name,G", [("c3", 3), ("c2_200", 4), ("c1", 2)])
@pytest.mark.parametrize("prec", [0, 1])
def test_ranges_join_to_the_whole_batch(name, G, prec):
    import torch
    import paper_2007_00308_gb300 as ps
    b = {"c3": lambda: W.c3_large_path(n_seg=800),
         "c2_200": lambda: W.c2_batching(n_paths=200, seed=W.SEED_BASE + 2),
         "c1": W.c1_plain_small}[name]()
    ctx = ps.Context()
    db = ps.DeviceBatch(b)
    whole = _run_whole(ps, ctx, db, prec)
    bounds = shard.split_links(shard.link_rib_estimates(b), G)
    assert all(bounds[r] < bounds[r + 1] for r in range(G))
    parts = []
    for r in range(G):
        l0, l1 = int(bounds[r]), int(bounds[r + 1])
        cap = int(whole["link_off"][l1] - whole["link_off"][l0])
        out = ps.TessOutput(l1 - l0, db.n_path, max(cap, 1), arclength=True)
        out.path_len.zero_()
        ps.ps_tessellate_links(ctx, db, out, l0, l1, prec, ps.PS_TESS_ARCLENGTH)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        R = int(out.n_rib.item())
        assert R == cap
        tag = out.tag[:R].cpu().numpy().view(np.uint32)
        s = out.s[:R].cpu().numpy()
        last_p = int(shard.path_of_link(b, l1 - 1))
        tail = float(s[-1]) if R and int(tag[-1] >> 2) == last_p else 0.0
        parts.append((out, R, tail))
    plan = shard.join_plan(b, bounds, [p[1] for p in parts], [p[2] for p in parts])
    for r, (out, R, _) in enumerate(parts):
        if plan["carry_path"][r] >= 0:
            ps.ps_add_s_carry(ctx, out, int(plan["carry_path"][r]), float(plan["carry"][r]),
                              bool(plan["with_len"][r]))
    torch.cuda.synchronize()
    assert ctx.status() == 0
    link_off = [parts[0][0].link_rib_off.cpu().numpy().astype(np.int64)]
    for r in range(1, G):
        link_off.append(parts[r][0].link_rib_off.cpu().numpy().astype(np.int64)[1:] +
                        plan["rib_offset"][r])
    assert np.array_equal(np.concatenate(link_off), whole["link_off"])
    rib = np.concatenate([p[0].rib[:p[1]].cpu().numpy() for p in parts])
    tag = np.concatenate([p[0].tag[:p[1]].cpu().numpy().view(np.uint32) for p in parts])
    s = np.concatenate([p[0].s[:p[1]].cpu().numpy().astype(np.float64) for p in parts])
    assert np.array_equal(rib, whole["rib"]) and np.array_equal(tag, whole["tag"])
    assert np.all(np.abs(s - whole["s"]) <= 1e-5 * np.maximum(whole["s"], 1.0))
    # each path's length from the range where it ends
    for r, (out, R, _) in enumerate(parts):
        pl = out.path_len.cpu().numpy().astype(np.float64)
        l0, l1 = int(bounds[r]), int(bounds[r + 1])
        for p in range(int(shard.path_of_link(b, l0)), int(shard.path_of_link(b, l1 - 1)) + 1):
            if shard.last_link(b, p) < l1:
                assert abs(pl[p] - whole["path_len"][p]) <= 1e-5 * max(whole["path_len"][p], 1.0)


def test_range_arguments_are_checked():
    import paper_2007_00308_gb300 as ps
    b = W.c1_plain_small()
    ctx = ps.Context()
    db = ps.DeviceBatch(b)
    out = ps.TessOutput(db.n_link, db.n_path, 16, arclength=True)
    for l0, l1 in ((-1, 3), (5, 5), (0, db.n_link + 1)):
        with pytest.raises(ps.PolarStrokeError):
            ps.ps_tessellate_links(ctx, db, out, l0, l1, 1, ps.PS_TESS_ARCLENGTH)
