"""Splitting a batch over ranks by links (paper_2007_00308_gb300/shard.py), on the
CPU: two gloo ranks each take a link range, reproduce what the library's range
call returns for it (from the FP64 oracle's run of the whole batch: ribs, tags
and counts of the range, offsets and s local to it), exchange (rib count, tail
length), and apply the plan; the joined result must equal the single-rank run:
counts, offsets and tags identical, s and path lengths within 1e-5 relative."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2007_00308_gb300 import shard
from paper_2007_00308_gb300 import workloads as W

LINK_START = 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def local_range(o, batch, l0, l1):
    """The range call's outputs for links [l0, l1), from a whole-batch run o."""
    off = o["link_rib_off"]
    a, b = int(off[l0]), int(off[l1])
    tag = o["tag"][a:b]
    s = o["s"][a:b].copy()
    p0 = int(shard.path_of_link(batch, l0))
    if shard.first_link(batch, p0) != l0 and b > a:
        lead = np.cumprod((tag >> 2) == p0).astype(bool)
        s[lead] -= o["s"][a]  # a link's first rib keeps the previous rib's s (chord 0)
    path_len = {}
    for i in range(b - a):
        p = int(tag[i] >> 2)
        if shard.last_link(batch, p) < l1 and (i + 1 == b - a or int(tag[i + 1] >> 2) != p):
            path_len[p] = s[i]
    last_p = int(shard.path_of_link(batch, l1 - 1))
    tail = float(s[-1]) if b > a and int(tag[-1] >> 2) == last_p else 0.0
    return dict(n_rib=b - a, tag=tag, s=s, link_off=off[l0:l1 + 1] - a, path_len=path_len,
                tail=tail)


def apply_plan(loc, plan, r):
    s = loc["s"].copy()
    p = int(plan["carry_path"][r])
    path_len = dict(loc["path_len"])
    if p >= 0:
        lead = np.cumprod((loc["tag"] >> 2) == p).astype(bool)
        s[lead] += plan["carry"][r]
        if plan["with_len"][r]:
            path_len[p] += plan["carry"][r]
    return s, path_len


def _case(name):
    if name == "c3":
        return W.c3_large_path(n_seg=300)
    return W.c2_batching(n_paths=60, seed=W.SEED_BASE + 2)


def _worker(rank, world, port, name, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _case(name)
    o = oracle.tessellate(b)
    bounds = shard.split_links(shard.link_rib_estimates(b), world)
    loc = local_range(o, b, int(bounds[rank]), int(bounds[rank + 1]))
    n_rib, tail = shard.exchange(loc["n_rib"], loc["tail"])
    plan = shard.join_plan(b, bounds, n_rib, tail)
    s, path_len = apply_plan(loc, plan, rank)
    q.put((rank, int(plan["rib_offset"][rank]), loc["link_off"] + plan["rib_offset"][rank],
           loc["tag"], s, path_len, [int(x) for x in bounds]))
    dist.barrier()
    dist.destroy_process_group()


def _join(parts):
    parts = sorted(parts, key=lambda x: x[0])
    link_off = np.concatenate([parts[0][2]] + [p[2][1:] for p in parts[1:]])
    tag = np.concatenate([p[3] for p in parts])
    s = np.concatenate([p[4] for p in parts])
    path_len = {}
    for p in parts:
        path_len.update(p[5])
    return link_off, tag, s, path_len


@pytest.mark.parametrize("name", ["c3", "c2_60"])
def test_two_ranks_join_to_the_single_rank_result(name):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, name, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    b = _case(name)
    o = oracle.tessellate(b)
    bounds = parts[0][6]
    assert 0 < bounds[1] < bounds[2]  # a real split
    if name == "c3":
        assert shard.path_of_link(b, bounds[1]) == 0  # the single path runs across the cut
    link_off, tag, s, path_len = _join(parts)
    assert np.array_equal(link_off, o["link_rib_off"])
    assert np.array_equal(tag, o["tag"])
    assert np.all(np.abs(s - o["s"]) <= 1e-5 * np.maximum(o["s"], 1.0))
    assert sorted(path_len) == list(range(b.n_path))
    for p, v in path_len.items():
        assert abs(v - o["path_len"][p]) <= 1e-5 * max(o["path_len"][p], 1.0)


@pytest.mark.parametrize("G", [3, 5])
def test_plan_joins_many_ranges_of_one_path(G):
    """Without a process group: G ranges over one long path (ranks entirely
    inside it pass the carry on) and over a batch cut at random link bounds,
    including empty ranges."""
    for b, bounds in ((_case("c3"), None), (_case("c2_60"), "random")):
        o = oracle.tessellate(b)
        L = b.n_link
        if bounds is None:
            bounds = shard.split_links(shard.link_rib_estimates(b), G)
        else:
            rng = np.random.default_rng(G)
            cuts = np.sort(rng.integers(0, L + 1, G - 1))
            bounds = np.concatenate([[0], cuts, [L]])
        locs = [local_range(o, b, int(bounds[r]), int(bounds[r + 1])) if bounds[r + 1] > bounds[r]
                else dict(n_rib=0, tag=np.zeros(0, np.uint32), s=np.zeros(0),
                          link_off=np.zeros(1, np.int64), path_len={}, tail=0.0)
                for r in range(G)]
        plan = shard.join_plan(b, bounds, [x["n_rib"] for x in locs], [x["tail"] for x in locs])
        s = np.concatenate([apply_plan(x, plan, r)[0] for r, x in enumerate(locs)])
        assert np.array_equal(plan["rib_offset"], np.concatenate([[0], np.cumsum([x["n_rib"] for x in locs])[:-1]]))
        assert np.all(np.abs(s - o["s"]) <= 1e-5 * np.maximum(o["s"], 1.0))


def test_estimates_balance_the_ranks():
    b = W.c2_batching(n_paths=300, seed=W.SEED_BASE + 2)
    est = shard.link_rib_estimates(b)
    n = oracle.tessellate(b)["link_nrib"]
    assert np.corrcoef(est, n)[0, 1] > 0.9
    bounds = shard.split_links(est, 4)
    per_rank = [int(n[bounds[r]:bounds[r + 1]].sum()) for r in range(4)]
    assert max(per_rank) <= 1.2 * (sum(per_rank) / 4)


# ---------------------------------------------------------------------------
# The raster split by canvas rows, on the CPU: each gloo rank routes the quads
# of its link range to the owners of the rows they reach (the routing rule of
# ps_route_quads, restated here on the oracle's snapped coordinates), one
# all-to-all moves them (shard.exchange_quads), each owner covers its rows with
# the oracle's raster, and the per-path counts and the canvas rows are merged
# (shard.merge_covered, shard.gather_rows).  The result must equal the oracle's
# raster of the whole batch bit for bit.

def _rows_reached(rib, W, H):
    """Pixel rows [py0, py1] whose sample rows a quad's snapped bounding box
    reaches (py0 > py1: none), for quads given as rib pairs [n, 8]."""
    v = np.rint(np.asarray(rib, np.float64) * 256.0).astype(np.int64)
    xs, ys = v[:, 0::2], v[:, 1::2]
    mnx, mxx, mny, mxy = xs.min(1), xs.max(1), ys.min(1), ys.max(1)
    px0 = np.maximum(-((248 - mnx) // 256), 0)
    px1 = np.minimum((mxx - 8) // 256, W - 1)
    py0 = np.maximum(-((248 - mny) // 256), 0)
    py1 = np.minimum((mxy - 8) // 256, H - 1)
    empty = (px0 > px1) | (py0 > py1)
    return np.where(empty, 1, py0), np.where(empty, 0, py1)


def host_route(rib, tag, W, H, bounds):
    """Quads (r-1, r) of a rib stream grouped by destination: ([n, 8] ribs,
    [n, 2] tags with the link-start bit on the first) and the counts."""
    r = np.nonzero((tag[1:] & LINK_START) == 0)[0] + 1
    q_rib = np.concatenate([rib[r - 1], rib[r]], axis=1)
    q_tag = np.stack([tag[r] | LINK_START, tag[r]], axis=1).astype(np.int64)
    py0, py1 = _rows_reached(q_rib, W, H)
    G = len(bounds) - 1
    out_r, out_t, cnt = [], [], []
    for d in range(G):
        a, b = int(bounds[d]), int(bounds[d + 1])
        sel = (py0 <= py1) & (py0 < b) & (py1 >= a) & (b > a)
        out_r.append(q_rib[sel])
        out_t.append(q_tag[sel])
        cnt.append(int(sel.sum()))
    return np.concatenate(out_r), np.concatenate(out_t), np.array(cnt, np.int64)


def oracle_rows(rib, tag, W, H, n_path, y0, h):
    """The oracle's coverage of picture rows [y0, y0 + h): canvas rows and the
    per-path samples inside them (each path rasterized alone: its union)."""
    canvas = np.zeros((h, W), np.uint16)
    cov = np.zeros(n_path, np.int64)
    paths = tag[1::2] >> 2
    for p in np.unique(paths):
        sel = np.repeat(paths == p, 2)
        c, _ = oracle.raster(rib[sel], tag[sel] & 3, W, H, 1)
        rows = c[y0:y0 + h]
        canvas |= rows
        cov[p] = int(np.unpackbits(rows.view(np.uint8)).sum())
    return canvas, cov


def _raster_case():
    return W.c2_batching(n_paths=40, seed=W.SEED_BASE + 2, canvas=512)


def _raster_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _raster_case()
    Wd, Ht = b.canvas
    o = oracle.tessellate(b)
    lb = shard.split_links(shard.link_rib_estimates(b), world)
    off = o["link_rib_off"]
    a, e = int(off[lb[rank]]), int(off[lb[rank + 1]])
    rb = shard.raster_rows(Ht, world)
    q_rib, q_tag, cnt = host_route(o["rib"][a:e], o["tag"][a:e], Wd, Ht, rb)
    r_rib, r_tag = shard.exchange_quads(torch.from_numpy(q_rib), torch.from_numpy(q_tag),
                                        torch.from_numpy(cnt))
    y0, h = int(rb[rank]), int(rb[rank + 1] - rb[rank])
    rows, cov = oracle_rows(r_rib.numpy(), r_tag.numpy().astype(np.uint32), Wd, Ht, b.n_path, y0, h)
    cov_t = shard.merge_covered(torch.from_numpy(cov))
    canvas = shard.gather_rows(torch.from_numpy(rows.astype(np.int32)), rb)
    q.put((rank, canvas.numpy().astype(np.uint16), cov_t.numpy(), int(cnt.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_the_raster_by_rows():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_raster_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    b = _raster_case()
    o = oracle.tessellate(b)
    canvas, cov = oracle.raster(o["rib"], o["tag"], b.canvas[0], b.canvas[1], b.n_path)
    for rank, c, cv, n in sorted(parts, key=lambda x: x[0]):
        assert n > 0
        assert np.array_equal(c, canvas)       # every rank holds the whole canvas
        assert np.array_equal(cv, cov.astype(np.int64))
