"""Splitting one batch over several GPUs by links, one process per GPU.

Links are independent (Sec. 4.4): rank r tessellates the links [l0_r, l1_r) of
the batch with ``ps_tessellate_links``, its offsets and arc length local to the
range.  Rib offsets (Eq. 13) and arc length (Eq. 18) are prefix sums, so the
ranks' results join after one exchange of G x (rib count int64, tail length
float64): each rank's global rib offset is the sum of the counts before it, and
the path that runs into its range from earlier ranks takes as its s carry the
lengths that path has on those ranks.  The cut points fall on link boundaries,
where a rib's chord is zero (a link's first rib continues the previous one's s).

The ranges balance an estimate of each link's ribs taken from the control
polygons on the host (no pass over the GPU): a segment's turning is at most its
control polygon's (the curve turns through no more than the polygon of a
positive-weight Bezier), so it takes about turning / q + 2 ribs; a round join
|delta| / q + 1, a round cap pi / q + 1, the other joins and caps their fixed
counts.  Only the balance depends on the estimate, never the result.
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as W

# fixed rib counts (J + 1) of the join and cap styles other than round
_JOIN_RIBS = {0: 0, 1: 2, 2: 4, 3: 4, 5: 3}   # none, bevel, miter, miter-truncate, triangle
_CAP_RIBS = {0: 0, 1: 5, 3: 3}                 # butt, square, triangle


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def _legs(batch):
    """Control polygon legs of every segment: [S, 3, 2] (quadratics, conics and
    lines use the legs A->B, B->D resp. A->D, the rest zero)."""
    P = batch.seg_pts.astype(np.float64)
    t = batch.seg_type
    legs = np.zeros((len(t), 3, 2))
    cub = t == W.CUBIC
    qk = (t == W.QUAD) | (t == W.CONIC)
    ln = t == W.LINE
    legs[cub] = P[cub, 1:] - P[cub, :-1]
    legs[qk, 0] = P[qk, 1] - P[qk, 0]
    legs[qk, 1] = P[qk, 3] - P[qk, 1]
    legs[ln, 0] = P[ln, 3] - P[ln, 0]
    return legs


def link_rib_estimates(batch) -> np.ndarray:
    """Estimated ribs of every link of the batch (int64, link order)."""
    q = float(batch.dtheta)
    legs = _legs(batch)
    nz = np.abs(legs).sum(axis=2) > 0
    ang = np.arctan2(legs[..., 1], legs[..., 0])
    S = len(batch.seg_type)
    turn = np.zeros(S)
    first_dir = np.full(S, np.nan)
    prev = np.full(S, np.nan)
    for i in range(3):
        a = np.where(nz[:, i], ang[:, i], np.nan)
        step = np.abs(_wrap(a - prev))
        turn += np.where(np.isnan(step), 0.0, step)
        first_dir = np.where(np.isnan(first_dir), a, first_dir)
        prev = np.where(nz[:, i], a, prev)
    last_dir = np.nan_to_num(prev)
    first_dir = np.nan_to_num(first_dir)
    seg_ribs = np.where(nz.any(axis=1), np.ceil(turn / q) + 2, 0).astype(np.int64)
    off = batch.path_seg_off.astype(np.int64)
    P = len(off) - 1
    est = np.zeros(2 * S + P, np.int64)
    # link index of segment s of path p: 2 s + p + 1; the join before it: 2 s + p
    seg_path = np.repeat(np.arange(P), np.diff(off))
    sidx = np.arange(S)
    est[2 * sidx + seg_path + 1] = seg_ribs
    join = batch.path_join.astype(np.int64)
    cap = batch.path_cap.astype(np.int64)
    jfix = np.vectorize(lambda j: _JOIN_RIBS.get(int(j), 4), otypes=[np.int64])
    cfix = np.vectorize(lambda c: _CAP_RIBS.get(int(c), 5), otypes=[np.int64])

    def join_est(paths, d):
        rnd = join[paths] == W.JOIN_ROUND
        return np.where(rnd, np.ceil(d / q) + 1, jfix(join[paths]) if len(paths) else 0).astype(np.int64)

    inner = sidx[(sidx > off[seg_path]) if S else np.zeros(0, bool)]
    if len(inner):
        d = np.abs(_wrap(first_dir[inner] - last_dir[inner - 1]))
        est[2 * inner + seg_path[inner]] = join_est(seg_path[inner], d)
    pid = np.arange(P)
    nonempty = np.diff(off) > 0
    closed = batch.path_closed.astype(bool) & nonempty
    opened = ~batch.path_closed.astype(bool) & nonempty
    if opened.any():
        po = pid[opened]
        c = np.where(cap[po] == W.CAP_ROUND, math.ceil(math.pi / q) + 1, cfix(cap[po]))
        est[2 * off[po] + po] = c
        est[2 * off[po + 1] + po] = c
    if closed.any():
        pc = pid[closed]
        d = np.abs(_wrap(first_dir[off[pc]] - last_dir[off[pc + 1] - 1]))
        est[2 * off[pc + 1] + pc] = join_est(pc, d)
    return est


def split_links(est: np.ndarray, G: int) -> np.ndarray:
    """G + 1 link boundaries (0 = b0 <= b1 <= ... <= bG = L) cutting the prefix
    of the estimates at r / G of its total (the nearest link boundary)."""
    L = len(est)
    pre = np.concatenate([[0], np.cumsum(est, dtype=np.int64)])
    total = pre[-1]
    b = np.zeros(G + 1, np.int64)
    b[G] = L
    for r in range(1, G):
        target = total * r / G
        i = int(np.searchsorted(pre, target))
        if i > 0 and target - pre[i - 1] < pre[min(i, L)] - target:
            i -= 1
        b[r] = min(max(i, b[r - 1]), L)
    return b


def path_of_link(batch, links) -> np.ndarray:
    """The path of each (global) link index."""
    off = batch.path_seg_off.astype(np.int64)
    lbase = 2 * off[:-1] + np.arange(len(off) - 1)
    return np.searchsorted(lbase, np.asarray(links), side="right") - 1


def first_link(batch, p) -> int:
    off = batch.path_seg_off.astype(np.int64)
    return int(2 * off[p] + p)


def last_link(batch, p) -> int:
    off = batch.path_seg_off.astype(np.int64)
    return int(2 * off[p + 1] + p)


def join_plan(batch, bounds, n_rib, tail):
    """The exchange's result for every rank, from the gathered rib counts and
    tail lengths (tail[r]: s of rank r's last rib when that rib belongs to the
    path of its last link, else 0).  Returns a dict of arrays over ranks:
      rib_offset   global index of the rank's first rib;
      carry        the s carry of the path running into the rank's range (0
                   when the range starts a path);
      carry_path   that path (-1 when none);
      with_len     whether that path also ends in the range (its length takes
                   the carry too)."""
    G = len(bounds) - 1
    n_rib = np.asarray(n_rib, np.int64)
    tail = np.asarray(tail, np.float64)
    rib_offset = np.concatenate([[0], np.cumsum(n_rib)[:-1]]).astype(np.int64)
    carry = np.zeros(G)
    carry_path = np.full(G, -1, np.int64)
    with_len = np.zeros(G, bool)
    for r in range(G):
        l0, l1 = int(bounds[r]), int(bounds[r + 1])
        if l1 <= l0 or r == 0:
            continue
        p = int(path_of_link(batch, l0))
        if first_link(batch, p) == l0:
            continue  # the range starts its first path
        # the previous non-empty range ends inside p
        q = r - 1
        while q > 0 and bounds[q + 1] <= bounds[q]:
            q -= 1
        if bounds[q + 1] <= bounds[q] or int(path_of_link(batch, bounds[q + 1] - 1)) != p:
            continue
        prev_starts_p = first_link(batch, p) >= bounds[q]
        carry[r] = tail[q] + (0.0 if prev_starts_p else carry[q])
        carry_path[r] = p
        with_len[r] = last_link(batch, p) < l1
    return {"rib_offset": rib_offset, "carry": carry, "carry_path": carry_path,
            "with_len": with_len}


def exchange(n_rib: int, tail: float, group=None):
    """The one exchange step: all-gather of (rib count, tail length) over the
    process group (gloo on CPU tensors, NCCL on the device).  Returns the
    gathered (n_rib [G] int64, tail [G] float64) as numpy arrays."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    G = dist.get_world_size(group)
    mine = torch.tensor([float(n_rib), float(tail)], dtype=torch.float64, device=dev)
    out = [torch.zeros(2, dtype=torch.float64, device=dev) for _ in range(G)]
    dist.all_gather(out, mine, group=group)
    arr = torch.stack(out).cpu().numpy()
    return arr[:, 0].astype(np.int64), arr[:, 1]


# ---------------------------------------------------------------------------
# The raster half: the canvas is split by tile rows, rank d owning pixel rows
# [bounds[d], bounds[d + 1]).  Each rank routes the quads of its links to the
# owners of the rows they reach (``ps_route_quads``, on the device), one
# all-to-all moves them, and each owner covers its rows from the quads of all
# ranks (``ps_rasterize_coverage_rows``): every tile then sees every quad of
# every path that reaches it, so its per-path unions (Sec. 3.3.6) are those of
# one rank stroking the whole batch.  Per-path sample counts add up over the
# windows (one all-reduce); the canvas is the windows stacked.

TILE_PX = 16


def raster_rows(height: int, G: int) -> np.ndarray:
    """G + 1 pixel-row bounds splitting a canvas of ``height`` rows into G
    windows of whole tile rows (int32; bounds[0] = 0, bounds[G] = height)."""
    tiles_y = -(-int(height) // TILE_PX)
    b = np.array([TILE_PX * ((r * tiles_y) // G) for r in range(G + 1)], np.int64)
    b = np.minimum(b, int(height))
    b[G] = int(height)
    return b.astype(np.int32)


def route(ps, ctx, rib, tag, n_rib, capacity, width, height, bounds, stream=None):
    """Group this rank's quads by destination rank (``ps_route_quads``).
    Returns (quad ribs float32 [Q, 8], quad tags int32 [Q, 2], counts int64 [G])
    on the device, grouped by destination in rank order."""
    import torch
    dev = rib.device
    G = len(bounds) - 1
    rb = torch.as_tensor(np.asarray(bounds, np.int32), device=dev)
    cnt = torch.zeros(G, dtype=torch.int64, device=dev)
    off = torch.zeros(G + 1, dtype=torch.int64, device=dev)
    # a quad reaches few windows: size the output from a counting call first
    ps.ps_route_quads(ctx, rib, tag, n_rib, capacity, width, height, rb, None, None, 0, cnt, off,
                      stream)
    Q = int(off[G].item())  # synchronizes
    out_rib = torch.empty((max(Q, 1), 8), dtype=torch.float32, device=dev)
    out_tag = torch.empty((max(Q, 1), 2), dtype=torch.int32, device=dev)
    ps.ps_route_quads(ctx, rib, tag, n_rib, capacity, width, height, rb, out_rib, out_tag, Q, cnt,
                      off, stream)
    return out_rib[:Q], out_tag[:Q], cnt


def exchange_quads(out_rib, out_tag, counts, group=None):
    """The all-to-all of routed quads: this rank's blocks (grouped by
    destination, ``counts[d]`` quads for rank d) go to their ranks, and the
    blocks addressed to this rank arrive in rank order.  Returns (ribs [2 n, 4],
    tags [2 n], the dtypes of the inputs) for ``ps_rasterize_coverage_rows``:
    the quads as a rib stream."""
    import torch
    import torch.distributed as dist
    send = [int(c) for c in torch.as_tensor(counts).cpu().tolist()]
    G = dist.get_world_size(group)
    c_in = torch.tensor(send, dtype=torch.int64, device=out_rib.device)
    c_out = torch.empty(G, dtype=torch.int64, device=out_rib.device)
    dist.all_to_all_single(c_out, c_in, group=group)
    recv = [int(c) for c in c_out.cpu().tolist()]
    n = sum(recv)
    r_rib = torch.empty((n, 8), dtype=out_rib.dtype, device=out_rib.device)
    r_tag = torch.empty((n, 2), dtype=out_tag.dtype, device=out_tag.device)
    dist.all_to_all_single(r_rib, out_rib.contiguous(), output_split_sizes=recv,
                           input_split_sizes=send, group=group)
    dist.all_to_all_single(r_tag, out_tag.contiguous(), output_split_sizes=recv,
                           input_split_sizes=send, group=group)
    return r_rib.reshape(2 * n, 4), r_tag.reshape(2 * n)


def merge_covered(covered, group=None):
    """Per-path sample counts of the whole canvas: the sum over the windows."""
    import torch.distributed as dist
    dist.all_reduce(covered, op=dist.ReduceOp.SUM, group=group)
    return covered


def gather_rows(canvas_rows, bounds, group=None):
    """The whole canvas on every rank: the windows stacked in row order."""
    import torch
    import torch.distributed as dist
    G = len(bounds) - 1
    hmax = max(int(bounds[d + 1] - bounds[d]) for d in range(G))
    W = canvas_rows.shape[1]
    pad = torch.zeros((hmax, W), dtype=canvas_rows.dtype, device=canvas_rows.device)
    pad[:canvas_rows.shape[0]] = canvas_rows
    parts = [torch.empty_like(pad) for _ in range(G)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[d][:int(bounds[d + 1] - bounds[d])] for d in range(G)])
