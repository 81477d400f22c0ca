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
