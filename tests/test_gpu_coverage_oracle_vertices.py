"""Coverage of the GPU's stroke against the oracle's stroke (Sec. 4.1, Sec. 3.3.6).

The GPU rasterizes its own ribs; the oracle's fixed-point raster (O2)
rasterizes the oracle's FP64 ribs.  The bar: at most 1e-4 of all samples of the
canvas differ, and every differing sample lies within 1/256 px of an edge of one
of the two sets of snapped triangles (two-triangle rule) or quads (crossing
rule).  Each test prints the differing fraction and the largest edge distance.

Samples that differ do so because a vertex's snapped position differs by one
1/256-px step between the two rib sets (the ribs agree to the vertex bar, and
snapping rounds either way near a half step), which moves an edge by at most
that step."""
import functools

import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W
from tests._parity import gpu_tessellate

pytestmark = pytest.mark.gpu

LINK_START = 1
TILE = 16  # px, the grid used to find the edges near a sample


def gpu_raster(g, batch, W_, H_, exact):
    import torch
    import paper_2007_00308_gb300 as ps
    canvas = torch.zeros((H_, W_), dtype=torch.int16, device="cuda")
    covered = torch.zeros(batch.n_path, dtype=torch.int64, device="cuda")
    out = g["out"]
    ps.ps_rasterize_coverage(g["ctx"], out.rib, out.tag, out.n_rib, out.capacity, batch.n_path,
                             W_, H_, canvas, covered, exact=exact)
    torch.cuda.synchronize()
    assert g["ctx"].status() == 0
    return canvas.cpu().numpy().view(np.uint16)


def edges_of(rib, tag, exact):
    """Snapped edges (1/256-px units) of the quads of a rib stream: for quad r
    (ribs r-1, r of one link) N0-P0, P0-P1, P1-N1, N1-N0, and for the
    two-triangle rule also the shared diagonal N0-P1.  Returns [E, 4] int64."""
    q = np.where((tag[1:] & LINK_START) == 0)[0] + 1
    v = np.rint(rib * 256.0).astype(np.int64)
    N0, P0, P1, N1 = v[q - 1, 0:2], v[q - 1, 2:4], v[q, 2:4], v[q, 0:2]
    pairs = [(N0, P0), (P0, P1), (P1, N1), (N1, N0)] + ([] if exact else [(N0, P1)])
    return np.concatenate([np.concatenate([a, b], axis=1) for a, b in pairs])


def tile_index(edges):
    """Map tile id -> edge indices for every 16-px tile an edge's box (grown by
    one 1/256-px step) touches."""
    lo = np.minimum(edges[:, 0:2], edges[:, 2:4]) - 1
    hi = np.maximum(edges[:, 0:2], edges[:, 2:4]) + 1
    t0 = np.floor_divide(lo, 256 * TILE)
    t1 = np.floor_divide(hi, 256 * TILE)
    nx = t1[:, 0] - t0[:, 0] + 1
    ny = t1[:, 1] - t0[:, 1] + 1
    cnt = nx * ny
    eid = np.repeat(np.arange(len(edges)), cnt)
    k = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    tx = t0[eid, 0] + k % nx[eid]
    ty = t0[eid, 1] + k // nx[eid]
    key = tx * 1_000_003 + ty
    order = np.argsort(key, kind="stable")
    return key[order], eid[order]


def seg_dist(px, py, e):
    """Distance (1/256-px units) from points (px, py) to segments e[:, 4]."""
    ax, ay, bx, by = (e[:, i][None, :].astype(np.float64) for i in range(4))
    dx, dy = bx - ax, by - ay
    L2 = dx * dx + dy * dy
    t = np.where(L2 > 0, ((px[:, None] - ax) * dx + (py[:, None] - ay) * dy) / np.where(L2 > 0, L2, 1), 0)
    t = np.clip(t, 0.0, 1.0)
    cx, cy = ax + t * dx - px[:, None], ay + t * dy - py[:, None]
    return np.sqrt(cx * cx + cy * cy)


def max_edge_distance(diff, edge_sets):
    """Largest, over the differing samples, of the distance (px) to the nearest
    edge of any of the edge sets."""
    ys, xs = np.nonzero(diff)
    if not len(ys):
        return 0.0
    k = np.arange(16)
    pts = []
    for y, x in zip(ys, xs):
        bits = int(diff[y, x])
        ks = k[(bits >> k) & 1 == 1]
        pts.append(np.stack([256 * x + 16 * ks + 8, 256 * y + 16 * ((5 * ks) % 16) + 8], 1))
    pts = np.concatenate(pts).astype(np.float64)
    best = np.full(len(pts), np.inf)
    tiles = np.floor_divide(pts.astype(np.int64), 256 * TILE)
    tkey = tiles[:, 0] * 1_000_003 + tiles[:, 1]
    for edges, (keys, eids) in edge_sets:
        for key in np.unique(tkey):
            sel = tkey == key
            a, b = np.searchsorted(keys, key), np.searchsorted(keys, key, side="right")
            if a == b:
                continue
            d = seg_dist(pts[sel, 0], pts[sel, 1], edges[eids[a:b]]).min(axis=1)
            best[sel] = np.minimum(best[sel], d)
    return float(best.max()) / 256.0


@functools.lru_cache(maxsize=None)
def _case_and_oracle(name):
    b = _case(name)
    return b, oracle.tessellate(b)


def _case(name):
    if name == "c1":
        return W.c1_plain_small()
    if name == "c2_300":
        return W.c2_batching(n_paths=300, seed=W.SEED_BASE + 2)
    if name == "c3_prefix":
        return W.c3_large_path(n_seg=600)
    if name == "c5_64":
        return W.c5_differentiation(n_paths=64)
    raise KeyError(name)


@pytest.mark.parametrize("exact", [False, True])
@pytest.mark.parametrize("name", ["c1", "c2_300", "c3_prefix", "c5_64"])
def test_coverage_against_oracle_vertices(name, exact):
    b, o = _case_and_oracle(name)
    Wd, Ht = b.canvas
    g = gpu_tessellate(b, 1, want_t=False)
    assert g["status"] == 0
    can = gpu_raster(g, b, Wd, Ht, exact)
    ocan, _ = oracle.raster(o["rib"], o["tag"], Wd, Ht, b.n_path, exact=exact)
    diff = can ^ ocan
    n_diff = int(np.unpackbits(diff.view(np.uint8)).sum())
    frac = n_diff / (Wd * Ht * 16.0)
    sets = []
    for rib, tag in ((g["rib"], g["tag"]), (o["rib"], o["tag"])):
        e = edges_of(rib, tag, exact)
        sets.append((e, tile_index(e)))
    dmax = max_edge_distance(diff, sets)
    print(f"{name} exact={exact}: {n_diff} of {Wd * Ht * 16} samples differ ({frac:.2e}); "
          f"farthest from an edge {dmax * 256:.3f}/256 px")
    assert frac <= 1e-4
    assert dmax <= 1.0 / 256.0 + 1e-12
