"""Seeded synthetic stroke workloads.

This module only draws random numbers and places control points; it holds none
of the stroking method's arithmetic, so both the CUDA path and the FP64 oracle
can take their inputs from it.

A batch follows the library's input layout (see ``include/polarstroke.h``):

* ``seg_type``  uint8[S]       0 line, 1 quadratic, 2 cubic, 3 conic
* ``seg_pts``   float32[S,4,2] control points A, B, C, D (quadratic and conic
  use A, B, D; a line uses A, D)
* ``seg_w``     float32[S]     conic weight w_B (ignored for other forms)
* ``path_seg_off`` int32[P+1]  path p owns segments [off[p], off[p+1])
* ``path_width`` float32[P], ``path_join`` uint8[P], ``path_cap`` uint8[P],
  ``path_miter`` float32[P], ``path_closed`` uint8[P]

The five workloads are the shapes of the paper's uses (single long paths, many
paths of mixed segment forms, cusps and loops, near-degenerate cubics); the
paper's own path data is not published, so these are synthetic stand-ins.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LINE, QUAD, CUBIC, CONIC = 0, 1, 2, 3
JOIN_NONE, JOIN_BEVEL, JOIN_MITER, JOIN_MITER_TRUNCATE, JOIN_ROUND, JOIN_TRIANGLE = range(6)
CAP_BUTT, CAP_SQUARE, CAP_ROUND, CAP_TRIANGLE = range(4)

SEED_BASE = 20200700


@dataclass
class StrokeBatch:
    name: str
    seg_type: np.ndarray
    seg_pts: np.ndarray
    seg_w: np.ndarray
    path_seg_off: np.ndarray
    path_width: np.ndarray
    path_join: np.ndarray
    path_cap: np.ndarray
    path_miter: np.ndarray
    path_closed: np.ndarray
    dtheta: float                      # radians, as the float32 value the library sees
    canvas: tuple = (0, 0)             # (W, H) in px; (0, 0) = not rasterized
    spp: int = 16
    dash: tuple | None = None          # (pattern list, offset)
    meta: dict = field(default_factory=dict)

    @property
    def n_seg(self) -> int:
        return int(self.seg_type.shape[0])

    @property
    def n_path(self) -> int:
        return int(self.path_width.shape[0])

    @property
    def n_link(self) -> int:
        return 2 * self.n_seg + self.n_path

    def subset(self, paths) -> "StrokeBatch":
        """The batch restricted to the given path indices (in that order)."""
        paths = np.asarray(paths, dtype=np.int64)
        segs = [np.arange(self.path_seg_off[p], self.path_seg_off[p + 1]) for p in paths]
        counts = np.array([len(s) for s in segs], dtype=np.int64)
        idx = np.concatenate(segs) if len(segs) else np.zeros(0, np.int64)
        off = np.zeros(len(paths) + 1, np.int32)
        off[1:] = np.cumsum(counts)
        return StrokeBatch(
            name=self.name + "[subset]",
            seg_type=self.seg_type[idx].copy(), seg_pts=self.seg_pts[idx].copy(),
            seg_w=self.seg_w[idx].copy(), path_seg_off=off,
            path_width=self.path_width[paths].copy(), path_join=self.path_join[paths].copy(),
            path_cap=self.path_cap[paths].copy(), path_miter=self.path_miter[paths].copy(),
            path_closed=self.path_closed[paths].copy(), dtheta=self.dtheta,
            canvas=self.canvas, spp=self.spp, dash=self.dash, meta=dict(self.meta))


def f32(x) -> float:
    return float(np.float32(x))


def make_batch(name, seg_type, seg_pts, seg_w, counts, width, join, cap, miter=4.0,
               closed=0, dtheta_deg=2.0, canvas=(0, 0), dash=None, meta=None) -> StrokeBatch:
    counts = np.asarray(counts, dtype=np.int64)
    P = len(counts)
    off = np.zeros(P + 1, np.int32)
    off[1:] = np.cumsum(counts)

    def per_path(v, dt):
        a = np.asarray(v, dtype=dt)
        return np.full(P, a, dt) if a.ndim == 0 else a.astype(dt)

    return StrokeBatch(
        name=name,
        seg_type=np.asarray(seg_type, np.uint8),
        seg_pts=np.asarray(seg_pts, np.float32).reshape(-1, 4, 2),
        seg_w=np.asarray(seg_w, np.float32),
        path_seg_off=off,
        path_width=per_path(width, np.float32),
        path_join=per_path(join, np.uint8),
        path_cap=per_path(cap, np.uint8),
        path_miter=per_path(miter, np.float32),
        path_closed=per_path(closed, np.uint8),
        dtheta=f32(math.radians(dtheta_deg)),
        canvas=tuple(canvas), dash=dash, meta=meta or {})


def single(seg_type, pts, w=1.0, width=8.0, join=JOIN_ROUND, cap=CAP_ROUND, dtheta_deg=2.0,
           miter=4.0, closed=0, canvas=(0, 0)) -> StrokeBatch:
    """One path made of the given segments (pts: list of 4 points each)."""
    seg_type = np.atleast_1d(np.asarray(seg_type, np.uint8))
    pts = np.asarray(pts, np.float64).reshape(-1, 4, 2)
    wv = np.broadcast_to(np.asarray(w, np.float32), seg_type.shape)
    return make_batch("single", seg_type, pts, wv, [len(seg_type)], width, join, cap, miter,
                      closed, dtheta_deg, canvas)


def _unit(h):
    return np.stack([np.cos(h), np.sin(h)], axis=-1)


def _grid(v, g=64.0):
    return np.round(np.asarray(v) * g) / g


# ---- c1: plain method, small -------------------------------------------------
def c1_plain_small(seed: int = SEED_BASE + 1) -> StrokeBatch:
    """One open path of 64 chained cubic Beziers; A of segment 0 and every B, C, D
    uniform in [0,512]^2; width 8 px; round joins and caps; dtheta 2 deg; 512x512 at
    16 samples/pixel."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 64
    pts = np.zeros((n, 4, 2))
    a = rng.uniform(0, 512, 2)
    for i in range(n):
        pts[i, 0] = a
        pts[i, 1:] = rng.uniform(0, 512, (3, 2))
        a = pts[i, 3]
    return make_batch("c1_plain_small", np.full(n, CUBIC), pts, np.ones(n), [n], 8.0,
                      JOIN_ROUND, CAP_ROUND, dtheta_deg=2.0, canvas=(512, 512))


# ---- c2: batching ---------------------------------------------------------------
_LOOP_UNIT = np.array([[0.0, 0.0], [1.5, 1.0], [-0.5, 1.0], [1.0, 0.0]])


def c2_batching(n_paths: int = 10000, seed: int = SEED_BASE + 2, canvas: int = 2048,
                mean_segs: float = 30.0, max_segs: int = 200) -> StrokeBatch:
    """Many open paths of mixed segment forms on a random walk.

    Segments per path ~ Geometric(1/mean) on {1, 2, ...}, redrawn above max_segs.
    Step length log-uniform [1, 200] px, heading change uniform in (-pi, pi); a step
    that would leave the canvas bounces off its edge.  Points sit on a 1/64-px grid so
    that exact constructions stay exact in FP32.  Forms: 20% line, 20% quadratic,
    45% cubic, 15% conic (w_B log-uniform [0.1, 10]).  20% of cubics are exact cusps
    (C = A + B - D, so g'(1/2) = 0) or loops (a similarity image of a fixed loop
    control polygon), half each.  Widths log-uniform [0.5, 64] px; joins uniform over
    {miter (limit 4), round, bevel}; caps uniform over {butt, square, round};
    dtheta 1 deg; canvas 2048^2 at 16 samples/pixel."""
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = rng.geometric(1.0 / mean_segs, n_paths)
    while (counts > max_segs).any():
        bad = counts > max_segs
        counts[bad] = rng.geometric(1.0 / mean_segs, int(bad.sum()))
    S = int(counts.sum())
    types = rng.choice([LINE, QUAD, CUBIC, CONIC], size=S, p=[0.2, 0.2, 0.45, 0.15])
    weights = np.exp(rng.uniform(math.log(0.1), math.log(10.0), S))
    special = rng.uniform(0, 1, S)
    pts = np.zeros((S, 4, 2))
    seg_w = np.ones(S)
    k = 0
    cw = float(canvas)
    for p in range(n_paths):
        a = _grid(rng.uniform(0, cw, 2))
        h = rng.uniform(-math.pi, math.pi)
        for _ in range(int(counts[p])):
            L = math.exp(rng.uniform(0.0, math.log(200.0)))
            hprev = h
            h = h + rng.uniform(-math.pi, math.pi)
            d = a + L * _unit(h)
            if not (0 <= d[0] <= cw):
                h = math.pi - h
            if not (0 <= d[1] <= cw):
                h = -h
            d = _grid(np.clip(a + L * _unit(h), 0, cw))
            t = types[k]
            pts[k, 0] = a
            pts[k, 3] = d
            if t == LINE:
                pts[k, 1] = a
                pts[k, 2] = d
            elif t in (QUAD, CONIC):
                b = _grid(a + (L / 2) * _unit(hprev + rng.uniform(-math.pi / 2, math.pi / 2)))
                pts[k, 1] = b
                pts[k, 2] = b
                if t == CONIC:
                    seg_w[k] = weights[k]
            else:
                sp = special[k]
                if sp < 0.10 and not np.array_equal(d, a):
                    # exact cusp: C = A + B - D  =>  g'(1/2) = 0; needs B != D
                    b = _grid(a + (L / 3) * _unit(hprev + rng.uniform(-math.pi / 2, math.pi / 2)))
                    if np.array_equal(b, d):
                        b = b + 1.0 / 64
                    pts[k, 1] = b
                    pts[k, 2] = a + b - d
                elif sp < 0.20 and not np.array_equal(d, a):
                    # loop: similarity image of a fixed loop polygon, endpoints A -> D
                    e = d - a
                    rot = np.array([[e[0], -e[1]], [e[1], e[0]]])
                    u = _LOOP_UNIT.copy()
                    if rng.uniform() < 0.5:
                        u[:, 1] = -u[:, 1]
                    q = a + u @ rot.T
                    pts[k, 1] = _grid(q[1])
                    pts[k, 2] = _grid(q[2])
                else:
                    pts[k, 1] = _grid(a + (L / 3) * _unit(hprev + rng.uniform(-math.pi / 2, math.pi / 2)))
                    pts[k, 2] = _grid(d - (L / 3) * _unit(h + rng.uniform(-math.pi / 2, math.pi / 2)))
            a = d
            k += 1
    widths = np.exp(rng.uniform(math.log(0.5), math.log(64.0), n_paths))
    joins = rng.choice([JOIN_MITER, JOIN_ROUND, JOIN_BEVEL], n_paths)
    caps = rng.choice([CAP_BUTT, CAP_SQUARE, CAP_ROUND], n_paths)
    return make_batch("c2_batching", types, pts, seg_w, counts, widths, joins, caps, 4.0, 0,
                      dtheta_deg=1.0, canvas=(canvas, canvas),
                      meta={"cusp_or_loop": special})


# ---- c3: large single path ------------------------------------------------------
def c3_large_path(n_seg: int = 5031, seed: int = SEED_BASE + 3, canvas: int = 4096) -> StrokeBatch:
    """One open random-walk chain of cubics: step L log-uniform [1,200] px, heading
    h_k = h_{k-1} + U(-pi, pi), D = A + L u(h_k), B = A + (L/3) u(h_{k-1} + U(-pi/2, pi/2)),
    C = D - (L/3) u(h_k + U(-pi/2, pi/2)); steps bounce off the canvas edges.  Width
    2 px, round joins and caps, dtheta 0.5 deg, dash [12 on, 6 off], 4096^2 at 16 spp."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = np.zeros((n_seg, 4, 2))
    cw = float(canvas)
    a = rng.uniform(0.25 * cw, 0.75 * cw, 2)
    h = rng.uniform(-math.pi, math.pi)
    for k in range(n_seg):
        L = math.exp(rng.uniform(0.0, math.log(200.0)))
        hprev = h
        h = h + rng.uniform(-math.pi, math.pi)
        d = a + L * _unit(h)
        if not (0 <= d[0] <= cw):
            h = math.pi - h
        if not (0 <= d[1] <= cw):
            h = -h
        d = np.clip(a + L * _unit(h), 0, cw)
        pts[k, 0] = a
        pts[k, 1] = a + (L / 3) * _unit(hprev + rng.uniform(-math.pi / 2, math.pi / 2))
        pts[k, 2] = d - (L / 3) * _unit(h + rng.uniform(-math.pi / 2, math.pi / 2))
        pts[k, 3] = d
        a = np.float32(d).astype(np.float64)  # chain on the stored FP32 value
    pts = pts.astype(np.float32)
    pts[1:, 0] = pts[:-1, 3]
    return make_batch("c3_large_path", np.full(n_seg, CUBIC), pts, np.ones(n_seg), [n_seg],
                      2.0, JOIN_ROUND, CAP_ROUND, dtheta_deg=0.5, canvas=(canvas, canvas),
                      dash=([12.0, 6.0], 0.0))


# ---- c4: precision stress --------------------------------------------------------
_CUSP_UNIT = np.array([[0.0, 0.0], [1.0, 1.0], [0.0, 1.0], [1.0, 0.0]])


def c4_precision(n: int = 1_000_000, seed: int = SEED_BASE + 4) -> StrokeBatch:
    """Isolated cubics near exact cusps (half) and near collinearity (half).

    Cusp half: the cubic (0,0),(1,1),(0,1),(1,0) (cusp at t = 1/2) under a random
    similarity: scale log-uniform [0.1, 1e3] px, uniform rotation, translation
    uniform in [-1e6, 1e6]^2 px.  Collinear half: four points on a random line at
    parameters 0, b, c, 1 with b, c uniform in [-0.5, 1.5] (back-tracking allowed),
    same similarity.  Then every coordinate moves by (size * r * sign) with r
    log-uniform [1e-6, 1e-2].  Width 1 px, butt caps, dtheta 1 deg, no raster."""
    rng = np.random.Generator(np.random.PCG64(seed))
    half = n // 2
    scale = np.exp(rng.uniform(math.log(0.1), math.log(1e3), n))
    rot = rng.uniform(-math.pi, math.pi, n)
    trans = rng.uniform(-1e6, 1e6, (n, 2))
    unit = np.zeros((n, 4, 2))
    unit[:half] = _CUSP_UNIT
    bc = rng.uniform(-0.5, 1.5, (n - half, 2))
    unit[half:, 1, 0] = bc[:, 0]
    unit[half:, 2, 0] = bc[:, 1]
    unit[half:, 3, 0] = 1.0
    c, s = np.cos(rot), np.sin(rot)
    R = np.stack([np.stack([c, -s], -1), np.stack([s, c], -1)], -2)  # [n,2,2]
    pts = np.einsum("nij,nkj->nki", R, unit) * scale[:, None, None] + trans[:, None, :]
    rel = np.exp(rng.uniform(math.log(1e-6), math.log(1e-2), (n, 4, 2)))
    sgn = rng.choice([-1.0, 1.0], (n, 4, 2))
    pts = pts + sgn * rel * scale[:, None, None]
    return make_batch("c4_precision", np.full(n, CUBIC), pts, np.ones(n), np.ones(n, np.int64),
                      1.0, JOIN_ROUND, CAP_BUTT, dtheta_deg=1.0,
                      meta={"near_cusp": np.arange(n) < half})


# ---- c5: differentiation ---------------------------------------------------------
def c5_differentiation(n_paths: int = 4096, n_seg: int = 32,
                       seed: int = SEED_BASE + 5) -> StrokeBatch:
    """n_paths open paths of n_seg chained cubics; all points uniform in [0,1024]^2;
    widths uniform [1, 16] px; round joins and caps; dtheta 2 deg."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.uniform(0, 1024, (n_paths, n_seg, 4, 2))
    pts[:, 1:, 0] = pts[:, :-1, 3]
    widths = rng.uniform(1, 16, n_paths)
    S = n_paths * n_seg
    return make_batch("c5_differentiation", np.full(S, CUBIC), pts.reshape(S, 4, 2), np.ones(S),
                      np.full(n_paths, n_seg), widths, JOIN_ROUND, CAP_ROUND, dtheta_deg=2.0,
                      canvas=(1024, 1024))


def facet_comparison(n_paths: int = 20000, seed: int = SEED_BASE + 6,
                     dtheta_deg: float = 4.0) -> StrokeBatch:
    """Single-cubic open paths for the uniform-parametric comparison: half
    serpentines (B and C on opposite sides of the chord), a quarter exact cusps
    (C = A + B - D on a 1/64-px grid), a quarter loops (a cusp with C pushed off
    along the chord); chord length log-uniform 20-400 px at a random angle,
    widths log-uniform 1-100 px, butt caps, dtheta 4 deg (the paper's figure)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = np.zeros((n_paths, 4, 2))
    kind = rng.uniform(0, 1, n_paths)
    for i in range(n_paths):
        L = math.exp(rng.uniform(math.log(20.0), math.log(400.0)))
        ang = rng.uniform(-math.pi, math.pi)
        c, s_ = math.cos(ang), math.sin(ang)
        rot = np.array([[c, -s_], [s_, c]])
        o = rng.uniform(0, 1024, 2)
        if kind[i] < 0.5:
            b = [rng.uniform(0.1, 0.6) * L, rng.uniform(0.2, 1.0) * L]
            cc = [rng.uniform(0.4, 0.9) * L, -rng.uniform(0.2, 1.0) * L]
            local = np.array([[0, 0], b, cc, [L, 0]])
        else:
            A, D = np.array([0.0, 0.0]), np.array([L, 0.0])
            B = np.array([rng.uniform(0.2, 1.2) * L, rng.uniform(0.3, 1.0) * L])
            C = A + B - D
            if kind[i] >= 0.75:
                C = C + np.array([rng.uniform(0.05, 0.3) * L, 0.0])
            local = np.array([A, B, C, D])
        pts[i] = _grid(local @ rot.T + o)
        if kind[i] >= 0.5 and kind[i] < 0.75:
            pts[i, 2] = pts[i, 0] + pts[i, 1] - pts[i, 3]  # exact on the grid
    widths = np.exp(rng.uniform(math.log(1.0), math.log(100.0), n_paths))
    return make_batch("facet_comparison", np.full(n_paths, CUBIC), pts, np.ones(n_paths),
                      np.ones(n_paths, np.int64), widths, JOIN_ROUND, CAP_BUTT,
                      dtheta_deg=dtheta_deg, canvas=(0, 0))


CONFIGS = {
    "c1": c1_plain_small,
    "c2": c2_batching,
    "c3": c3_large_path,
    "c4": c4_precision,
    "c5": c5_differentiation,
}
