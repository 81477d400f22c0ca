"""Oracle pins for capped dash ends (Sec. 5.2, reading R18): every on-stretch
gets the path's cap style at its ends inside the path, as a path cap about the
boundary rib."""
import math

import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W


def line_batch(cap, width=10.0, length=100.0, y=20.0, dtheta_deg=2.0):
    return W.single(W.LINE, [[0, y], [0, y], [length, y], [length, y]], width=width, cap=cap,
                    dtheta_deg=dtheta_deg)


def test_butt_caps_change_nothing():
    b = line_batch(W.CAP_BUTT)
    o = oracle.tessellate(b)
    d0 = oracle.dash(o["rib"], o["s"], o["tag"], [12, 6], 0.0)
    d1 = oracle.dash_capped(o["rib"], o["s"], o["tag"], [12, 6], 0.0, b.path_cap, b.dtheta)
    for k in ("rib", "s", "tag", "src"):
        assert np.array_equal(d0[k], d1[k])


def test_round_dash_caps_are_semicircles():
    """Line from (0, 20) to (100, 20), w = 10, pattern [12, 6]: stretches [0,12),
    [18,30), ..., [90,102).  Each stretch end inside (0, 100] gets a half disc
    ahead of it, each start inside (0, 100) one behind it; the path's own caps
    remain where the pattern is on at s = 0 and s = 100."""
    b = line_batch(W.CAP_ROUND)
    q = b.dtheta
    J = int(math.ceil(math.pi / q - 1e-4))
    o = oracle.tessellate(b)
    d = oracle.dash_capped(o["rib"], o["s"], o["tag"], [12, 6], 0.0, b.path_cap, q)
    starts = np.where(d["tag"] & oracle.TAG_LINK_START)[0]
    ends = np.r_[starts[1:], len(d["s"])]
    # dash caps are strips of J + 1 ribs at constant s (the path's own cap quads
    # come out of the dasher as 2-rib pieces)
    caps = [(a, e) for a, e in zip(starts, ends) if e - a > 2]
    dash_ends = [12.0 + 18 * k for k in range(5)]    # 12, 30, ..., 84
    dash_starts = [18.0 + 18 * k for k in range(5)]  # 18, 36, ..., 90
    assert len(caps) == len(dash_ends) + len(dash_starts)
    seen_end, seen_start = [], []
    for a, e in caps:
        assert e - a == J + 1
        assert not ((d["tag"][a:e] >> 1) & 1).any()
        sv = d["s"][a]
        assert np.all(d["s"][a:e] == sv)
        c = np.array([sv, 20.0])
        N, P = d["rib"][a:e, 0:2], d["rib"][a:e, 2:4]
        assert np.abs(P - c).max() < 1e-9  # inner radius 0: P is the centre
        assert np.abs(np.hypot(*(N - c).T) - 5.0).max() < 1e-9
        ang = np.unwrap(np.arctan2(N[:, 1] - c[1], N[:, 0] - c[0]))
        assert np.abs(np.diff(ang) - math.pi / J).max() < 1e-9  # counter-clockwise sweep
        if (N[:, 0] - sv >= -1e-9).all():
            seen_end.append(sv)      # half disc ahead of the stretch's end
        elif (N[:, 0] - sv <= 1e-9).all():
            seen_start.append(sv)    # half disc behind the stretch's start
    assert sorted(seen_end) == dash_ends
    assert sorted(seen_start) == dash_starts


def _raster_count(rib, tag, Wc, Hc):
    can, cov = oracle.raster(rib, tag, Wc, Hc, 1)
    return can, int(cov[0])


def test_square_capped_dashes_cover_exactly_their_rectangles():
    """Square caps extend each stretch by w/2 at both ends, so the capped dashed
    line covers exactly the samples inside the union of the rectangles
    [a - 5, min(b, 100) + 5] x [15, 25] (the path's own square caps extend the
    first and last stretch past 0 and 100)."""
    b = line_batch(W.CAP_SQUARE)
    o = oracle.tessellate(b)
    d = oracle.dash_capped(o["rib"], o["s"], o["tag"], [12, 6], 0.0, b.path_cap, b.dtheta)
    Wc, Hc = 128, 48
    can, n = _raster_count(d["rib"], d["tag"], Wc, Hc)
    xs = oracle.sample_positions(Wc, Hc)
    X, Y = xs[..., 0], xs[..., 1]
    inside = np.zeros(X.shape, bool)
    for a0 in np.arange(0, 100, 18.0):
        lo, hi = a0 - 5.0, min(a0 + 12.0, 100.0) + 5.0
        inside |= (X >= lo) & (X <= hi) & (Y >= 15.0) & (Y <= 25.0)
    exp = np.zeros((Hc, Wc), np.uint16)
    for k in range(16):
        exp |= (inside[..., k].astype(np.uint16) << k)
    assert np.array_equal(can, exp)
    assert n == int(inside.sum())


def test_cap_count_matches_stretch_ends_on_curves():
    rng = np.random.default_rng(11)
    for cap in (W.CAP_ROUND, W.CAP_SQUARE, W.CAP_TRIANGLE):
        pts = rng.uniform(0, 300, (4, 2))
        b = W.single(W.CUBIC, pts, width=6, cap=cap, dtheta_deg=2.0)
        o = oracle.tessellate(b)
        pat = [float(rng.uniform(3, 20)), float(rng.uniform(2, 10))]
        off = float(rng.uniform(0, 10))
        d0 = oracle.dash(o["rib"], o["s"], o["tag"], pat, off)
        d = oracle.dash_capped(o["rib"], o["s"], o["tag"], pat, off, b.path_cap, b.dtheta)
        J = {W.CAP_ROUND: int(math.ceil(math.pi / b.dtheta - 1e-4)), W.CAP_SQUARE: 4,
             W.CAP_TRIANGLE: 2}[cap]
        L = float(o["path_len"][0])
        period = pat[0] + pat[1]
        n_caps = 0
        k = math.floor(off / period) - 1
        while k * period - off <= L:
            a, e = k * period - off, k * period - off + pat[0]
            n_caps += int(0.0 < a < L) + int(0.0 < e <= L)
            k += 1
        assert len(d["s"]) == len(d0["s"]) + n_caps * (J + 1)
        # the pieces themselves are unchanged
        seg = ((d["tag"] >> 1) & 1) == 1
        seg0 = ((d0["tag"] >> 1) & 1) == 1
        assert np.array_equal(d["rib"][seg], d0["rib"][seg0])
