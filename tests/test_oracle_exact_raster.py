"""Pins for the exact quad raster (reading R19: quads filled as polygons by the
crossing rule, bow-ties as such; Sec. 4.1 and Sec. 7), against geometry that
does not use the crossing rule: a convex quad is its two triangles, a simple
concave quad is split along its interior diagonal, a bow-tie quad is the two
lobe triangles at the crossing point of its ribs (an exact rational point)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W


def quad_stream(N0, P0, P1, N1):
    rib = np.array([[*N0, *P0], [*N1, *P1]], np.float64)
    tag = np.array([1 | 2, 2], np.uint32)  # one path, one segment link of two ribs
    return rib, tag


def snapped(v):
    return int(np.rint(v * 256.0))


def samples(Wc, Hc):
    xs = oracle.sample_positions(Wc, Hc)
    return (np.rint(xs[..., 0] * 256).astype(np.int64), np.rint(xs[..., 1] * 256).astype(np.int64))


def side(a, b, px, py):
    return (b[0] - a[0]) * (py - a[1]) - (b[1] - a[1]) * (px - a[0])


def in_tri(a, b, c, px, py):
    """Closed triangle test in exact integer (or rational) arithmetic, vectorised
    over sample arrays of Python objects."""
    s0, s1, s2 = side(a, b, px, py), side(b, c, px, py), side(c, a, px, py)
    return ((s0 >= 0) & (s1 >= 0) & (s2 >= 0)) | ((s0 <= 0) & (s1 <= 0) & (s2 <= 0))


def on_any_line(pts, px, py):
    hit = np.zeros(px.shape, bool)
    for i in range(len(pts)):
        for j in range(i + 1, len(pts)):
            hit |= side(pts[i], pts[j], px, py) == 0
    return hit


def to_mask(inside):
    m = np.zeros(inside.shape[:2], np.uint16)
    for k in range(16):
        m |= inside[..., k].astype(np.uint16) << k
    return m


def test_bow_tie_is_its_two_lobes():
    # ribs N0-P0 and N1-P1 cross; off-grid coordinates keep samples off every line
    N0, P0, N1, P1 = (10.3, 10.1), (50.2, 49.7), (49.9, 10.4), (10.6, 50.3)
    Wc, Hc = 64, 64
    rib, tag = quad_stream(N0, P0, P1, N1)
    can, cov = oracle.raster(rib, tag, Wc, Hc, 1, exact=True)
    can2, _ = oracle.raster(rib, tag, Wc, Hc, 1)
    v = {k: (snapped(x), snapped(y)) for k, (x, y) in zip("NPnp", (N0, P0, N1, P1))}
    # crossing point of the ribs, exactly
    (ax, ay), (bx, by), (cx, cy), (dx, dy) = v["N"], v["P"], v["n"], v["p"]
    den = (bx - ax) * (dy - cy) - (by - ay) * (dx - cx)
    t = Fraction((cx - ax) * (dy - cy) - (cy - ay) * (dx - cx), den)
    X = (ax + t * (bx - ax), ay + t * (by - ay))
    assert 0 < t < 1
    sx, sy = samples(Wc, Hc)
    SX, SY = sx.astype(object), sy.astype(object)
    lobe_a = in_tri(X, v["P"], v["p"], SX, SY)
    lobe_b = in_tri(X, v["n"], v["N"], SX, SY)
    assert not on_any_line([v["N"], v["P"], v["n"], v["p"], X], SX, SY)[lobe_a | lobe_b].any()
    exp = to_mask(lobe_a | lobe_b)
    assert np.array_equal(can, exp)
    assert int(cov[0]) == int((lobe_a | lobe_b).sum())
    # the two-triangle raster covers the lobes and more (the excess of Sec. 7)
    assert np.array_equal(can2 & can, can) and (can2 != can).any()


@pytest.mark.parametrize("seed", range(6))
def test_convex_and_concave_quads(seed):
    rng = np.random.default_rng(500 + seed)
    Wc, Hc = 48, 48
    done = 0
    while done < 20:
        pts = rng.uniform(4, 44, (4, 2)) + rng.uniform(0, 1, (4, 2)) * 0.37
        N0, P0, P1, N1 = (tuple(p) for p in pts)
        q = [(snapped(x), snapped(y)) for x, y in (N0, P0, P1, N1)]
        # skip self-intersecting polygons here (bow-ties have their own pin)
        def cr(a, b, c):
            return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
        def segs_cross(a, b, c, d):
            return cr(a, b, c) * cr(a, b, d) < 0 and cr(c, d, a) * cr(c, d, b) < 0
        if segs_cross(q[0], q[1], q[2], q[3]) or segs_cross(q[1], q[2], q[3], q[0]):
            continue
        turns = [cr(q[i], q[(i + 1) % 4], q[(i + 2) % 4]) for i in range(4)]
        if 0 in turns:
            continue
        sx, sy = samples(Wc, Hc)
        SX, SY = sx.astype(object), sy.astype(object)
        if on_any_line(q, SX, SY).any():
            continue
        # a convex quad is either diagonal's two triangles; a simple concave one
        # splits along the diagonal from its reflex vertex
        convex = all(t > 0 for t in turns) or all(t < 0 for t in turns)
        if convex:
            inside = in_tri(q[0], q[1], q[2], SX, SY) | in_tri(q[0], q[2], q[3], SX, SY)
        else:
            r = next(i for i in range(4)
                     if np.sign(turns[(i - 1) % 4]) != np.sign(sum(np.sign(turns))))
            # reflex vertex at index r: the diagonal from it is interior
            a, b, c, d = (q[(r + k) % 4] for k in range(4))
            inside = in_tri(a, b, c, SX, SY) | in_tri(a, c, d, SX, SY)
        rib, tag = quad_stream(tuple(np.array(q[0]) / 256.0), tuple(np.array(q[1]) / 256.0),
                               tuple(np.array(q[2]) / 256.0), tuple(np.array(q[3]) / 256.0))
        can, cov = oracle.raster(rib, tag, Wc, Hc, 1, exact=True)
        assert np.array_equal(can, to_mask(inside)), (seed, done, convex)
        if convex:
            can2, _ = oracle.raster(rib, tag, Wc, Hc, 1)
            assert np.array_equal(can, can2)
        done += 1


def test_exact_stroke_coverage_within_two_triangle_coverage():
    """A wide stroke around a tight bend folds its inner side into bow-tie quads
    (ribs crossing).  Each bow-tie quad alone covers strictly less exactly than
    as two triangles (the excess of Sec. 7); the path's exact coverage lies
    inside its two-triangle coverage (here the neighbouring quads hide the
    excess of the union, as Sec. 7 notes for round joins)."""
    b = W.single(W.CUBIC, [[20, 100], [220, 20], [-60, 20], [150, 100]], width=40,
                 join=W.JOIN_ROUND, cap=W.CAP_BUTT, dtheta_deg=4.0, canvas=(200, 140))
    o = oracle.tessellate(b)
    Wc, Hc = 200, 140
    ex, _ = oracle.raster(o["rib"], o["tag"], Wc, Hc, 1, exact=True)
    tt, _ = oracle.raster(o["rib"], o["tag"], Wc, Hc, 1)
    assert np.array_equal(tt & ex, ex)

    def cr(a, b, c):
        return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
    rib, tag = o["rib"], o["tag"]
    bows = 0
    for i in range(1, len(rib)):
        if tag[i] & oracle.TAG_LINK_START:
            continue
        N0, P0, N1, P1 = (tuple(np.rint(np.array(v) * 256).astype(np.int64))
                          for v in (rib[i - 1, :2], rib[i - 1, 2:], rib[i, :2], rib[i, 2:]))
        if not (cr(N0, P0, N1) * cr(N0, P0, P1) < 0 and cr(N1, P1, N0) * cr(N1, P1, P0) < 0):
            continue
        bows += 1
        q = np.array([rib[i - 1], rib[i]])
        qt = np.array([3, 2], np.uint32)
        e1, c1 = oracle.raster(q, qt, Wc, Hc, 1, exact=True)
        t1, c2 = oracle.raster(q, qt, Wc, Hc, 1)
        assert np.array_equal(t1 & e1, e1)
        assert int(c1[0]) < int(c2[0])
    assert bows > 5
