"""Pins for the pixel-scale boost of q (Sec. 7 names it as a heuristic; reading
R21 gives its rule).  The boosted step must keep every boundary edge within tau
px of the true stroke boundary; for round joins and caps, whose boundary is a
circle, it must also be the largest step that does (fewest ribs).  Checked
against closed-form sagittas and against dense sampling of the exact offset
curves, not against the rule's own formulas."""
import math

import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W


def _links(o):
    off = o["link_rib_off"]
    for l in range(len(off) - 1):
        a, b = int(off[l]), int(off[l + 1])
        if b > a:
            yield l, a, b


def _seg_dist(p, a, b):
    """Distance of points p[k] to the segment a-b."""
    ab = b - a
    L2 = float(ab @ ab)
    if L2 == 0.0:
        return np.hypot(*(p - a).T)
    t = np.clip(((p - a) @ ab) / L2, 0.0, 1.0)
    return np.hypot(*(p - (a + t[:, None] * ab)).T)


def _arc_gap(centre, r, v0, v1, n=200):
    """Largest distance from the arc of radius r about centre, between the
    directions of v0 and v1 (the short way), to the chord v0-v1."""
    a0 = math.atan2(v0[1] - centre[1], v0[0] - centre[0])
    a1 = math.atan2(v1[1] - centre[1], v1[0] - centre[0])
    d = (a1 - a0 + math.pi) % (2 * math.pi) - math.pi
    ang = a0 + d * np.linspace(0.0, 1.0, n)
    pts = np.stack([centre[0] + r * np.cos(ang), centre[1] + r * np.sin(ang)], 1)
    return float(_seg_dist(pts, np.asarray(v0), np.asarray(v1)).max())


def test_zero_tolerance_changes_nothing():
    b = W.c2_batching(n_paths=40, canvas=512)
    o0 = oracle.tessellate(b)
    o1 = oracle.tessellate(b, tau=0.0)
    for k in ("rib", "s", "tag", "link_nrib"):
        assert np.array_equal(o0[k], o1[k])


@pytest.mark.parametrize("width,tau,deg", [(8.0, 0.25, 2.0), (30.0, 0.1, 1.0), (3.0, 0.05, 1.0),
                                           (20.0, 1.0, 0.5)])
def test_round_caps_take_the_fewest_steps_within_tau(width, tau, deg):
    """A line with round caps: each cap's outer boundary is a half circle of
    radius r = w/2.  J steps of pi/J leave a gap r (1 - cos(pi / 2J)) between
    arc and chord; the cap must take the smallest J with gap <= tau."""
    b = W.single(W.LINE, [[50, 60], [50, 60], [250, 60], [250, 60]], width=width,
                 cap=W.CAP_ROUND, dtheta_deg=deg)
    r = 0.5 * width
    o = oracle.tessellate(b, tau=tau)
    q = b.dtheta
    J_q = math.ceil(math.pi / q - 1e-4)  # the unboosted count
    J_min = next(J for J in range(1, 10000) if r * (1 - math.cos(math.pi / (2 * J))) <= tau)
    caps = []
    for l, a, e in _links(o):
        if (o["tag"][a] >> 1) & 1:
            continue
        caps.append((a, e))
        J = e - a - 1
        assert J == min(J_q, J_min), (J, J_q, J_min)
        centre = np.array([50.0, 60.0]) if a == 0 else np.array([250.0, 60.0])
        N = o["rib"][a:e, 0:2]
        for j in range(1, J + 1):
            assert _arc_gap(centre, r, N[j - 1], N[j]) <= tau * (1 + 1e-9)
    assert len(caps) == 2


@pytest.mark.parametrize("turn_deg", [30.0, 90.0, 150.0, 179.0])
def test_round_joins_take_the_fewest_steps_within_tau(turn_deg):
    w, tau, deg = 12.0, 0.2, 1.0
    r = 0.5 * w
    th = math.radians(turn_deg)
    P0, P1 = np.array([100.0, 100.0]), np.array([200.0, 100.0])
    P2 = P1 + 100.0 * np.array([math.cos(th), math.sin(th)])
    pts = [[P0, P0, P1, P1], [P1, P1, P2, P2]]
    b = W.single([W.LINE, W.LINE], np.array(pts), width=w, join=W.JOIN_ROUND, cap=W.CAP_BUTT,
                 dtheta_deg=deg)
    o = oracle.tessellate(b, tau=tau)
    # the join turns by the angle between the lines (as stored in FP32)
    e = b.seg_pts[1, 3].astype(np.float64) - b.seg_pts[1, 0].astype(np.float64)
    delta = math.atan2(e[1], e[0])
    J_q = math.ceil(abs(delta) / b.dtheta - 1e-4)
    J_min = next(J for J in range(1, 10000) if r * (1 - math.cos(abs(delta) / (2 * J))) <= tau)
    joins = [(a, e) for l, a, e in _links(o) if not (o["tag"][a] >> 1) & 1]
    assert len(joins) == 1
    a, e = joins[0]
    assert e - a - 1 == min(J_q, J_min)
    # the outer side of a left turn is N; every chord within tau of its arc
    N = o["rib"][a:e, 0:2]
    for j in range(1, e - a):
        assert _arc_gap(P1, r, N[j - 1], N[j]) <= tau * (1 + 1e-9)


@pytest.mark.parametrize("R,w,tau", [(5.0, 3.0, 0.2), (0.5, 20.0, 0.25), (1.0, 40.0, 0.1)])
def test_quarter_circle_conic_closed_form(R, w, tau):
    """A = (R, 0), B = (R, R), D = (0, R), w_B = cos 45 deg is a quarter circle
    whose control polygon has length 2R; the ribs stay on the circles of radii
    |R +- r| at uniform angles, N = ceil((pi/2) / q_link), and every outer chord
    lies within tau of the radius-(R + r) circle.  The first case is bound by the
    control polygon's length, the other two by the width (the third with the
    two terms within 12% of each other)."""
    r = 0.5 * w
    b = W.single(W.CONIC, [[R, 0], [R, R], [R, R], [0, R]], w=math.cos(math.pi / 4), width=w,
                 cap=W.CAP_BUTT, dtheta_deg=1.0)
    o = oracle.tessellate(b, tau=tau)
    q_link = max(b.dtheta, min(2 * math.atan(tau / (2 * R)), math.sqrt(math.pi * tau / (2 * r)),
                               math.pi / 2))
    n_exp = math.ceil((math.pi / 2) / q_link - 1e-4)
    segs = [(a, e) for l, a, e in _links(o) if (o["tag"][a] >> 1) & 1]
    assert len(segs) == 1
    a, e = segs[0]
    assert e - a - 1 == n_exp < math.ceil((math.pi / 2) / b.dtheta - 1e-4)
    N, P = o["rib"][a:e, 0:2], o["rib"][a:e, 2:4]
    # the curve turns counter-clockwise, so its outer side is N (radius R + r)
    assert np.abs(np.hypot(*N.T) - (R + r)).max() < 1e-5
    assert np.abs(np.hypot(*P.T) - abs(R - r)).max() < 1e-5
    for j in range(1, e - a):
        assert _arc_gap((0.0, 0.0), R + r, N[j - 1], N[j]) <= tau
        if R >= r:  # the inner side does not fold
            assert _arc_gap((0.0, 0.0), R - r, P[j - 1], P[j]) <= tau


def _offset_points(g_eval, d_eval, t, r, side):
    """Exact offset curve g(t) + side * r * n(t), n the left normal of g'(t)."""
    g = g_eval(t)
    d = d_eval(t)
    n = np.stack([-d[:, 1], d[:, 0]], 1) / np.hypot(*d.T)[:, None]
    return g + side * r * n


def _cubic(P):
    A, B, C, D = (np.asarray(p, np.float64) for p in P)

    def g(t):
        t = t[:, None]
        u = 1 - t
        return u ** 3 * A + 3 * u * u * t * B + 3 * u * t * t * C + t ** 3 * D

    def d(t):
        t = t[:, None]
        u = 1 - t
        return 3 * (u * u * (B - A) + 2 * u * t * (C - B) + t * t * (D - C))

    def dd(t):
        t = t[:, None]
        return 6 * ((1 - t) * (C - 2 * B + A) + t * (D - 2 * C + B))
    return g, d, dd


@pytest.mark.parametrize("seed", range(4))
def test_segment_boundary_within_tau_by_dense_sampling(seed):
    """Small cubics (pixel-scale to tens of px) with widths 1-12 px: on every
    step of the boosted tessellation, the exact offset boundary on each side
    that does not fold (the outer side, or an inner side whose radius of
    curvature stays >= r) lies within tau of the quad's edge on that side."""
    rng = np.random.default_rng(900 + seed)
    tau = 0.25
    checked = boosted = 0
    for _ in range(25):
        scale = float(np.exp(rng.uniform(np.log(0.5), np.log(30.0))))
        P = rng.uniform(0, 1, (4, 2)) * scale + 100.0
        P = np.round(P * 64) / 64  # on the 1/64 grid, exact in FP32
        w = float(np.float32(np.exp(rng.uniform(0.0, np.log(12.0)))))
        b = W.single(W.CUBIC, P, width=w, cap=W.CAP_BUTT, dtheta_deg=1.0)
        o0 = oracle.tessellate(b)
        o = oracle.tessellate(b, tau=tau)
        r = 0.5 * w
        g, d, dd = _cubic(P)
        segs = [(a, e) for l, a, e in _links(o) if (o["tag"][a] >> 1) & 1]
        segs0 = [(a, e) for l, a, e in _links(o0) if (o0["tag"][a] >> 1) & 1]
        if not segs:
            continue
        (a, e), (a0, e0) = segs[0], segs0[0]
        assert e - a <= e0 - a0
        boosted += (e - a) < (e0 - a0)
        t = o["t"][a:e]
        psi = o["psi"][a:e]
        for j in range(1, e - a):
            if t[j] == t[j - 1]:
                # a pivot at a cusp: both sides sweep arcs of radius r about g(t)
                c = g(np.array([t[j]]))[0]
                for k in (0, 2):
                    v0, v1 = o["rib"][a + j - 1, k:k + 2], o["rib"][a + j, k:k + 2]
                    assert _arc_gap(c, r, v0, v1) <= tau * (1 + 1e-6) + 1e-9
                    checked += 1
                continue
            if t[j] < t[j - 1]:
                continue
            ts = np.linspace(t[j - 1], t[j], 65)[1:-1]
            if len(ts) == 0:
                continue
            dv, ddv = d(ts), dd(ts)
            cr = dv[:, 0] * ddv[:, 1] - dv[:, 1] * ddv[:, 0]
            sp = np.hypot(*dv.T)
            if (sp < 1e-9).any():
                continue
            rho = np.where(np.abs(cr) > 0, sp ** 3 / np.maximum(np.abs(cr), 1e-300), np.inf)
            turn = np.sign(cr[len(cr) // 2])
            for k, side in ((0, -1.0), (2, 1.0)):
                # N = g - r n is outer for a left (counter-clockwise) turn
                outer = (side < 0) == (turn > 0) or turn == 0
                if not outer and rho.min() < r:
                    continue
                pts = _offset_points(g, d, ts, r, side)
                v0, v1 = o["rib"][a + j - 1, k:k + 2], o["rib"][a + j, k:k + 2]
                gap = float(_seg_dist(pts, v0, v1).max())
                assert gap <= tau * (1 + 1e-6) + 1e-9, (seed, j, k, gap, float(psi[j]))
                checked += 1
    assert checked > 500 and boosted > 5


def test_large_tolerance_limits():
    """tau far above every link's size: segment steps cap at pi/2 (an interval
    turning by |delta| takes ceil(|delta| / (pi/2)) steps) and round joins and
    caps take a single step."""
    pts = [[[20, 100], [220, 20], [-60, 20], [150, 100]],
           [[150, 100], [300, 200], [100, 200], [250, 120]]]
    b = W.single([W.CUBIC, W.CUBIC], np.array(pts, np.float64), width=4, join=W.JOIN_ROUND,
                 cap=W.CAP_ROUND, dtheta_deg=1.0)
    o = oracle.tessellate(b, tau=1e6)
    for l, a, e in _links(o):
        n = e - a - 1
        if (o["tag"][a] >> 1) & 1:
            # the segment as tessellated plainly at q = pi/2
            iv = oracle.segment_intervals(W.CUBIC, b.seg_pts[(l - 1) // 2], 1.0, math.pi / 2)
            assert n == iv["N"]
        else:
            assert n == 1


def test_counts_never_grow_with_tau():
    b = W.c2_batching(n_paths=60, canvas=512)
    prev = oracle.tessellate(b)["link_nrib"]
    for tau in (0.01, 0.05, 0.25, 1.0, 4.0):
        cur = oracle.tessellate(b, tau=tau)["link_nrib"]
        assert (cur <= prev).all()
        prev = cur
    assert prev.sum() < oracle.tessellate(b)["link_nrib"].sum()
