"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every check is a closed form, an
invariant stated in the paper, a finite-difference / dense-sampling measurement
written independently in numpy, or a brute-force predicate.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
LINE, QUAD, CUBIC, CONIC = 0, 1, 2, 3


def q32(deg):
    return float(np.float32(math.radians(deg)))


STEP_SNAP = 1e-4  # reading R13: a ratio within 1e-4 step above an integer rounds down


def ceil_ratio(angle, q):
    return max(1, int(math.ceil(angle / q - STEP_SNAP)))


def bezier_eval(kind, pts, w, t):
    """Table 1 generator curves, written directly with numpy for measurements."""
    t = np.asarray(t, np.float64)[:, None]
    u = 1 - t
    A, B, C, D = (np.asarray(p, np.float64) for p in pts)
    if kind == CUBIC:
        return u**3 * A + 3 * u**2 * t * B + 3 * u * t**2 * C + t**3 * D
    if kind == QUAD:
        return u**2 * A + 2 * u * t * B + t**2 * D
    if kind == CONIC:
        return (u**2 * A + 2 * u * t * w * B + t**2 * D) / (u**2 + 2 * u * t * w + t**2)
    return u * A + t * D


def random_segment(rng, kind):
    pts = rng.uniform(0, 100, (4, 2)).astype(np.float32)
    w = float(np.float32(math.exp(rng.uniform(math.log(0.1), math.log(10))))) if kind == CONIC else 1.0
    if kind in (QUAD, CONIC):
        pts[2] = pts[1]
    return pts, w


# ---- derivative formulas against finite differences -----------------------------
@pytest.mark.parametrize("kind", [LINE, QUAD, CUBIC, CONIC])
def test_hodograph_matches_finite_difference(kind):
    rng = np.random.default_rng(1 + kind)
    for _ in range(20):
        pts, w = random_segment(rng, kind)
        ts = np.linspace(0.02, 0.98, 25)
        h = 1e-6
        fd = (bezier_eval(kind, pts, w, ts + h) - bezier_eval(kind, pts, w, ts - h)) / (2 * h)
        H = oracle.probe(kind, pts, w, 1, ts)
        c = oracle.probe(kind, pts, w, 3, ts)[:, 0]
        g = oracle.probe(kind, pts, w, 0, ts)
        assert np.allclose(g, bezier_eval(kind, pts, w, ts), rtol=0, atol=1e-10)
        assert np.all(c > 0)
        scale = np.abs(fd).max() + 1e-12
        assert np.abs(c[:, None] * H - fd).max() < 1e-6 * scale
        # H' against a finite difference of H
        Hp = oracle.probe(kind, pts, w, 1, ts + h)
        Hm = oracle.probe(kind, pts, w, 1, ts - h)
        Hd = oracle.probe(kind, pts, w, 2, ts)
        assert np.abs(Hd - (Hp - Hm) / (2 * h)).max() < 1e-5 * (np.abs(Hd).max() + 1)


@pytest.mark.parametrize("kind", [QUAD, CUBIC, CONIC])
def test_curvature_sign_polynomial(kind):
    """C(t) is a positive multiple of g'(t) x g''(t) (the curvature's numerator)."""
    rng = np.random.default_rng(11 + kind)
    for _ in range(20):
        pts, w = random_segment(rng, kind)
        ts = np.linspace(0.01, 0.99, 33)
        h = 1e-5
        g0 = bezier_eval(kind, pts, w, ts)
        gp = bezier_eval(kind, pts, w, ts + h)
        gm = bezier_eval(kind, pts, w, ts - h)
        d1 = (gp - gm) / (2 * h)
        d2 = (gp - 2 * g0 + gm) / (h * h)
        kap = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
        C = oracle.probe(kind, pts, w, 4, ts)[:, 0]
        c = oracle.probe(kind, pts, w, 3, ts)[:, 0]  # g' = c H, so g' x g'' = c^2 H x H'
        big = np.abs(kap) > 1e-3 * np.abs(kap).max()
        assert np.all(np.sign(C[big]) == np.sign(kap[big]))
        ratio = kap[big] / (C[big] * c[big] ** 2)
        assert ratio.min() > 0 and ratio.max() / ratio.min() < 1 + 1e-3


# ---- line: exactly one quad (Sec. 4.2.1) ----------------------------------------
def test_line_single_quad():
    b = W.single(LINE, [[0, 0], [0, 0], [30, 40], [30, 40]], width=4, cap=W.CAP_BUTT)
    o = oracle.tessellate(b)
    assert len(o["s"]) == 2
    n = np.array([-0.8, 0.6])  # <-sin psi, cos psi> of direction (0.6, 0.8)
    A, D = np.array([0.0, 0.0]), np.array([30.0, 40.0])
    exp = np.array([np.r_[A - 2 * n, A + 2 * n], np.r_[D - 2 * n, D + 2 * n]])
    assert np.abs(o["rib"] - exp).max() < 1e-12
    assert o["s"][-1] == pytest.approx(50.0, abs=1e-12)
    assert o["path_len"][0] == pytest.approx(50.0, abs=1e-12)


# ---- circle-arc conic: closed forms ------------------------------------------------
@pytest.mark.parametrize("deg", [0.5, 1.0, 2.0, 3.0, 7.0])
def test_circle_arc_conic(deg):
    R, width = 100.0, 8.0
    w = math.cos(math.pi / 4)  # quarter circle: w_B = cos(half the arc)
    b = W.single(CONIC, [[R, 0], [R, R], [R, R], [0, R]], w=w, width=width, cap=W.CAP_BUTT,
                 dtheta_deg=deg)
    o = oracle.tessellate(b)
    q = b.dtheta
    N = len(o["s"]) - 1
    assert N == ceil_ratio(math.pi / 2, q)
    # FP32 rounding of w_B perturbs the circle by ~3e-7 relative
    tol = 1e-6 * R
    rN = np.hypot(o["rib"][:, 0], o["rib"][:, 1])
    rP = np.hypot(o["rib"][:, 2], o["rib"][:, 3])
    assert np.abs(rN - (R + width / 2)).max() < tol  # N side is outside (right of travel)
    assert np.abs(rP - (R - width / 2)).max() < tol
    # uniform tangent steps put the ribs at uniform polar angles
    ang = np.arctan2(o["rib"][:, 1], o["rib"][:, 0])
    assert np.abs(ang - np.arange(N + 1) * (math.pi / 2) / N).max() < 1e-6
    # arc length: N chords of a circle, biased low (Sec. 7)
    s_exact = 2 * R * N * math.sin((math.pi / 2) / (2 * N))
    assert o["path_len"][0] == pytest.approx(s_exact, rel=1e-6)
    assert o["path_len"][0] < math.pi * R / 2


def test_arc_length_converges_quadratically():
    R = 100.0
    errs = []
    for deg in (4.0, 2.0, 1.0):
        b = W.single(CONIC, [[R, 0], [R, R], [R, R], [0, R]], w=math.cos(math.pi / 4), width=2,
                     cap=W.CAP_BUTT, dtheta_deg=deg)
        errs.append(math.pi * R / 2 - oracle.tessellate(b)["path_len"][0])
    assert errs[0] > errs[1] > errs[2] > 0
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def _gauss_legendre_length(kind, pts, w, n=4000):
    x, wt = np.polynomial.legendre.leggauss(64)
    total = 0.0
    edges = np.linspace(0, 1, n + 1)
    h = 1e-7
    for a, b_ in zip(edges[:-1], edges[1:]):
        t = 0.5 * (b_ - a) * x + 0.5 * (a + b_)
        d = (bezier_eval(kind, pts, w, t + h) - bezier_eval(kind, pts, w, t - h)) / (2 * h)
        total += 0.5 * (b_ - a) * np.sum(wt * np.hypot(d[:, 0], d[:, 1]))
    return total


def test_arc_length_below_integral_and_close():
    rng = np.random.default_rng(5)
    for _ in range(6):
        pts, w = random_segment(rng, CUBIC)
        b = W.single(CUBIC, pts, width=1, cap=W.CAP_BUTT, dtheta_deg=1.0)
        s = oracle.tessellate(b)["path_len"][0]
        L = _gauss_legendre_length(CUBIC, pts, w, n=200)
        assert s <= L + 1e-7
        assert (L - s) / L < 1e-3


# ---- parabola: tangent turn between the control-polygon legs ---------------------
def test_parabola_turning_and_angles():
    rng = np.random.default_rng(7)
    for _ in range(30):
        pts, _ = random_segment(rng, QUAD)
        A, B, D = pts[0].astype(float), pts[1].astype(float), pts[3].astype(float)
        u, v = B - A, D - B
        turn = abs(math.atan2(u[0] * v[1] - u[1] * v[0], np.dot(u, v)))
        q = q32(2.0)
        I = oracle.segment_intervals(QUAD, pts, 1.0, q)
        if abs(turn / q - round(turn / q)) < 1e-6:
            continue
        assert I["M"] == 1
        assert I["N"] == ceil_ratio(turn, q)


# ---- exact cusp: the paper's cusp chart structure (Sec. 6.2) -------------------------
def _golden_cusp():
    rows = []
    with open(os.path.join(HERE, "golden", "cusp_chart.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("row", _golden_cusp())
def test_exact_cusp_chart(row):
    qdeg, N, j0, j1 = row
    pts = [[0, 0], [1, 1], [0, 1], [1, 0]]
    q = q32(qdeg)
    I = oracle.segment_intervals(CUBIC, pts, 1.0, q)
    assert I["M"] == 2
    assert np.allclose(I["p"], [0, 0.5, 1], atol=1e-15)
    assert np.allclose(np.degrees(I["delta"]), [135, 135], atol=1e-12)
    assert I["N"] == int(N)
    b = W.single(CUBIC, pts, width=0.2, cap=W.CAP_BUTT, dtheta_deg=qdeg)
    o = oracle.tessellate(b)
    at_half = np.where(np.abs(o["t"] - 0.5) < 1e-9)[0]
    others = np.abs(o["t"] - 0.5)[np.abs(o["t"] - 0.5) >= 1e-9]
    assert others.min() > 1e-4  # the band is unambiguous
    assert at_half.min() == int(j0) and at_half.max() == int(j1)
    assert len(at_half) == int(j1 - j0 + 1)
    psi = np.degrees(o["psi"][at_half])
    # the fan's normals sweep (almost) 180 degrees about the cusp point
    assert psi.max() - psi.min() > 180 - 2 * qdeg
    # all of its ribs are centred on g(1/2)
    mid = 0.5 * (o["rib"][at_half, :2] + o["rib"][at_half, 2:])
    assert np.abs(mid - [0.5, 0.75]).max() < 1e-12


# ---- per-step invariants ----------------------------------------------------------
def _segment_ribs(o):
    """Yield (lo, hi) rib ranges of segment links."""
    tag = o["tag"]
    starts = np.where(tag & 1)[0]
    ends = np.r_[starts[1:], len(tag)]
    for a, b in zip(starts, ends):
        if tag[a] & 2:
            yield a, b


@pytest.mark.parametrize("kind", [QUAD, CUBIC, CONIC])
def test_step_turn_bounded_and_tangent_matches(kind):
    rng = np.random.default_rng(21 + kind)
    q = q32(3.0)
    for _ in range(25):
        pts, w = random_segment(rng, kind)
        b = W.single(kind, pts, w=w, width=1, cap=W.CAP_BUTT, dtheta_deg=3.0)
        o = oracle.tessellate(b)
        for a, e in _segment_ribs(o):
            dpsi = np.angle(np.exp(1j * np.diff(o["psi"][a:e])))
            assert np.all(np.abs(dpsi) <= q * (1 + STEP_SNAP + 1e-12))
            # at every rib whose t is interior to its interval the curve's tangent
            # points along psi(j)
            t = o["t"][a:e]
            H = oracle.probe(kind, pts, w, 1, t)
            good = np.hypot(H[:, 0], H[:, 1]) > 1e-6 * np.abs(H).max()
            ang = np.arctan2(H[good, 1], H[good, 0])
            diff = np.angle(np.exp(1j * (ang - o["psi"][a:e][good])))
            assert np.abs(diff).max() < 1e-9


def _dense_total_turning(kind, pts, w, n=400001):
    t = np.linspace(0, 1, n)
    h = 1e-7
    d = (bezier_eval(kind, pts, w, np.clip(t + h, 0, 1)) - bezier_eval(kind, pts, w, np.clip(t - h, 0, 1)))
    a = np.unwrap(np.arctan2(d[:, 1], d[:, 0]))
    return np.abs(np.diff(a)).sum()


@pytest.mark.parametrize("case", ["loop", "serpentine2", "random", "conic", "external_ellipse"])
def test_total_turning_matches_dense_sampling(case):
    rng = np.random.default_rng(3)
    if case == "loop":
        segs = [(CUBIC, np.array([[0, 0], [150, 100], [-50, 100], [100, 0]], np.float32), 1.0)]
    elif case == "serpentine2":
        segs = [(CUBIC, np.array([[86, 54], [30, 42], [3, 12], [67, 65]], np.float32), 1.0)]
    elif case == "random":
        segs = [(CUBIC, random_segment(rng, CUBIC)[0], 1.0) for _ in range(10)]
    elif case == "conic":
        segs = [(CONIC,) + random_segment(rng, CONIC) for _ in range(10)]
    else:
        segs = [(CONIC, np.array([[0, 0], [50, 50], [50, 50], [100, 0]], np.float32), -0.5)]
    q = q32(1.0)
    for kind, pts, w in segs:
        I = oracle.segment_intervals(kind, pts, w, q)
        tot = np.abs(I["delta"]).sum()
        assert tot == pytest.approx(_dense_total_turning(kind, pts, w), abs=1e-4)
        assert np.all(np.abs(I["delta"]) < math.pi)   # split halves (Sec. 3.3.5)
        assert tot < 2 * math.pi                       # hodograph bound (Sec. 3.3.5)
        assert I["M"] <= 6


def test_serpentine_with_two_inflections_has_three_intervals():
    pts = np.array([[86, 54], [30, 42], [3, 12], [67, 65]], np.float32)
    I = oracle.segment_intervals(CUBIC, pts, 1.0, q32(1.0))
    # two sign changes of g' x g'' in (0,1): measure independently
    t = np.linspace(1e-4, 1 - 1e-4, 100001)
    h = 1e-5
    g0 = bezier_eval(CUBIC, pts, 1, t)
    d1 = (bezier_eval(CUBIC, pts, 1, t + h) - bezier_eval(CUBIC, pts, 1, t - h)) / (2 * h)
    d2 = (bezier_eval(CUBIC, pts, 1, t + h) - 2 * g0 + bezier_eval(CUBIC, pts, 1, t - h)) / h**2
    k = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    flips = t[np.where(np.diff(np.sign(k)) != 0)[0]]
    assert len(flips) == 2
    assert I["M"] == 3
    assert np.allclose(I["p"][1:3], flips, atol=2e-5)


# ---- chord error and facet angles (Sec. 4.2) -------------------------------------------
def test_chord_error_bound():
    """Between consecutive ribs the tangent turns by at most q, so the curve stays
    within (c/2) tan(q/2) of the chord of length c."""
    rng = np.random.default_rng(9)
    q = q32(2.0)
    for _ in range(10):
        pts, w = random_segment(rng, CUBIC)
        b = W.single(CUBIC, pts, width=1, cap=W.CAP_BUTT, dtheta_deg=2.0)
        o = oracle.tessellate(b)
        t = o["t"]
        for j in range(1, len(t)):
            if t[j] <= t[j - 1]:
                continue
            ts = np.linspace(t[j - 1], t[j], 50)
            c = bezier_eval(CUBIC, pts, w, ts)
            a, e = c[0], c[-1]
            L = np.hypot(*(e - a))
            if L < 1e-9:
                continue
            nrm = np.array([-(e - a)[1], (e - a)[0]]) / L
            dev = np.abs((c - a) @ nrm).max()
            assert dev <= 0.5 * L * math.tan(q / 2) + 1e-9


def test_ordinary_facet_angles_below_2q():
    """Sec. 4.2: ordinary facet angles of the offset boundary are < 2q.  With w/2
    well below the radius of curvature every facet is ordinary."""
    rng = np.random.default_rng(13)
    q = q32(4.0)
    checked = 0
    for _ in range(20):
        pts, w = random_segment(rng, CUBIC)
        b = W.single(CUBIC, pts, width=0.02, cap=W.CAP_BUTT, dtheta_deg=4.0)
        o = oracle.tessellate(b)
        rho = o["rho"][1:-1]
        if (rho[rho > 0] < 1.0).any():
            continue
        for side in (slice(0, 2), slice(2, 4)):
            v = o["rib"][:, side]
            e = np.diff(v, axis=0)
            ln = np.hypot(e[:, 0], e[:, 1])
            ok = ln > 1e-9
            e = e[ok]
            ang = np.arctan2(e[:, 1], e[:, 0])
            facet = np.abs(np.angle(np.exp(1j * np.diff(ang))))
            assert facet.max() < 2 * q
            checked += len(facet)
    assert checked > 100


# ---- joins and caps (Sec. 4.3) -------------------------------------------------------
def _two_lines(turn_deg, join, miter=4.0, width=2.0, dtheta_deg=2.0):
    a = math.radians(turn_deg)
    pts = [[[0, 0], [0, 0], [10, 0], [10, 0]],
           [[10, 0], [10, 0], [10 + 10 * math.cos(a), 10 * math.sin(a)],
            [10 + 10 * math.cos(a), 10 * math.sin(a)]]]
    return W.single([LINE, LINE], pts, width=width, join=join, cap=W.CAP_BUTT,
                    dtheta_deg=dtheta_deg, miter=miter)


def _link_ribs(o, link):
    off = o["link_rib_off"]
    return o["rib"][off[link]:off[link + 1]]


@pytest.mark.parametrize("turn", [30.0, 90.0, -90.0, 150.0, -170.0])
def test_round_join(turn):
    b = _two_lines(turn, W.JOIN_ROUND)
    o = oracle.tessellate(b)
    q = b.dtheta
    J = ceil_ratio(abs(math.radians(turn)), q)
    ribs = _link_ribs(o, 2)
    assert len(ribs) == J + 1
    at = np.array([10.0, 0.0])
    outer, inner = (ribs[:, :2], ribs[:, 2:]) if turn > 0 else (ribs[:, 2:], ribs[:, :2])
    assert np.abs(np.hypot(*(outer - at).T) - 1.0).max() < 1e-12
    assert np.abs(inner - at).max() < 1e-12
    # the outer side is the gap: for a left turn it is on the right of travel (y < 0 side)
    mid = outer[J // 2] - at
    bis = np.array([math.cos(math.radians(turn) / 2), math.sin(math.radians(turn) / 2)])
    right = np.array([bis[1], -bis[0]])
    assert np.dot(mid, right if turn > 0 else -right) > 0.99


def test_join_counts_and_bevel_triangle_miter():
    for style, J in [(W.JOIN_NONE, 0), (W.JOIN_BEVEL, 1), (W.JOIN_TRIANGLE, 2), (W.JOIN_MITER, 3),
                     (W.JOIN_MITER_TRUNCATE, 3)]:
        o = oracle.tessellate(_two_lines(90.0, style))
        assert o["link_nrib"][2] == (J + 1 if J else 0)
    # tangent-continuous: no join region
    o = oracle.tessellate(_two_lines(0.0, W.JOIN_ROUND))
    assert o["link_nrib"][2] == 0
    # miter accepted for a 90 degree left turn: tip at (10 + r, -r)
    o = oracle.tessellate(_two_lines(90.0, W.JOIN_MITER, miter=4.0))
    ribs = _link_ribs(o, 2)
    assert np.allclose(ribs[1, :2], [11, -1], atol=1e-12) and np.allclose(ribs[2, :2], [11, -1], atol=1e-12)
    assert np.allclose(ribs[0, :2], [10, -1], atol=1e-12) and np.allclose(ribs[3, :2], [11, 0], atol=1e-12)
    # miter ratio 1/sin(45) = 1.414 > 1.2: revert to bevel (ribs 1,2 copy the end ribs)
    o = oracle.tessellate(_two_lines(90.0, W.JOIN_MITER, miter=1.2))
    ribs = _link_ribs(o, 2)
    assert np.allclose(ribs[1, :2], ribs[0, :2]) and np.allclose(ribs[2, :2], ribs[3, :2])
    # truncate: clip points at distance limit * r along the bisector
    o = oracle.tessellate(_two_lines(90.0, W.JOIN_MITER_TRUNCATE, miter=1.2))
    ribs = _link_ribs(o, 2)
    bis = np.array([1, -1]) / math.sqrt(2)
    for v in (ribs[1, :2], ribs[2, :2]):
        assert np.dot(v - [10, 0], bis) == pytest.approx(float(np.float32(1.2)), abs=1e-12)
    # right turn: outer side is P; bevel
    o = oracle.tessellate(_two_lines(-90.0, W.JOIN_BEVEL))
    ribs = _link_ribs(o, 2)
    assert np.allclose(ribs[:, :2], [10, 0]) and np.allclose(ribs[:, 2:], [[10, 1], [11, 0]])
    # triangular join: middle rib on the bisector at r
    o = oracle.tessellate(_two_lines(90.0, W.JOIN_TRIANGLE))
    ribs = _link_ribs(o, 2)
    assert np.allclose(ribs[1, :2], np.array([10, 0]) + bis, atol=1e-12)


@pytest.mark.parametrize("cap,J", [(W.CAP_BUTT, 0), (W.CAP_TRIANGLE, 2), (W.CAP_SQUARE, 4),
                                   (W.CAP_ROUND, None)])
def test_caps(cap, J):
    b = W.single(LINE, [[0, 0], [0, 0], [10, 0], [10, 0]], width=2, cap=cap, dtheta_deg=2.0)
    o = oracle.tessellate(b)
    if J is None:
        J = ceil_ratio(math.pi, b.dtheta)
    assert o["link_nrib"][0] == (J + 1 if J else 0) and o["link_nrib"][2] == (J + 1 if J else 0)
    if not J:
        return
    start, stop = _link_ribs(o, 0), _link_ribs(o, 2)
    # caps sweep the N side from the left offset, around the end, to the right offset
    assert np.allclose(start[0, :2], [0, 1]) and np.allclose(start[-1, :2], [0, -1])
    assert np.allclose(stop[0, :2], [10, -1]) and np.allclose(stop[-1, :2], [10, 1])
    assert np.allclose(start[:, 2:], [0, 0]) and np.allclose(stop[:, 2:], [10, 0])
    if J % 2 == 0:
        mid_s, mid_e = start[J // 2, :2], stop[J // 2, :2]
        assert np.allclose(mid_s, [-1, 0], atol=1e-12) and np.allclose(mid_e, [11, 0], atol=1e-12)
    else:  # the cap reaches r behind / ahead to within the step's sagitta
        q = b.dtheta
        assert -1 - 1e-12 <= start[:, 0].min() <= -math.cos(q / 2) + 1e-12
        assert 11 + 1e-12 >= stop[:, 0].max() >= 10 + math.cos(q / 2) - 1e-12
    if cap == W.CAP_SQUARE:
        assert np.allclose(start[1, :2], [-1, 1], atol=1e-12) and np.allclose(start[3, :2], [-1, -1], atol=1e-12)
        assert np.allclose(stop[1, :2], [11, -1], atol=1e-12) and np.allclose(stop[3, :2], [11, 1], atol=1e-12)
    if cap == W.CAP_ROUND:
        assert np.abs(np.hypot(*(start[:, :2]).T) - 1).max() < 1e-12


def test_zero_length_segment_is_dropped():
    pts = [[[0, 0], [0, 0], [10, 0], [10, 0]], [[10, 0], [10, 0], [10, 0], [10, 0]],
           [[10, 0], [10, 0], [10, 10], [10, 10]]]
    b = W.single([LINE, CUBIC, LINE], pts, width=2, join=W.JOIN_BEVEL, cap=W.CAP_BUTT)
    o = oracle.tessellate(b)
    # links: cap, L, join(0->1), C0, join(1->2), L, cap
    assert list(o["link_nrib"]) == [0, 2, 0, 0, 2, 2, 0]


def test_collinear_backtracking_cubic_pivots():
    """Collinear control points with a reversal: a flat piece, a +pi pivot at the
    reversal t, a flat piece (reading R5); its coverage reaches past D."""
    pts = np.array([[0, 0], [30, 0], [-10, 0], [10, 0]], np.float32)
    I = oracle.segment_intervals(CUBIC, pts, 1.0, q32(2.0))
    assert I["pivot"].sum() >= 1
    assert np.allclose(np.abs(I["delta"][I["pivot"] == 1]), math.pi)
    b = W.single(CUBIC, pts, width=2, cap=W.CAP_BUTT, dtheta_deg=2.0)
    o = oracle.tessellate(b)
    xs = 0.5 * (o["rib"][:, 0] + o["rib"][:, 2])
    # the curve's x-extent from dense sampling
    c = bezier_eval(CUBIC, pts, 1, np.linspace(0, 1, 100001))
    assert xs.max() == pytest.approx(c[:, 0].max(), abs=1e-9)
    assert xs.min() == pytest.approx(c[:, 0].min(), abs=1e-9)


def test_miter_ratio_uses_interior_angle():
    """60 degree turn: interior angle 120, miter ratio 1/sin(60) = 1.1547 <= 1.5, so the
    miter is kept, tip at r * ratio along the outer bisector."""
    o = oracle.tessellate(_two_lines(60.0, W.JOIN_MITER, miter=1.5))
    ribs = _link_ribs(o, 2)
    a = math.radians(30.0)
    bis = np.array([math.sin(a), -math.cos(a)])  # outer (right-hand) bisector normal
    tip = np.array([10.0, 0.0]) + bis / math.cos(a)
    assert np.allclose(ribs[1, :2], tip, atol=1e-12) and np.allclose(ribs[2, :2], tip, atol=1e-12)
    o = oracle.tessellate(_two_lines(60.0, W.JOIN_MITER, miter=1.1))
    ribs = _link_ribs(o, 2)
    assert np.allclose(ribs[1, :2], ribs[0, :2]) and np.allclose(ribs[2, :2], ribs[3, :2])


@pytest.mark.parametrize("kind,pts,w", [
    (CUBIC, [[0, 0], [0, 0], [10, 10], [20, 0]], 1.0),       # B = A: start along C - A
    (CUBIC, [[0, 0], [0, 0], [0, 0], [20, 5]], 1.0),         # B = C = A: along D - A
    (CUBIC, [[0, 0], [10, 10], [20, 0], [20, 0]], 1.0),      # C = D: end along D - B
    (CUBIC, [[0, 0], [20, 5], [20, 5], [20, 5]], 1.0),       # B = C = D: end along D - A
    (QUAD, [[0, 0], [0, 0], [0, 0], [20, 5]], 1.0),          # B = A
    (QUAD, [[0, 0], [20, 5], [20, 5], [20, 5]], 1.0),        # B = D
    (CONIC, [[0, 0], [10, 10], [10, 10], [20, 0]], -0.5),    # negative weight flips
    (CONIC, [[0, 0], [10, 10], [10, 10], [20, 0]], 3.0),
])
def test_end_gradients_are_one_sided_limits(kind, pts, w):
    """Table 1's normalized end gradients equal the one-sided limits of g'/|g'|."""
    pts = np.array(pts, np.float32)
    I = oracle.segment_intervals(kind, pts, w, q32(1.0))
    # where g' vanishes at an end the chord is second order in h, so the chord
    # direction converges like O(h); h = 1e-5 keeps rounding far below that
    h = 1e-5
    g = lambda t: bezier_eval(kind, pts, w, np.array([t]))[0]
    d0 = g(h) - g(0.0)
    d1 = g(1.0) - g(1.0 - h)
    a0, a1 = math.atan2(d0[1], d0[0]), math.atan2(d1[1], d1[0])
    assert abs(np.angle(np.exp(1j * (I["Psi"][0] - a0)))) < 1e-3
    assert abs(np.angle(np.exp(1j * (I["Psi"][-1] - a1)))) < 1e-3


@pytest.mark.parametrize("pts,n_pivot", [
    ([[0, 0], [30, 0], [-10, 0], [10, 0]], 2),   # forward, back past A, forward past D
    ([[0, 0], [10, 0], [0, 0], [10, 0]], 0),     # A B A B: g' touches zero at t=1/2 (kink)
    ([[0, 0], [20, 0], [10, 0], [10, 0]], 1),    # C = D: one reversal inside, root at t=1 excluded
    ([[0, 0], [0, 0], [20, 0], [10, 0]], 1),     # B = A: root at t=0 excluded
])
def test_collinear_reversal_count(pts, n_pivot):
    """The number of direction reversals of a collinear cubic, measured from the sign
    changes of g'(t) . (D - A) on a dense grid."""
    pts = np.array(pts, np.float32)
    I = oracle.segment_intervals(CUBIC, pts, 1.0, q32(2.0))
    assert int(I["pivot"].sum()) == n_pivot
    t = np.linspace(1e-6, 1 - 1e-6, 200001)
    h = 1e-7
    d = (bezier_eval(CUBIC, pts, 1, t + h) - bezier_eval(CUBIC, pts, 1, t - h))[:, 0]
    sgn = np.sign(d[np.abs(d) > 1e-12])
    assert int((np.diff(sgn) != 0).sum()) == n_pivot
