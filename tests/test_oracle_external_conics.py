"""Oracle pins for conics with negative weight (Sec. 3.3.3, reading R15).

An external ellipse (-1 < w_B < 0) is the complementary arc of the ellipse its
control polygon spans with the weight -w_B: bounded, no tangent reversal, and a
total turning of 2 pi minus the positive-weight arc's.  w_B = 0 is the segment
A-D.  For w_B <= -1 the rational denominator vanishes inside [0, 1] and the
curve passes through infinity; the oracle rejects such segments."""
import math

import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W

K = W.CONIC
STEP_SNAP = 1e-4


def ceil_ratio(angle, q):
    return max(1, int(math.ceil(angle / q - STEP_SNAP)))


def conic(pts, w, t):
    t = np.asarray(t, np.float64)[:, None]
    u = 1 - t
    A, B, D = (np.asarray(p, np.float64) for p in (pts[0], pts[1], pts[3]))
    return (u**2 * A + 2 * u * t * w * B + t**2 * D) / (u**2 + 2 * u * t * w + t**2)


@pytest.mark.parametrize("deg", [2.0, 1.0, 0.5])
def test_external_circle_arc(deg):
    """A = (R, 0), B = (R, R), D = (0, R) with w_B = -cos(pi/4) is the 270-degree arc of
    the radius-R circle that the quarter arc (w_B = +cos(pi/4)) leaves out."""
    R, width = 100.0, 8.0
    w = -math.cos(math.pi / 4)
    b = W.single(K, [[R, 0], [R, R], [R, R], [0, R]], w=w, width=width, cap=W.CAP_BUTT,
                 dtheta_deg=deg)
    o = oracle.tessellate(b)
    q = b.dtheta
    N = len(o["s"]) - 1
    # one interval of 3 pi / 2 turning, split at its middle into two of 3 pi / 4
    assert N == 2 * ceil_ratio(3 * math.pi / 4, q)
    tol = 1e-6 * R
    rN = np.hypot(o["rib"][:, 0], o["rib"][:, 1])
    rP = np.hypot(o["rib"][:, 2], o["rib"][:, 3])
    # the travel is clockwise, so the N side (g - r n) is the inner one
    assert np.abs(rN - (R - width / 2)).max() < tol
    assert np.abs(rP - (R + width / 2)).max() < tol
    # uniform tangent steps on a circle are uniform polar steps, clockwise from 0
    ang = np.unwrap(np.arctan2(o["rib"][:, 1], o["rib"][:, 0]))
    assert np.abs(ang - (-np.arange(N + 1) * (1.5 * math.pi) / N)).max() < 1e-6
    s_exact = 2 * R * N * math.sin((1.5 * math.pi) / (2 * N))
    assert o["path_len"][0] == pytest.approx(s_exact, rel=1e-6)
    assert o["path_len"][0] < 1.5 * math.pi * R


def test_external_conic_turning_and_ribs():
    """Random external ellipses: the intervals' turning adds up to 2 pi minus the
    control polygon's turning angle, every step turns at most q, and each rib is
    centred on the curve at its t with half-width w/2 along the curve normal."""
    rng = np.random.default_rng(7)
    q = float(np.float32(math.radians(1.0)))
    for _ in range(40):
        pts = np.float32(rng.uniform(0, 200, (3, 2))).astype(np.float64)  # FP32 inputs
        w = -float(np.exp(rng.uniform(math.log(0.02), math.log(0.98))))
        P4 = [pts[0], pts[1], pts[1], pts[2]]
        d0, d1 = pts[1] - pts[0], pts[2] - pts[1]
        theta = abs(math.atan2(d0[0] * d1[1] - d0[1] * d1[0], d0 @ d1))
        iv = oracle.segment_intervals(K, P4, w=1.0, dtheta=q)
        ivn = oracle.segment_intervals(K, P4, w=np.float32(w), dtheta=q)
        turn = float(np.abs(ivn["delta"]).sum())
        assert turn == pytest.approx(2 * math.pi - theta, abs=1e-9)
        assert all(abs(d) < math.pi + 1e-12 for d in ivn["delta"])  # split keeps each < pi
        assert abs(float(np.abs(iv["delta"]).sum()) - theta) < 1e-9
        b = W.single(K, P4, w=w, width=6, cap=W.CAP_BUTT, dtheta_deg=1.0)
        o = oracle.tessellate(b)
        ww = float(np.float32(w))
        P32 = np.float32(P4).astype(np.float64)
        g = conic(P32, ww, o["t"])
        mid = 0.5 * (o["rib"][:, 0:2] + o["rib"][:, 2:4])
        assert np.abs(mid - g).max() < 1e-7 * (1 + np.abs(g).max())
        half = 0.5 * np.hypot(*(o["rib"][:, 2:4] - o["rib"][:, 0:2]).T)
        assert np.abs(half - 3.0).max() < 1e-9
        # consecutive rib normals turn by at most q (uniform tangent steps)
        nrm = o["rib"][:, 2:4] - o["rib"][:, 0:2]
        a = np.unwrap(np.arctan2(nrm[:, 1], nrm[:, 0]))
        assert np.abs(np.diff(a)).max() <= q * (1 + 1e-4) + 1e-9


def test_conic_weight_zero_is_the_segment_a_d():
    b = W.single(K, [[0, 0], [30, 80], [30, 80], [100, 20]], w=0.0, width=4, cap=W.CAP_BUTT)
    o = oracle.tessellate(b)
    assert len(o["s"]) == 2  # one flat interval: one quad
    d = np.array([100.0, 20.0]) / math.hypot(100.0, 20.0)
    n = np.array([-d[1], d[0]])
    exp = np.array([[*(-2 * n), *(2 * n)], [*(np.array([100, 20]) - 2 * n),
                                            *(np.array([100, 20]) + 2 * n)]])
    assert np.abs(o["rib"] - exp).max() < 1e-12
    assert o["path_len"][0] == pytest.approx(math.hypot(100, 20), rel=1e-15)


@pytest.mark.parametrize("w", [-1.0, -1.5, -4.0])
def test_external_parabola_and_hyperbola_rejected(w):
    b = W.single(K, [[0, 0], [50, 60], [50, 60], [100, 0]], w=w, width=4)
    with pytest.raises(oracle.OracleError):
        oracle.tessellate(b)


@pytest.mark.parametrize("w", [-1.0, -1.25, -3.0, -20.0])
def test_corrected_reversal_parameter(w):
    """The denominator (1-t)^2 + 2 w (1-t) t + t^2 vanishes at
    t = 1/2 +- sqrt(w^2 - 1) / (2 (1 - w)) (reading R15), and the printed form
    (-2 +- 2 sqrt(w^2 - 1)) / (4 w - 4) does not give its roots."""
    def den(t):
        return (1 - t) ** 2 + 2 * w * (1 - t) * t + t ** 2
    r = math.sqrt(w * w - 1) / (2 * (1 - w))
    for t in (0.5 - r, 0.5 + r):
        assert 0.0 <= t <= 1.0
        assert abs(den(t)) < 1e-12
    roots = np.roots([2 - 2 * w, 2 * w - 2, 1])
    assert np.allclose(sorted(roots.real), [0.5 - r, 0.5 + r], atol=1e-12)
    printed = (-2 + 2 * math.sqrt(w * w - 1)) / (4 * w - 4)
    assert abs(den(printed)) > 1e-3
