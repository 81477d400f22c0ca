"""SVG elliptical arcs as conic segments (host function of the library, no GPU).

Pinned by geometry the converter must reproduce, not by its own formulas: the
pieces chain exactly from the start to the end point with continuous tangents,
every point of every piece lies on one ellipse with the given axis ratio and
rotation (centre and scale fitted here), the pieces turn the
way the sweep flag says and span more than half the ellipse iff the large-arc
flag is set, and the quarter circle is the textbook conic."""
import math

import numpy as np
import pytest

import oracle
import paper_2007_00308_gb300 as ps
from paper_2007_00308_gb300 import workloads as W


def eval_conic(A, B, D, w, t):
    t = np.asarray(t, np.float64)[:, None]
    u = 1 - t
    A, B, D = (np.asarray(p, np.float64) for p in (A, B, D))
    return (u * u * A + 2 * u * t * w * B + t * t * D) / (u * u + 2 * u * t * w + t * t)


def test_quarter_circle_is_the_textbook_conic():
    pts, w = ps.svg_arc_to_conics(100, 0, 100, 100, 0, 0, 1, 0, 100)
    assert pts.shape == (1, 4, 2)
    assert np.allclose(pts[0], [[100, 0], [100, 100], [100, 100], [0, 100]], atol=1e-4)
    assert w[0] == pytest.approx(math.cos(math.pi / 4), abs=1e-7)


def test_degenerate_inputs():
    pts, w = ps.svg_arc_to_conics(5, 5, 10, 20, 30, 0, 1, 5, 5)
    assert len(w) == 0
    pts, w = ps.svg_arc_to_conics(0, 0, 0, 20, 30, 1, 1, 10, 4)
    assert len(w) == 1 and w[0] == 1.0
    assert np.allclose(pts[0], [[0, 0], [5, 2], [5, 2], [10, 4]])
    with pytest.raises(ps.PolarStrokeError):
        ps.svg_arc_to_conics(0, 0, float("nan"), 20, 30, 1, 1, 10, 4)


def _fit_ellipse(P, rx, ry, phi):
    """In the ellipse's own axes with y scaled by rx / ry the points lie on a circle
    of radius s rx: fit it linearly (x^2 + y^2 + a x + b y + c = 0).  Returns the
    scale s and the largest relative radial residual."""
    c, s = math.cos(phi), math.sin(phi)
    x = c * P[:, 0] + s * P[:, 1]
    y = (-s * P[:, 0] + c * P[:, 1]) * (rx / ry)
    M = np.c_[x, y, np.ones_like(x)]
    sol, *_ = np.linalg.lstsq(M, -(x * x + y * y), rcond=None)
    cx, cy = -sol[0] / 2, -sol[1] / 2
    r = math.sqrt(cx * cx + cy * cy - sol[2])
    d = np.hypot(x - cx, y - cy)
    return r / rx, np.abs(d / r - 1).max()


@pytest.mark.parametrize("seed", range(12))
def test_random_arcs_lie_on_one_ellipse(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(8):
        x0, y0, x1, y1 = rng.uniform(-200, 200, 4)
        rx, ry = rng.uniform(5, 250, 2)
        phi_deg = rng.uniform(-180, 180)
        large, sweep = rng.integers(0, 2, 2)
        pts, w = ps.svg_arc_to_conics(x0, y0, rx, ry, phi_deg, large, sweep, x1, y1)
        n = len(w)
        assert 1 <= n <= 4
        p64 = pts.astype(np.float64)
        assert np.array_equal(pts[0, 0], np.float32([x0, y0]))
        assert np.array_equal(pts[-1, 3], np.float32([x1, y1]))
        for i in range(n - 1):
            assert np.array_equal(pts[i, 3], pts[i + 1, 0])
            t_end = p64[i, 3] - p64[i, 1]
            t_start = p64[i + 1, 1] - p64[i + 1, 0]
            cr = t_end[0] * t_start[1] - t_end[1] * t_start[0]
            assert abs(cr) <= 1e-5 * np.linalg.norm(t_end) * np.linalg.norm(t_start)
            assert t_end @ t_start > 0
        assert (w >= math.cos(math.pi / 4) - 1e-6).all() and (w <= 1).all()
        # all points on one ellipse of the given axis ratio and rotation
        P = np.concatenate([eval_conic(p64[i, 0], p64[i, 1], p64[i, 3], float(w[i]),
                                       np.linspace(0, 1, 9)) for i in range(n)])
        s, err = _fit_ellipse(P, rx, ry, math.radians(phi_deg))
        scale = min(rx, ry) * s
        assert err < 2e-6 * (1 + max(abs(x0), abs(y0), abs(x1), abs(y1)) / scale)
        assert s > 1 - 1e-5
        # turning direction from the sweep flag (y up: sweep 1 turns counter-clockwise)
        turn = 0.0
        for i in range(n):
            a, b = p64[i, 1] - p64[i, 0], p64[i, 3] - p64[i, 1]
            turn += math.atan2(a[0] * b[1] - a[1] * b[0], a @ b)
        assert (turn > 0) == bool(sweep)
        span = float(np.sum(2 * np.arccos(np.clip(w.astype(np.float64), -1, 1))))
        if s > 1 + 1e-4:  # radii scaled up: exactly half the ellipse
            assert span == pytest.approx(math.pi, abs=1e-4)
        else:
            assert (span > math.pi) == bool(large)


def test_arc_path_strokes_like_its_circle():
    """A full circle from two half-circle arcs, stroked by the oracle: every rib is
    at radius R +- w/2 from the centre."""
    R = 50.0
    segs, ws = [], []
    for (a, b) in (((R, 0), (-R, 0)), ((-R, 0), (R, 0))):
        pts, w = ps.svg_arc_to_conics(a[0], a[1], R, R, 0, 0, 1, b[0], b[1])
        segs += [p.tolist() for p in pts]
        ws += [float(v) for v in w]
    b = W.single([W.CONIC] * len(segs), segs, w=ws, width=6, join=W.JOIN_ROUND, closed=1,
                 dtheta_deg=2.0)
    o = oracle.tessellate(b)
    r = np.hypot(o["rib"][:, 0::2], o["rib"][:, 1::2])
    seg = (o["tag"] >> 1) & 1
    r = r[seg == 1]
    assert np.abs(np.sort(r, axis=1) - [R - 3, R + 3]).max() < 1e-4
