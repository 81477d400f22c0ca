"""Oracle pins for the Sec. 8.1 comparison: uniform parametric ribs and facet
angles (reading R17: the angle where one quad's boundary edge meets the next;
ordinary when each edge points between the tangents of its end ribs, which
leaves out the facets next to offset cusps)."""
import math

import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W

C, Q, K = W.CUBIC, W.QUAD, W.CONIC


def seg_runs(o):
    """(start, end) rib ranges of the segment links of a tessellation."""
    off = o["link_rib_off"]
    seg = (o["tag"] >> 1) & 1
    out = []
    for l in range(len(off) - 1):
        a, b = off[l], off[l + 1]
        if b > a and seg[a]:
            out.append((a, b))
    return out


def test_polar_facets_of_a_circle_equal_the_step():
    R = 100.0
    b = W.single(K, [[R, 0], [R, R], [R, R], [0, R]], w=math.cos(math.pi / 4), width=10,
                 cap=W.CAP_BUTT, dtheta_deg=1.0)
    o = oracle.tessellate(b)
    N = len(o["s"]) - 1
    ang, ordn = oracle.facet_angles(o["rib"])
    inner = ang[1:-1]
    assert ordn[1:-1].all()
    assert np.abs(inner - (math.pi / 2) / N).max() < 1e-7


def test_uniform_parabola_facets_match_the_midpoint_tangents():
    """The chord of a parabola between t_a and t_b is parallel to g'((t_a + t_b)/2),
    so with zero width the facet at rib j is the angle between g'((j - 1/2)/N) and
    g'((j + 1/2)/N)."""
    A, B, D = np.array([0.0, 0.0]), np.array([60.0, 140.0]), np.array([150.0, 10.0])
    N = 37
    rib = oracle.uniform_ribs(Q, [A, B, B, D], 1.0, N, 0.0)
    t = np.arange(N + 1) / N
    g = ((1 - t) ** 2)[:, None] * A + (2 * (1 - t) * t)[:, None] * B + (t ** 2)[:, None] * D
    assert np.abs(rib[:, 0:2] - g).max() < 1e-12 and np.abs(rib[:, 2:4] - g).max() < 1e-12
    ang, ordn = oracle.facet_angles(rib)
    tm = (np.arange(N) + 0.5) / N
    H = (1 - tm)[:, None] * (B - A) + tm[:, None] * (D - B)
    h = np.arctan2(H[:, 1], H[:, 0])
    exp = np.abs(np.angle(np.exp(1j * (h[1:] - h[:-1]))))
    assert ordn[1:-1].all()
    assert np.abs(ang[1:-1, 0] - exp).max() < 1e-12
    assert np.abs(ang[1:-1, 1] - exp).max() < 1e-12


def test_uniform_ribs_geometry():
    """Rib j is centred on g(j/N), has length w and is perpendicular to g'(j/N)."""
    rng = np.random.default_rng(3)
    for kind in (Q, C, K):
        pts = np.float32(rng.uniform(0, 200, (4, 2))).astype(np.float64)  # probe takes FP32
        if kind != C:
            pts[2] = pts[1]
        w = float(np.float32(0.6)) if kind == K else 1.0
        rib = oracle.uniform_ribs(kind, pts, w, 25, 8.0)
        t = np.arange(26) / 25
        g = oracle.probe(kind, pts, w, 0, t)
        H = oracle.probe(kind, pts, w, 1, t)
        mid = 0.5 * (rib[:, 0:2] + rib[:, 2:4])
        d = rib[:, 2:4] - rib[:, 0:2]
        assert np.abs(mid - g).max() < 1e-9 * (1 + np.abs(g).max())
        assert np.abs(np.hypot(d[:, 0], d[:, 1]) - 8.0).max() < 1e-9
        cosang = np.abs((d * H).sum(1)) / (np.hypot(*d.T) * np.hypot(*H.T))
        assert cosang.max() < 1e-9
        # N = g - r n lies right of the direction of travel, P left of it
        assert ((H[:, 0] * d[:, 1] - H[:, 1] * d[:, 0]) > 0).all()


@pytest.mark.parametrize("deg", [1.0, 4.0])
@pytest.mark.parametrize("width", [2.0, 30.0, 100.0])
def test_polar_ordinary_facets_below_twice_the_step(deg, width):
    """Sec. 4.2: ordinary facet angles stay below 2q."""
    rng = np.random.default_rng(int(deg * 100 + width))
    q = math.radians(deg)
    worst = 0.0
    for _ in range(30):
        pts = rng.uniform(0, 300, (4, 2))
        b = W.single(C, pts, width=width, cap=W.CAP_BUTT, dtheta_deg=deg)
        o = oracle.tessellate(b)
        for a, e in seg_runs(o):
            ang, ordn = oracle.facet_angles(o["rib"][a:e])
            if ordn.any():
                worst = max(worst, ang[ordn].max())
    assert worst < 2 * q


def test_polar_beats_uniform_on_a_serpentine():
    """Sec. 8.1's comparison on a serpentine cubic at q = 4 deg, w = 100, equal quad
    counts: polar stroking's largest ordinary facet angle and its spread are the
    smaller ones."""
    pts = [[0, 0], [250, 400], [150, -300], [400, 100]]
    b = W.single(C, pts, width=100, cap=W.CAP_BUTT, dtheta_deg=4.0)
    o = oracle.tessellate(b)
    (a, e), = seg_runs(o)
    n_quads = e - a - 1
    pa, po = oracle.facet_angles(o["rib"][a:e])
    ua, uo = oracle.facet_angles(oracle.uniform_ribs(C, pts, 1.0, n_quads, 100.0))
    p, u = pa[po], ua[uo]
    assert len(p) > 0 and len(u) > 0
    assert p.max() < u.max()
    assert p.std() < u.std()
