"""Pins of the oracle's raster (O2), brute-force distance (O3) and dasher."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W

LINE, QUAD, CUBIC, CONIC = 0, 1, 2, 3


def _strip(quads_per_path):
    """Rib stream from lists of rib lists per path (each inner list one link)."""
    ribs, tags = [], []
    for p, links in enumerate(quads_per_path):
        for link in links:
            for j, r in enumerate(link):
                ribs.append(r)
                tags.append((p << 2) | (1 if j == 0 else 0) | 2)
    return np.array(ribs, np.float64), np.array(tags, np.uint32)


def _samples(Wd, Ht):
    return oracle.sample_positions(Wd, Ht)  # [H, W, 16, 2]


def _popcount16(a):
    a = a.astype(np.int64)
    return sum(((a >> k) & 1).sum() for k in range(16))


def test_raster_axis_aligned_rectangles_count_exactly():
    rng = np.random.default_rng(0)
    Wd, Ht = 24, 20
    S = _samples(Wd, Ht)
    for _ in range(40):
        x0, x1 = np.sort(rng.integers(-256, 256 * (Wd + 1), 2)) / 256.0
        y0, y1 = np.sort(rng.integers(-256, 256 * (Ht + 1), 2)) / 256.0
        if x1 == x0 or y1 == y0:
            continue
        # one quad: N0=(x0,y0) P0=(x0,y1) N1=(x1,y0) P1=(x1,y1)
        rib, tag = _strip([[[[x0, y0, x0, y1], [x1, y0, x1, y1]]]])
        canvas, cov = oracle.raster(rib, tag, Wd, Ht, 1)
        inside = (S[..., 0] >= x0) & (S[..., 0] <= x1) & (S[..., 1] >= y0) & (S[..., 1] <= y1)
        assert int(cov[0]) == int(inside.sum())
        bits = np.zeros((Ht, Wd), np.int64)
        for k in range(16):
            bits |= inside[..., k].astype(np.int64) << k
        assert np.array_equal(canvas.astype(np.int64), bits)


def _inside_exact(tri, px, py):
    """Closed-triangle membership with exact rational barycentric coordinates."""
    (ax, ay), (bx, by), (cx, cy) = tri
    det = (bx - ax) * (cy - ay) - (cx - ax) * (by - ay)
    if det == 0:
        return False
    l1 = Fraction((px - ax) * (cy - ay) - (cx - ax) * (py - ay), det)
    l2 = Fraction((bx - ax) * (py - ay) - (px - ax) * (by - ay), det)
    return l1 >= 0 and l2 >= 0 and l1 + l2 <= 1


def test_raster_triangles_match_exact_barycentric():
    rng = np.random.default_rng(1)
    Wd, Ht = 8, 8
    for it in range(30):
        v = rng.integers(-64, 256 * 8 + 64, (4, 2))  # in 1/256 px
        # quad (N0,P0,N1,P1) -> triangles (N0,P0,P1), (N0,P1,N1)
        N0, P0, N1, P1 = v
        rib, tag = _strip([[[np.r_[N0, P0] / 256.0, np.r_[N1, P1] / 256.0]]])
        canvas, cov = oracle.raster(rib, tag, Wd, Ht, 1)
        tris = [(N0, P0, P1), (N0, P1, N1)]
        count = 0
        for y in range(Ht):
            for x in range(Wd):
                m = 0
                for k in range(16):
                    sx, sy = 256 * x + 16 * k + 8, 256 * y + 16 * ((5 * k) % 16) + 8
                    if any(_inside_exact([tuple(map(int, p)) for p in t], sx, sy) for t in tris):
                        m |= 1 << k
                assert int(canvas[y, x]) == m
                count += bin(m).count("1")
        assert int(cov[0]) == count


def test_raster_union_within_path_sum_across_paths():
    sq = [[1.0, 1.0, 1.0, 3.0], [3.0, 1.0, 3.0, 3.0]]
    # the same square twice in one path (two links) counts once; in two paths twice
    rib, tag = _strip([[sq, sq]])
    c1, cov1 = oracle.raster(rib, tag, 6, 6, 1)
    rib2, tag2 = _strip([[sq], [sq]])
    c2, cov2 = oracle.raster(rib2, tag2, 6, 6, 2)
    assert np.array_equal(c1, c2)
    assert int(cov2.sum()) == 2 * int(cov1[0]) and int(cov2[0]) == int(cov1[0])
    assert int(cov1[0]) == _popcount16(c1)


def test_distance_to_line_and_circle_closed_forms():
    b = W.single(LINE, [[2, 3], [2, 3], [10, 7], [10, 7]])
    d = oracle.centreline_distance(b, 12, 10, n_dense=200)
    S = _samples(12, 10)
    A, D = np.array([2.0, 3.0]), np.array([10.0, 7.0])
    u = D - A
    t = np.clip(((S - A) @ u) / (u @ u), 0, 1)
    exp = np.hypot(*(S - (A + t[..., None] * u)).transpose(3, 0, 1, 2))
    assert np.abs(d - exp).max() < 1e-9
    R = 6.0
    b = W.single(CONIC, [[R, 0], [R, R], [R, R], [0, R]], w=math.cos(math.pi / 4))
    d = oracle.centreline_distance(b, 8, 8, n_dense=400)
    S = _samples(8, 8)
    ang = np.arctan2(S[..., 1], S[..., 0])
    radial = np.abs(np.hypot(S[..., 0], S[..., 1]) - R)
    sel = (ang > 0.05) & (ang < math.pi / 2 - 0.05) & (radial < 1.5)
    assert np.abs(d[sel] - radial[sel]).max() < 1e-5  # FP32 weight: circle to ~1e-6 R


def _coverage_case(name):
    if name == "cusp":
        return W.single(CUBIC, np.array([[4, 4], [36, 36], [4, 36], [36, 4]]), width=5, dtheta_deg=4)
    if name == "loop":
        return W.single(CUBIC, np.array([[6, 10], [46, 40], [-4, 40], [36, 10]]), width=4, dtheta_deg=3)
    if name == "chain":
        rng = np.random.default_rng(4)
        pts = rng.uniform(6, 34, (3, 4, 2))
        pts[1:, 0] = pts[:-1, 3]
        return W.single([CUBIC] * 3, pts, width=3, dtheta_deg=2)
    if name == "mixed":
        pts = [[[5, 5], [5, 5], [25, 8], [25, 8]],
               [[25, 8], [35, 20], [35, 20], [20, 30]],
               [[20, 30], [8, 36], [8, 36], [6, 20]]]
        return W.single([LINE, CONIC, QUAD], pts, w=[1, 2.5, 1], width=6, dtheta_deg=2)
    if name == "wide_tight":  # w/2 larger than the radius of curvature: offset cusps
        return W.single(CUBIC, np.array([[8, 8], [40, 30], [0, 30], [32, 8]]), width=14, dtheta_deg=2)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["cusp", "loop", "chain", "mixed", "wide_tight"])
def test_coverage_of_round_strokes_matches_brute_force(name):
    """O2 on the oracle's own ribs agrees with O3 (distance <= w/2) on every sample
    farther than eps from the boundary, eps = the polygon's chord bound plus the
    8-bit snapping error."""
    b = _coverage_case(name)
    Wd = Ht = 40
    o = oracle.tessellate(b)
    rib32 = o["rib"].astype(np.float32).astype(np.float64)
    canvas, cov = oracle.raster(rib32, o["tag"], Wd, Ht, 1)
    d = oracle.centreline_distance(b, Wd, Ht, n_dense=1500)
    r = 0.5 * float(b.path_width[0])
    # chord bound: between ribs the tangent turns <= q, so boundary edges of length c
    # sit within (c/2) tan(q/2) of the true offset curve; plus snapping (sqrt(2)/512)
    e = np.diff(rib32.reshape(-1, 2, 2), axis=0)
    c = np.hypot(e[..., 0], e[..., 1]).max()
    eps = 0.5 * c * math.tan(b.dtheta / 2) + math.sqrt(2) / 512 + 1e-6
    bits = np.stack([(canvas >> k) & 1 for k in range(16)], axis=-1).astype(bool)
    inside = d <= r
    far = np.abs(d - r) > eps
    bad = (bits != inside) & far
    assert far.sum() > 0.9 * far.size
    assert not bad.any(), f"{bad.sum()} samples disagree beyond eps={eps:.4f}"
    assert int(cov[0]) == int(bits.sum())


def test_dash_straight_line_pieces():
    b = W.single(LINE, [[0, 0], [0, 0], [100, 0], [100, 0]], width=2, cap=W.CAP_BUTT)
    o = oracle.tessellate(b)
    for pattern, offset, expect in [
        ([12, 6], 0.0, [(0, 12), (18, 30), (36, 48), (54, 66), (72, 84), (90, 100)]),
        ([12, 6], 5.0, [(0, 7), (13, 25), (31, 43), (49, 61), (67, 79), (85, 97)]),
        ([10], 0.0, [(0, 10), (20, 30), (40, 50), (60, 70), (80, 90)]),  # odd count repeats
        ([5, 5, 20, 10], 0.0, [(0, 5), (10, 30), (40, 45), (50, 70), (80, 85), (90, 100)]),
    ]:
        dd = oracle.dash(o["rib"], o["s"], o["tag"], pattern, offset)
        got = [(dd["s"][i], dd["s"][i + 1]) for i in range(0, len(dd["s"]), 2)]
        assert np.allclose(got, expect, atol=1e-12), (pattern, offset, got)
        for i, (a, e) in enumerate(got):
            assert np.allclose(dd["rib"][2 * i], [a, -1, a, 1], atol=1e-12)
            assert np.allclose(dd["rib"][2 * i + 1], [e, -1, e, 1], atol=1e-12)
        assert np.all(dd["tag"][0::2] & 1) and not np.any(dd["tag"][1::2] & 1)


def test_dash_keeps_zero_length_quads_only_when_on():
    # 90 degree bevel join at s = 10: on for pattern [12, 6]; off for [8, 4]
    pts = [[[0, 0], [0, 0], [10, 0], [10, 0]], [[10, 0], [10, 0], [10, 10], [10, 10]]]
    b = W.single([LINE, LINE], pts, width=2, join=W.JOIN_BEVEL, cap=W.CAP_BUTT)
    o = oracle.tessellate(b)
    seg = (o["tag"] & 2) != 0
    on = oracle.dash(o["rib"], o["s"], o["tag"], [12, 6])
    off = oracle.dash(o["rib"], o["s"], o["tag"], [8, 4])
    join_on = [i for i in range(0, len(on["src"]), 2) if not seg[on["src"][i]]]
    join_off = [i for i in range(0, len(off["src"]), 2) if not seg[off["src"][i]]]
    assert len(join_on) == 1 and len(join_off) == 0
