"""The seeded input generators against the recipes they state (CPU): sizes,
form mix, distributions' ranges, the 1/64-px grid, exact cusp constructions and
chaining, and determinism per seed."""
import math

import numpy as np

from paper_2007_00308_gb300 import workloads as W


def _chained(b):
    off = b.path_seg_off.astype(np.int64)
    for p in range(len(off) - 1):
        s0, s1 = off[p], off[p + 1]
        if s1 - s0 > 1 and not np.array_equal(b.seg_pts[s0 + 1:s1, 0], b.seg_pts[s0:s1 - 1, 3]):
            return False
    return True


def test_generators_are_deterministic_per_seed():
    a, b = W.c2_batching(n_paths=300), W.c2_batching(n_paths=300)
    for f in ("seg_type", "seg_pts", "seg_w", "path_seg_off", "path_width", "path_join",
              "path_cap"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    c = W.c2_batching(n_paths=300, seed=W.SEED_BASE + 99)
    assert not np.array_equal(a.seg_pts[:10], c.seg_pts[:10])


def test_c2_recipe():
    b = W.c2_batching(n_paths=3000)
    counts = np.diff(b.path_seg_off)
    assert counts.min() >= 1 and counts.max() <= 200
    assert 26.0 < counts.mean() < 34.0  # Geometric(1/30), redrawn above 200
    t = b.seg_type
    frac = [np.mean(t == k) for k in (W.LINE, W.QUAD, W.CUBIC, W.CONIC)]
    for f, want in zip(frac, (0.20, 0.20, 0.45, 0.15)):
        assert abs(f - want) < 0.02
    wc = b.seg_w[t == W.CONIC]
    assert wc.min() >= 0.1 * (1 - 1e-6) and wc.max() <= 10.0 * (1 + 1e-6)
    p = b.seg_pts.astype(np.float64)
    ends = p[:, [0, 3]]  # the walk's steps bounce off the canvas; control points may leave it
    assert ends.min() >= 0.0 and ends.max() <= 2048.0
    assert np.array_equal(p * 64, np.round(p * 64))  # the 1/64-px grid
    assert _chained(b)
    # exact cusps: C + D = A + B on the grid (so g'(1/2) = 0), for about 10% of cubics
    cub = p[t == W.CUBIC]
    cusp = np.all(cub[:, 2] + cub[:, 3] == cub[:, 0] + cub[:, 1], axis=1) & \
        np.any(cub[:, 3] != cub[:, 0], axis=1)
    assert 0.08 < cusp.mean() < 0.12
    assert b.path_width.min() >= 0.5 * (1 - 1e-6) and b.path_width.max() <= 64.0 * (1 + 1e-6)
    assert set(np.unique(b.path_join)) <= {W.JOIN_MITER, W.JOIN_ROUND, W.JOIN_BEVEL}
    assert set(np.unique(b.path_cap)) <= {W.CAP_BUTT, W.CAP_SQUARE, W.CAP_ROUND}
    assert math.isclose(float(b.dtheta), math.radians(1.0), rel_tol=1e-6)
    assert tuple(b.canvas) == (2048, 2048)


def test_c1_c3_c5_recipes():
    c1 = W.c1_plain_small()
    assert len(c1.seg_type) == 64 and np.all(c1.seg_type == W.CUBIC) and len(c1.path_width) == 1
    assert float(c1.path_width[0]) == 8.0 and _chained(c1)
    assert math.isclose(float(c1.dtheta), math.radians(2.0), rel_tol=1e-6)
    assert c1.seg_pts.min() >= 0 and c1.seg_pts.max() <= 512  # every point uniform in the canvas

    c3 = W.c3_large_path()
    assert len(c3.seg_type) == 5031 and len(c3.path_width) == 1 and _chained(c3)
    assert float(c3.path_width[0]) == 2.0 and c3.dash == ([12.0, 6.0], 0.0)
    assert math.isclose(float(c3.dtheta), math.radians(0.5), rel_tol=1e-6)
    ends = c3.seg_pts[:, [0, 3]]
    assert ends.min() >= 0 and ends.max() <= 4096

    c5 = W.c5_differentiation(n_paths=16)
    assert np.all(np.diff(c5.path_seg_off) == 32) and _chained(c5)
    assert c5.path_width.min() >= 1 and c5.path_width.max() <= 16
    assert c5.seg_pts.min() >= 0 and c5.seg_pts.max() <= 1024


def test_c4_recipe():
    n = 2000
    b = W.c4_precision(n=n)
    assert len(b.seg_type) == n and len(b.path_width) == n and np.all(b.seg_type == W.CUBIC)
    p = b.seg_pts.astype(np.float64)
    assert np.abs(p).max() <= 1e6 + 4e3
    size = np.linalg.norm(p[:, 3] - p[:, 0], axis=1)
    # near-cusp half: C + D - A - B stays within the perturbations (relative 1e-2 at most)
    dev = np.linalg.norm(p[:, 2] + p[:, 3] - p[:, 0] - p[:, 1], axis=1)
    half = n // 2
    assert np.all(dev[:half] <= 0.1 * size[:half] + 1e-3 * np.abs(p[:half]).max(axis=(1, 2)))
    # near-collinear half: B and C within the perturbations of the line A D
    d = p[half:, 3] - p[half:, 0]
    nrm = np.stack([-d[:, 1], d[:, 0]], 1) / np.linalg.norm(d, axis=1)[:, None]
    off = np.abs(np.einsum("ij,ij->i", p[half:, 1] - p[half:, 0], nrm))
    assert np.all(off <= 0.1 * size[half:] + 1e-3 * np.abs(p[half:]).max(axis=(1, 2)))
