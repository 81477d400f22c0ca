"""Autotuner host logic (no GPU): coordinate descent, the JSON cache, signatures.
The GPU test checks that every tuning gives identical outputs."""
import json

import numpy as np
import pytest

import paper_2007_00308_gb300 as ps
from paper_2007_00308_gb300 import autotune as AT
from paper_2007_00308_gb300 import workloads as W


class FakeCtx:
    """Stands in for ps.Context: the tunables only."""

    def __init__(self):
        self.t = {ps.PS_TUNE_EMIT_SLABS: 32, ps.PS_TUNE_SETUP_LINKS: 2, ps.PS_TUNE_BIN_BLOCKS: 0}
        self.reserved = []

    def set_tuning(self, k, v):
        assert v in ps.TUNE_CANDIDATES[k]
        self.t[k] = v

    def get_tuning(self, k):
        return self.t[k]

    def reserve(self, **kw):
        self.reserved.append(kw)


def _cost(ctx):
    # separable bowl with its minimum at (8, 4, 4)
    e, s, b = (ctx.t[ps.PS_TUNE_EMIT_SLABS], ctx.t[ps.PS_TUNE_SETUP_LINKS],
               ctx.t[ps.PS_TUNE_BIN_BLOCKS])
    return 10.0 + abs(np.log2(e) - 3) + abs(s - 4) * 0.5 + abs(b - 4) * 0.25


def test_coordinate_descent_finds_the_minimum():
    ctx = FakeCtx()
    res = AT.tune(ctx, step=lambda: None, timer=lambda: _cost(ctx), reps=3)
    assert res["params"] == {"emit_slabs": 8, "setup_links": 4, "bin_blocks": 4}
    assert res["ms"] == pytest.approx(10.0)
    assert res["default_ms"] > res["ms"]
    n_cand = sum(len(v) for v in ps.TUNE_CANDIDATES.values())
    assert n_cand <= len(res["trials"]) <= 3 * n_cand


def test_cache_round_trip_and_apply(tmp_path):
    path = str(tmp_path / "tune.json")
    ctx = FakeCtx()
    calls = []

    def timer():
        calls.append(1)
        return _cost(ctx)

    r1 = AT.tuned(ctx, lambda: None, "dev|k", cache_path=path, timer=timer, reps=2)
    assert not r1["cached"]
    n1 = len(calls)
    data = json.load(open(path))
    assert data["dev|k"]["params"] == r1["params"]
    ctx2 = FakeCtx()
    r2 = AT.tuned(ctx2, lambda: None, "dev|k", cache_path=path, timer=timer, reps=2)
    assert r2["cached"] and len(calls) == n1
    assert AT.current(ctx2) == r1["params"]
    # a damaged cache entry is re-tuned, not trusted
    data["dev|k"]["params"].pop("bin_blocks")
    json.dump(data, open(path, "w"))
    r3 = AT.tuned(FakeCtx(), lambda: None, "dev|k", cache_path=path, timer=timer, reps=2)
    assert not r3["cached"]


def test_signature_buckets_sizes():
    a = AT.signature("GB300", 295431, 10000, 43024706, (2048, 2048))
    b = AT.signature("GB300", 300000, 10100, 44000000, (2048, 2048))
    c = AT.signature("GB300", 600000, 10000, 43024706, (2048, 2048))
    assert a == b and a != c


def test_reserve_bins_adds_headroom():
    ctx = FakeCtx()
    n = AT.reserve_bins(ctx, 16384, 1000000)
    assert n >= 1050000 and ctx.reserved[-1] == {"n_tile": 16384, "n_pair": n}


@pytest.mark.gpu
def test_every_tuning_gives_identical_outputs():
    import torch
    b = W.c2_batching(n_paths=150)
    ctx = ps.Context()
    db = ps.DeviceBatch(b)
    R = ps.ps_count_ribs_sync(ctx, db, ps.TessOutput(db.n_link, db.n_path, 0, arclength=False),
                              ps.PS_PREC_MIXED)
    out = ps.TessOutput(db.n_link, db.n_path, R, arclength=True)
    canvas = torch.zeros((2048, 2048), dtype=torch.int16, device="cuda")
    cov = torch.zeros(b.n_path, dtype=torch.int64, device="cuda")

    def run():
        ps.ps_tessellate_strokes(ctx, db, out, ps.PS_PREC_MIXED, ps.PS_TESS_ARCLENGTH)
        ps.ps_rasterize_coverage(ctx, out.rib, out.tag, out.n_rib, out.capacity, b.n_path, 2048,
                                 2048, canvas, cov)
        torch.cuda.synchronize()
        assert ctx.status() == 0
        return (out.rib[:R].clone(), out.tag[:R].clone(), out.s[:R].clone(), canvas.clone(),
                cov.clone())

    ref = run()
    for key, cands in ps.TUNE_CANDIDATES.items():
        for v in cands:
            ctx.set_tuning(key, v)
            got = run()
            for a, g in zip(ref, got):
                assert torch.equal(a, g), (ps.TUNE_NAMES[key], v)
        ctx.set_tuning(key, {ps.PS_TUNE_EMIT_SLABS: 16, ps.PS_TUNE_SETUP_LINKS: 2,
                             ps.PS_TUNE_BIN_BLOCKS: 0}[key])
    with pytest.raises(ps.PolarStrokeError):
        ctx.set_tuning(ps.PS_TUNE_EMIT_SLABS, 5)
    with pytest.raises(ps.PolarStrokeError):
        ctx.set_tuning(99, 1)


def test_each_tunable_is_judged_by_its_own_kernels():
    """With per-kernel samples, a tunable is chosen by its kernels' time even
    when the whole step's time (here: noise that favours other values) says
    otherwise."""
    ctx = FakeCtx()
    rng = np.random.default_rng(0)

    def timer():
        e, s, b = (ctx.t[ps.PS_TUNE_EMIT_SLABS], ctx.t[ps.PS_TUNE_SETUP_LINKS],
                   ctx.t[ps.PS_TUNE_BIN_BLOCKS])
        k = {"k_emit": 1.0 + 0.1 * abs(np.log2(e) - 5), "k_link_setup": 0.4 + 0.1 * abs(s - 2),
             "k_bin_count": 1.0 + 0.05 * abs(b - 2), "k_bin_scatter": 1.0 + 0.05 * abs(b - 2)}
        k["step"] = 20.0 + sum(k.values()) + float(rng.uniform(-1.0, 1.0))
        return k

    res = AT.tune(ctx, step=lambda: None, timer=timer, reps=3)
    assert res["params"] == {"emit_slabs": 32, "setup_links": 2, "bin_blocks": 2}
