"""Failure detection on the GPU without a fault: every inter-CTA wait of the
library is bounded.  The self-check makes one of those waits run out (its
predecessor's flag is never set) and the kernel must come back with
PS_ERR_TIMEOUT in the status word, leaving the context usable: the next
tessellation on it matches the oracle's counts on
every link the oracle does not flag fragile."""
import time

import numpy as np
import pytest

import oracle
from paper_2007_00308_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_gives_up_and_reports(which):
    import torch
    import paper_2007_00308_gb300 as ps
    ctx = ps.Context()
    assert ctx.status() == ps.PS_OK
    t0 = time.perf_counter()
    ps.ps_check_wait_timeout(ctx, which)
    elapsed = time.perf_counter() - t0
    assert ctx.status() == ps.PS_ERR_TIMEOUT
    assert ctx.status() == ps.PS_OK  # read-and-clear
    print("wait", which, "gave up after", round(elapsed, 2), "s")
    assert elapsed < 60
    with pytest.raises(ps.PolarStrokeError):
        ps.ps_check_wait_timeout(ctx, 2)
    b = W.c1_plain_small()
    db = ps.DeviceBatch(b)
    out = ps.tessellate(ctx, db, ps.PS_PREC_MIXED, arclength=True)
    torch.cuda.synchronize()
    assert ctx.status() == ps.PS_OK
    o = oracle.tessellate(b)
    lo = out.link_rib_off.cpu().numpy().astype(np.int64)
    firm = (o["link_info"] & oracle.FRAGILE64) == 0
    assert np.array_equal(np.diff(lo)[firm], o["link_nrib"][firm])
