"""Failure detection on the GPU without a fault: a bounded wait that nothing completes gives up,
is reported as GWAS_ERR_TIMEOUT, and the context stays usable for the next scan."""
import numpy as np
import pytest

import synth
from oracle import gls
from gpu_util import run, max_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    assert torch.cuda.is_available()
    import paper_1207_2169_gb300 as g
    return g


def test_bounded_wait_gives_up_and_context_survives(g):
    import time
    t0 = time.perf_counter()
    st = g.gwas_selftest_timeout(0, 300)
    dt = time.perf_counter() - t0
    assert st == -7, g.gwas_last_error()
    assert 0.25 < dt < 10.0, dt
    # the device still runs the scan path correctly afterwards
    c = synth.small_problem(71, n=200, q=3, m=300, t=4)
    Bref, Wref, Vref = gls.gls_grid(c.Phi, c.XL, c.XR, c.Y, c.h2, c.s2)
    B, W, _ = run(g, c, "eig", "split_bf16")
    eb, ew = max_errors(B, W, Bref, Wref, Vref)
    assert eb < 1e-4 and ew < 1e-4


def test_sync_reports_no_timeout_after_clean_scans(g):
    import torch
    c = synth.small_problem(72, n=150, q=2, m=200, t=1)
    h = g.gwas_setup(c.Phi, c.XL, c.Y, c.h2, c.s2, precision="split_bf16")
    try:
        G = g.gwas_pack_genotypes(torch.from_numpy(np.ascontiguousarray(c.XR)).cuda())
        B = torch.empty((c.m, 1, c.p), device="cuda")
        g.gwas_scan_packed(h, G, B)
        g.gwas_sync(h)  # raises on a timeout
    finally:
        g.gwas_destroy(h)
