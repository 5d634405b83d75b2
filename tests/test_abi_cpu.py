"""The C-ABI library loads and exports what include/gwas.h declares; argument checks (CPU only).

No call here reaches a CUDA compute path: argument validation runs before any device work.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))


@pytest.fixture(scope="module")
def g():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1207_2169_gb300 as g
    return g


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gwas_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(g):
    declared = _declared()
    assert declared, "no declarations parsed"
    out = subprocess.run(["nm", "-D", "--defined-only", g.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gwas_[a-z0-9_]+)", out))
    assert declared <= exported, declared - exported
    assert set(g.EXPORTS) == declared
    for name in declared:
        assert hasattr(g.lib, name)


def test_default_options(g):
    o = g.gwas_default_options()
    assert (o.algo, o.precision, o.block_snps, o.validate_genotypes, o.device) == (0, 2, 0, 0, 0)
    assert (o.out_mode, o.genetic_model) == (0, 0)


def test_destroy_null_is_noop(g):
    g.lib.gwas_destroy(None)


@pytest.mark.parametrize("case", ["n0", "q0", "q8", "t0", "h2_one", "h2_neg", "s2_zero", "algo", "prec",
                                  "model"])
def test_setup_rejects_bad_arguments(g, case):
    n, q, t = 6, 2, 2
    Phi = np.eye(n); XL = np.ones((n, q)); Y = np.zeros((n, t))
    h2 = np.full(t, 0.5); s2 = np.ones(t)
    opt = g.gwas_default_options()
    nn, qq, tt = n, q, t
    if case == "n0": nn = 0
    if case == "q0": qq = 0
    if case == "q8": qq = 8
    if case == "t0": tt = 0
    if case == "h2_one": h2[1] = 1.0
    if case == "h2_neg": h2[0] = -0.1
    if case == "s2_zero": s2[0] = 0.0
    if case == "algo": opt.algo = 7
    if case == "prec": opt.precision = 9
    if case == "model": opt.genetic_model = 7
    XLb = np.ones((n, 8))
    out = ctypes.c_void_p(123)
    st = g.lib.gwas_setup(Phi.ctypes.data, nn, XLb.ctypes.data, qq, Y.ctypes.data, tt,
                          h2.ctypes.data, s2.ctypes.data, ctypes.byref(opt), ctypes.byref(out))
    assert st == -1, (case, st, g.gwas_last_error())
    assert out.value is None
    assert g.gwas_last_error() != ""


def test_setup_null_pointers(g):
    out = ctypes.c_void_p()
    assert g.lib.gwas_setup(None, 4, None, 1, None, 1, None, None, None, ctypes.byref(out)) == -1
    assert g.lib.gwas_setup(None, 4, None, 1, None, 1, None, None, None, None) == -1


def test_null_handle_calls(g):
    assert g.lib.gwas_scan(None, None, 10, 1, None, None, 1, None) == -1
    assert g.lib.gwas_scan_f64(None, None, 10, 1, None, None, 1, None) == -1
    # the allocation-free entry point checks its handle before anything else, even for m = 0
    assert g.lib.gwas_scan_static(None, None, 10, None, None, None) == -1
    assert g.lib.gwas_scan_static(None, None, 0, None, None, None) == -1
    assert g.lib.gwas_singular_count(None) == -1
    ms = ctypes.c_double()
    assert g.lib.gwas_setup_timing(None, ctypes.byref(ms)) == -1
    assert g.lib.gwas_info(None, None, None, None, None, None) == -1
    assert g.lib.gwas_genetic_columns(None) == -1
    assert g.lib.gwas_split_pieces(None) == -1
    assert g.lib.gwas_fp8_traits(None) == -1
    assert g.lib.gwas_eig_chunk(None) == -1
    assert g.lib.gwas_chol_routed_traits(None) == -1
    assert g.lib.gwas_batch_tuning(None, None, None, None) == -1
    assert g.lib.gwas_stream_info(None, None, None, None, None, None, None) == -1
    assert g.lib.gwas_stage_timing(None, 1) == -1
    ms8 = (ctypes.c_double * 8)()
    assert g.lib.gwas_stage_times(None, ms8, None) == -1


def _decode_packed(G, n):
    """Reads genotype k of each row from byte k // 4, bits 2 (k % 4) .. +1 (the documented
    layout), one genotype at a time."""
    m = G.shape[0]
    out = np.zeros((m, n), np.int64)
    for k in range(n):
        out[:, k] = (G[:, k // 4].astype(np.int64) >> (2 * (k % 4))) & 3
    return out


def test_packed_row_bytes(g):
    assert [g.gwas_packed_row_bytes(n) for n in (0, 1, 63, 64, 65, 1000, 16384)] == \
        [0, 16, 16, 16, 32, 256, 4096]


@pytest.mark.parametrize("n", [1, 7, 64, 97, 130])
def test_host_packing_layout(g, n):
    rs = np.random.default_rng(n)
    X = rs.integers(0, 3, size=(37, n)).astype(np.int8)
    G = g.gwas_pack_genotypes(X)
    rb = g.gwas_packed_row_bytes(n)
    assert G.shape == (37, rb) and G.dtype == np.uint8
    assert np.array_equal(_decode_packed(G, n), X)
    # every code past the n-th genotype of a row is zero
    assert np.all(_decode_packed(G, 4 * rb)[:, n:] == 0)


def test_host_packing_rejects_invalid_values(g):
    X = np.zeros((3, 10), np.int8)
    X[1, 4] = 3
    X[2, 9] = -1
    G = np.zeros((3, 16), np.uint8)
    st = g.lib.gwas_pack_genotypes(X.ctypes.data, 3, 10, G.ctypes.data, 0, None)
    assert st == -6
    d = _decode_packed(G, 10)
    assert d[1, 4] == 3 and d[2, 9] == 3 and d.sum() == 6  # invalid values -> code 3, rest packed
    assert g.lib.gwas_pack_genotypes(None, 3, 10, G.ctypes.data, 0, None) == -1
    assert g.lib.gwas_pack_genotypes(X.ctypes.data, 3, 0, G.ctypes.data, 0, None) == -1
    assert g.lib.gwas_pack_genotypes(X.ctypes.data, 0, 10, None, 0, None) == 0


def test_scan_packed_null_handle(g):
    assert g.lib.gwas_scan_packed(None, None, 10, 1, None, None, 1, None) == -1


def test_batch_argument_checks(g):
    out = ctypes.c_void_p(7)
    assert g.lib.gwas_setup_batch(0, None, None, ctypes.byref(out)) == -1 and out.value is None
    Phi = np.eye(4, order="F"); XL = np.ones((4, 1), order="F"); Y = np.zeros((4, 1), order="F")
    h2 = np.array([0.5]); s2 = np.array([1.0])
    arr = (g.gwas_cohort * 1)()
    arr[0] = g.gwas_cohort(Phi.ctypes.data, 4, XL.ctypes.data, 1, Y.ctypes.data, 1, h2.ctypes.data,
                           s2.ctypes.data)
    opt = g.gwas_default_options(precision="fp64")
    assert g.lib.gwas_setup_batch(1, arr, ctypes.byref(opt), ctypes.byref(out)) == -5
    assert g.lib.gwas_setup_batch(300, arr, None, ctypes.byref(out)) == -1
    assert g.lib.gwas_scan_batch(None, None, None) == -1
    assert g.lib.gwas_batch_plan(None, None, None) == -1
    assert g.lib.gwas_batch_handle(None, 0) is None
    g.lib.gwas_destroy_batch(None)


def test_sync_and_selftest_argument_checks(g):
    assert g.lib.gwas_sync(None) == -1
    assert g.lib.gwas_selftest_timeout(0, 0) == -1
    assert g.lib.gwas_selftest_timeout(0, 20000) == -1


def test_wald_pvalues_host(g):
    from scipy.stats import chi2
    w = np.array([0.0, 3.841458820694124, 6.634896601021214, 0.5, 25.0, np.nan], np.float32)
    pv = g.gwas_wald_pvalues(w)
    ref = chi2.sf(w.astype(np.float64), 1)
    assert np.isnan(pv[-1])
    assert np.allclose(pv[:-1], ref[:-1], rtol=1e-6, atol=0)
    assert abs(pv[1] - 0.05) < 1e-7 and abs(pv[2] - 0.01) < 1e-7 and pv[0] == 1.0
    assert g.lib.gwas_wald_pvalues(None, 3, None, 0, None) == -1
    assert g.lib.gwas_wald_pvalues(None, 0, None, 0, None) == 0


def test_wald_pvalues_two_dof_host(g):
    """The joint test of the two-column model: chi-square(2) upper tail (scipy), 5 % at 5.991."""
    from scipy.stats import chi2
    w = np.array([0.0, 5.991464547107979, 9.21034037197618, 0.5, 40.0, np.nan], np.float32)
    pv = g.gwas_wald_pvalues_dof(w, 2)
    ref = chi2.sf(w.astype(np.float64), 2)
    assert np.isnan(pv[-1])
    assert np.allclose(pv[:-1], ref[:-1], rtol=1e-6, atol=0)
    assert abs(pv[1] - 0.05) < 1e-7 and abs(pv[2] - 0.01) < 1e-7 and pv[0] == 1.0
    assert np.array_equal(g.gwas_wald_pvalues_dof(w, 1), g.gwas_wald_pvalues(w), equal_nan=True)
    for dof in (0, 3):
        assert g.lib.gwas_wald_pvalues_dof(w.ctypes.data, 6, dof, w.ctypes.data, 0, None) == -1


def test_out_mode_option(g):
    o = g.gwas_default_options(out_mode="snp")
    assert o.out_mode == 1 and g.gwas_default_options().out_mode == 0


def test_estimate_argument_checks(g):
    """gwas_estimate rejects bad sizes, pointers and criteria before touching a device."""
    n, q, t = 6, 2, 2
    Phi = np.asfortranarray(np.eye(n))
    XL = np.asfortranarray(np.ones((n, q)))
    Y = np.asfortranarray(np.zeros((n, t)))
    h2, s2 = np.zeros(t), np.zeros(t)
    P, X, Yp, H, S = (a.ctypes.data for a in (Phi, XL, Y, h2, s2))
    L = g.lib.gwas_estimate
    assert L(None, n, X, q, Yp, t, 0, 0, H, S, None, None) == -1
    assert L(P, n, X, q, Yp, t, 0, 0, None, S, None, None) == -1
    assert L(P, 1, X, q, Yp, t, 0, 0, H, S, None, None) == -1
    assert L(P, n, X, 0, Yp, t, 0, 0, H, S, None, None) == -1
    assert L(P, n, X, n, Yp, t, 0, 0, H, S, None, None) == -1
    assert L(P, n, X, 8, Yp, t, 0, 0, H, S, None, None) == -1
    assert L(P, n, X, q, Yp, 0, 0, 0, H, S, None, None) == -1
    assert L(P, n, X, q, Yp, t, 2, 0, H, S, None, None) == -1
    assert g.EST_METHOD == {"ml": 0, "reml": 1}
