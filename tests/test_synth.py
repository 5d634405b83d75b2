"""The seeded input generator: shapes, value sets and distributions (CPU only)."""
import numpy as np

import synth


def test_genotypes_are_hard_calls_with_binomial_frequencies():
    g = synth.genotypes(synth.rng(9, 0), 4000, 300)
    assert g.dtype == np.int8 and g.shape == (300, 4000)
    assert set(np.unique(g)) <= {0, 1, 2}
    f = g.mean(axis=1) / 2.0
    assert f.min() > 0.03 and f.max() < 0.53
    # Hardy-Weinberg: P(1) = 2f(1-f)
    het = (g == 1).mean(axis=1)
    assert np.max(np.abs(het - 2 * f * (1 - f))) < 0.04


def test_generator_is_deterministic():
    a = synth.make_cohort(0, m=50)
    b = synth.make_cohort(0, m=50)
    assert np.array_equal(a.XR, b.XR) and np.array_equal(a.Y, b.Y) and np.array_equal(a.Phi, b.Phi)


def test_kinship_is_standardised_and_spd():
    c = synth.make_cohort(0, m=1)
    assert np.allclose(np.diag(c.Phi).mean(), 1.0 + synth.KINSHIP_RIDGE, atol=1e-12)
    w = np.linalg.eigvalsh(c.Phi)
    assert w.min() > 0.5 * synth.KINSHIP_RIDGE
    assert np.allclose(c.Phi, c.Phi.T)


def test_trait_covariance_matches_model():
    n, t = 30, 20000
    g = synth.rng(11, 0)
    Gs = synth.kinship_factor(g, n, n_snps=200)
    Phi = synth.kinship(Gs)
    XL = synth.covariates(g, n, 1)
    h2 = np.full(t, 0.6)
    s2 = np.full(t, 1.5)
    Y, beta = synth.traits(g, XL, Gs, h2, s2)
    R = Y - XL @ beta
    C = R @ R.T / t
    target = 1.5 * (0.6 * Phi + 0.4 * np.eye(n))
    assert np.max(np.abs(C - target)) < 6 * 1.5 / np.sqrt(t) * 2
