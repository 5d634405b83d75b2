"""Seeded synthetic GWAS inputs shaped like the paper's simulated workloads.

The paper (Supplementary Note, Section 4, "Simulated data") generates artificial data sets that
meet given n (individuals), m (SNPs), t (traits) and p (covariates) but does not describe the
generator.  This module is the stand-in: it only draws random numbers.  It holds no step of the
GLS method (no covariance matrix M, no factorisation, no solve), so the oracle and the CUDA path
can both take their inputs from here without sharing any of the method's arithmetic.

Recipe (fixed seeds: PCG64 keyed by 12072169 + workload index):

* genotypes: per SNP a minor-allele frequency f ~ U(0.05, 0.5); each of the n hard calls is
  Binomial(2, f), drawn as one uniform u per call: 0 if u < (1-f)^2, 2 if u >= 1-f^2, else 1.
  Stored SNP-major as int8 (one SNP's n calls contiguous).
* kinship: 2,000 further SNPs drawn the same way, each standardised by its sample mean and
  standard deviation (monomorphic ones redrawn); Phi = Gs Gs^T / 2000 + 1e-3 I.
* covariates X_L = [1 | N(0,1) columns].
* traits: beta_j ~ N(0,1)^q and y_j = X_L beta_j + sigma_j (h_j g_j + sqrt(1-h_j^2) e_j) where
  g_j = Gs u_j / sqrt(2000) + sqrt(1e-3) e'_j has covariance exactly Phi (no factorisation needed).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 12072169
KINSHIP_SNPS = 2000
KINSHIP_RIDGE = 1e-3


def rng(workload: int, stream: int = 0) -> np.random.Generator:
    """Independent PCG64 stream per (workload, purpose)."""
    return np.random.Generator(np.random.PCG64([SEED_BASE + workload, stream]))


def genotypes(g: np.random.Generator, n: int, m: int, block: int = 65536) -> np.ndarray:
    """(m, n) int8 hard calls in {0,1,2}; MAF ~ U(0.05, 0.5) per SNP."""
    out = np.empty((m, n), dtype=np.int8)
    for s in range(0, m, block):
        e = min(m, s + block)
        f = g.uniform(0.05, 0.5, size=e - s).astype(np.float32)
        u = g.random((e - s, n), dtype=np.float32)
        lo = ((1.0 - f) ** 2)[:, None]
        hi = (1.0 - f * f)[:, None]
        blk = out[s:e]
        np.greater_equal(u, lo, out=blk, casting="unsafe")
        blk += (u >= hi)
    return out


def kinship_factor(g: np.random.Generator, n: int, n_snps: int = KINSHIP_SNPS) -> np.ndarray:
    """Standardised genotype matrix Gs (n x n_snps): each column has mean 0, ddof-0 SD 1."""
    G = genotypes(g, n, n_snps).astype(np.float64)
    while True:
        sd = G.std(axis=1)
        bad = np.flatnonzero(sd == 0.0)
        if bad.size == 0:
            break
        G[bad] = genotypes(g, n, bad.size).astype(np.float64)
    mu = G.mean(axis=1)
    sd = G.std(axis=1)
    return ((G - mu[:, None]) / sd[:, None]).T.copy()


def kinship(Gs: np.ndarray, ridge: float = KINSHIP_RIDGE) -> np.ndarray:
    n, k = Gs.shape
    Phi = Gs @ Gs.T / k
    Phi[np.diag_indices(n)] += ridge
    return Phi


def covariates(g: np.random.Generator, n: int, q: int) -> np.ndarray:
    """X_L = [1 | N(0,1) ...], n x q float64 (q = p - 1 >= 1)."""
    XL = np.empty((n, q))
    XL[:, 0] = 1.0
    if q > 1:
        XL[:, 1:] = g.standard_normal((n, q - 1))
    return XL


def traits(g: np.random.Generator, XL: np.ndarray, Gs: np.ndarray, h2: np.ndarray,
           s2: np.ndarray, ridge: float = KINSHIP_RIDGE, chunk: int = 4096):
    """Y (n x t) with columns ~ N(X_L beta_j, s2_j (h2_j Phi + (1-h2_j) I)); returns (Y, beta)."""
    n, q = XL.shape
    k = Gs.shape[1]
    t = len(h2)
    beta = g.standard_normal((q, t))
    Y = np.empty((n, t))
    for s in range(0, t, chunk):
        e = min(t, s + chunk)
        u = g.standard_normal((k, e - s))
        e1 = g.standard_normal((n, e - s))
        e2 = g.standard_normal((n, e - s))
        gen = Gs @ u / math.sqrt(k) + math.sqrt(ridge) * e1
        Y[:, s:e] = XL @ beta[:, s:e] + np.sqrt(s2[s:e]) * (
            np.sqrt(h2[s:e]) * gen + np.sqrt(1.0 - h2[s:e]) * e2)
    return Y, beta


@dataclasses.dataclass
class Cohort:
    """One GWAS problem: Phi (n x n), X_L (n x q), Y (n x t), h2 (t), s2 (t), XR (m x n int8)."""
    Phi: np.ndarray
    XL: np.ndarray
    Y: np.ndarray
    h2: np.ndarray
    s2: np.ndarray
    XR: np.ndarray | None
    beta: np.ndarray

    @property
    def n(self):
        return self.Phi.shape[0]

    @property
    def q(self):
        return self.XL.shape[1]

    @property
    def p(self):
        return self.XL.shape[1] + 1

    @property
    def t(self):
        return self.Y.shape[1]

    @property
    def m(self):
        return 0 if self.XR is None else self.XR.shape[0]


# The five workloads: sizes, value distributions and h2 / s2 recipes.
WORKLOADS = {
    0: dict(name="chol_fp64_n256_m10k", n=256, q=3, m=10_000, t=1, h2=0.4, s2=1.0,
            algo="chol", block=10_000),
    1: dict(name="chol_split_bf16_n1000_m2M", n=1000, q=3, m=2_000_000, t=1, h2=0.5, s2=1.0,
            algo="chol", block=65_536),
    2: dict(name="eig_n1000_t1000_m100k", n=1000, q=3, m=100_000, t=1000, h2=(0.05, 0.95),
            s2=(0.5, 2.0), algo="eig", block=32_768),
    3: dict(name="eig_omics_n1000_t30000_m1M", n=1000, q=3, m=1_000_000, t=30_000,
            h2=(0.05, 0.95), s2=(0.5, 2.0), algo="eig", block=32_768),
}


def _params(g, spec, t):
    if isinstance(spec["h2"], tuple):
        h2 = g.uniform(*spec["h2"], size=t)
        s2 = g.uniform(*spec["s2"], size=t)
    else:
        h2 = np.full(t, float(spec["h2"]))
        s2 = np.full(t, float(spec["s2"]))
    return h2, s2


def make_cohort(workload: int, n=None, q=None, m=None, t=None, with_genotypes=True) -> Cohort:
    """Build workload `workload`'s problem, optionally shrunk (n, q, m, t overrides)."""
    spec = dict(WORKLOADS[workload])
    n = spec["n"] if n is None else n
    q = spec["q"] if q is None else q
    m = spec["m"] if m is None else m
    t = spec["t"] if t is None else t
    Gs = kinship_factor(rng(workload, 1), n)
    Phi = kinship(Gs)
    XL = covariates(rng(workload, 2), n, q)
    gp = rng(workload, 3)
    h2, s2 = _params(gp, spec, t)
    Y, beta = traits(gp, XL, Gs, h2, s2)
    XR = genotypes(rng(workload, 4), n, m) if with_genotypes else None
    return Cohort(Phi=Phi, XL=XL, Y=Y, h2=h2, s2=s2, XR=XR, beta=beta)


def snp_block(workload: int, n: int, m: int, block_index: int) -> np.ndarray:
    """Genotype block `block_index` (m x n int8) from its own stream: lets a long scan draw
    blocks lazily without holding the whole genome."""
    return genotypes(rng(workload, 1000 + block_index), n, m)


# Workload 4: a batch of uneven cohorts, each with its own kinship (drawn as in workload 0),
# n log-uniform in [500, 5000], p = q + 1 uniform in {3..8}, t log-uniform in [10, 2000],
# h2 ~ U(0.05, 0.95), s2 ~ U(0.5, 2), m = 200,000 SNPs each.
BATCH = dict(name="batch16_uneven_m200k", cohorts=16, n=(500, 5000), p=(3, 8), t=(10, 2000),
             m=200_000, h2=(0.05, 0.95), s2=(0.5, 2.0))


def batch_shapes(cohorts: int | None = None):
    """(n, q, t) of each cohort of workload 4."""
    spec = BATCH
    k = spec["cohorts"] if cohorts is None else cohorts
    g = rng(4, 0)
    n = np.rint(np.exp(g.uniform(np.log(spec["n"][0]), np.log(spec["n"][1]), size=k))).astype(int)
    p = g.integers(spec["p"][0], spec["p"][1] + 1, size=k)
    t = np.rint(np.exp(g.uniform(np.log(spec["t"][0]), np.log(spec["t"][1]), size=k))).astype(int)
    return [(int(a), int(b) - 1, int(c)) for a, b, c in zip(n, p, t)]


def batch_cohort(i: int, n: int, q: int, t: int) -> Cohort:
    """Cohort i of workload 4 without genotypes (they are drawn on the device, see
    device_genotypes): its own kinship, covariates and traits."""
    g = np.random.Generator(np.random.PCG64([SEED_BASE + 4, 100 + i]))
    Gs = kinship_factor(g, n)
    Phi = kinship(Gs)
    XL = covariates(g, n, q)
    h2 = g.uniform(*BATCH["h2"], size=t)
    s2 = g.uniform(*BATCH["s2"], size=t)
    Y, beta = traits(g, XL, Gs, h2, s2)
    return Cohort(Phi=Phi, XL=XL, Y=Y, h2=h2, s2=s2, XR=None, beta=beta)


def device_genotypes(seed: int, n: int, m: int, device="cuda"):
    """m x n int8 hard calls drawn on a CUDA device (torch generator seeded by `seed`): per SNP
    MAF ~ U(0.05, 0.5), each call Binomial(2, MAF) from one uniform -- the recipe of `genotypes`
    with another generator, for batches too large to draw on the host."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(SEED_BASE * 1000 + seed)
    f = torch.rand((m, 1), generator=gen, device=device) * 0.45 + 0.05
    u = torch.rand((m, n), generator=gen, device=device)
    x = (u >= (1.0 - f) ** 2).to(torch.int8)   # as `genotypes`: one uniform per call
    x += (u >= 1.0 - f * f).to(torch.int8)
    return x


def workload_genotypes(workload: int, m: int | None = None, start: int = 0) -> np.ndarray:
    """SNPs [start, start + m) (default: the whole genome) of workload `workload`'s genome, m x n
    int8, assembled from its per-block streams (snp_block), so that every SNP is the same
    whatever range it is drawn in: any prefix, and any rank's shard of a longer genome."""
    spec = WORKLOADS[workload]
    n, blk = spec["n"], spec["block"]
    m = spec["m"] if m is None else m
    XR = np.empty((m, n), dtype=np.int8)
    end = start + m
    for b in range(start // blk, (end + blk - 1) // blk):
        lo, hi = max(start, b * blk), min(end, (b + 1) * blk)
        XR[lo - start:hi - start] = snp_block(workload, n, blk, b)[lo - b * blk:hi - b * blk]
    return XR


def small_problem(seed: int, n: int, q: int, m: int, t: int, h2=None, s2=None) -> Cohort:
    """Small random problem for parity tests (any n, q, m, t)."""
    g = np.random.Generator(np.random.PCG64([SEED_BASE, 77, seed]))
    Gs = kinship_factor(g, n, n_snps=max(2 * n, 64))
    Phi = kinship(Gs)
    XL = covariates(g, n, q)
    h2 = g.uniform(0.05, 0.95, size=t) if h2 is None else np.broadcast_to(np.asarray(h2, float), (t,)).copy()
    s2 = g.uniform(0.5, 2.0, size=t) if s2 is None else np.broadcast_to(np.asarray(s2, float), (t,)).copy()
    Y, beta = traits(g, XL, Gs, h2, s2)
    XR = genotypes(g, n, m)
    return Cohort(Phi=Phi, XL=XL, Y=Y, h2=h2, s2=s2, XR=XR, beta=beta)
