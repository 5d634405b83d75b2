"""FP64 CPU oracle for the 2-D grid of GLS problems (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs may import
this package.  The CUDA library never calls it and shares no code with it.

Modules:
  gls   -- the definition (Eq. "GLS" and Eq. "probDef", Supplementary Note Section 1) solved
           per problem by the single-GLS Cholesky algorithm (Algorithm 1), the single-GLS
           eigen algorithm (Algorithm 2), and the two sequence algorithms in the paper's
           order (Algorithm 3 CLAK-Chol, Algorithm 4 CLAK-Eig).
  exact -- the same definition in exact rational arithmetic (Fractions), for tiny problems.
  estimate -- step 1 of the two-step method: per-trait (h^2, sigma^2) by maximum likelihood or
           restricted maximum likelihood of the reduced model (Supplementary Note Section 1).
"""
from .gls import (form_M, gls_chol, gls_eig, gls_grid, chol_sequence, eig_sequence,
                  wald_from, wald_block, genetic_columns, GENETIC_MODELS, rel_err_b,
                  rel_err_wald, max_rel_errors)

__all__ = ["form_M", "gls_chol", "gls_eig", "gls_grid", "chol_sequence", "eig_sequence",
           "wald_from", "wald_block", "genetic_columns", "GENETIC_MODELS", "rel_err_b",
           "rel_err_wald", "max_rel_errors"]
