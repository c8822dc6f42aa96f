"""FP64 CPU oracle for SP-SVM (sparse primal kernel SVM, Section 4, Eq. 4).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute anything in this package: only the tests, the smoke check
and the CPU-baseline leg of the benchmark use it.  It shares no code with
the CUDA library (no kernels, headers, helpers or constants); the only
common inputs are the arrays produced by the seeded synthetic generators.

Every function here is written to be checked by eye against the paper:
plain float64 numpy, library primitives (matmul, Cholesky, sort) used only
as whole steps, no blocking, fusion or reordering beyond the definitions.

Parity status of each function (see the pins in tests/test_oracle_*.py):
  rbf_kernel, objective, gradient, hessian, newton_direction, line_search,
  score_candidates, score_candidates_exact, select_top, draw_candidates, fit,
  predict, ovo_pairs,
  ovo_vote, fit_ovo, predict_ovo: pinned.
  Accuracy figures of the paper's Table 1: parity unpinned (datasets absent).
"""
from .spsvm import (  # noqa: F401
    rbf_kernel, objective, gradient, hessian, newton_solve, jittered_cholesky, cholesky_solve,
    jitter_shift, JITTER_MAX_LEVEL, line_search,
    line_search_derivative, score_candidates, score_candidates_exact, select_top, draw_candidates,
    splitmix64, newton, fit, predict, FitResult, ovo_pairs, ovo_vote, fit_ovo, predict_ovo,
)
from .dual import squared_hinge_dual_bruteforce  # noqa: F401
