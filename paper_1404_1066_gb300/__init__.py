"""GB300 (sm_103a) SP-SVM: sparse primal kernel SVM of "Parallel Support
Vector Machines in Practice", Section 4, Eq. 4, as hand-written CUDA behind
the C ABI of include/spsvm.h.

    import paper_1404_1066_gb300 as sp
    model = sp.spsvm_fit(X, y, gamma, lam, budget, tol, precision="bf16split")
    f = sp.spsvm_predict(model, Xq)

The CUDA library is built in-tree on first use (paper_1404_1066_gb300.build)
and is required: there is no CPU path.
"""
from .api import (  # noqa: F401
    KMat, Model, Points, kmat_empty, make_options, spsvm_cholesky, spsvm_cholesky_solve,
    spsvm_compact_active, spsvm_decision, spsvm_draw_candidates, spsvm_fit,
    spsvm_fit_workspace_bytes, spsvm_gemv, spsvm_gram, spsvm_kernel_block, spsvm_line_search,
    spsvm_outputs, spsvm_predict, spsvm_prepare_points, spsvm_score_candidates,
    spsvm_score_candidates_noalloc, spsvm_score_candidates_exact, spsvm_fit_batched, spsvm_solve_mixed, spsvm_cholesky_mixed, spsvm_fit_ovo,
    spsvm_solve_lowrank, spsvm_active_diff, spsvm_predict_work_bytes,
    spsvm_predict_ovo, Server,
)
from ._lib import SPSVM_BF16SPLIT, SPSVM_FP32, SpsvmError, load  # noqa: F401
