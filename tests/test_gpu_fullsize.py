"""Parity at the full workload sizes, in the launch configuration the
benchmark times (BF16SPLIT kernel values, FP64 Newton system, kappa = 256
candidates, q = 64 added per round, tol 1e-6):

  * Gaussian mixture n = 500,000, d = 128, |J| = 4096 (64 rounds);
  * sparse teacher n = 100,000, d = 784, |J| = 1024 (16 rounds).

The float64 oracle cannot refit these sizes in a test, so it checks what it
can compute one output at a time from the GPU's basis J and coefficients
beta (direct-difference kernels, float64):

  * training outputs o_i = sum_j k(x_i, x_j) beta_j on sampled rows;
  * decision values on sampled held-out queries;
  * the objective, with lambda/2 beta^T K_JJ beta recomputed by the oracle;
  * stationarity of the exact objective (Eq. 4 divided by C) on sampled
    coordinates of the gradient g_j = lambda (K_JJ beta)_j +
    sum_{i in S} k(x_i, x_j) (o_i - y_i).

Tolerances follow from the stored arithmetic: a BF16SPLIT kernel value carries
|dK| <= 6e-5 gamma (|x|^2 + |z|^2) + 1e-5 K + 2e-6 (split dot products,
hi+lo storage, exp2 epilogue), the FP32 predict path |dK| <= 2e-6 +
4 eps32 gamma (|x|^2 + |z|^2), and sums promote to FP64 every 32 terms
(1e-5 of the sum of absolute terms).  Stationarity: the fit stops when its
own gradient is below 2e-5 ||K_SJ^T y_S||, and the exact gradient differs
from it by the kernel errors above; the threshold on each sampled |g_j|,
1e-4 of the magnitude of its terms, is empirical (measured 1.2e-7 on the
mixture and 1.5e-5 on the sparse teacher), whereas a beta that is not
stationary gives 1e-2 to 1 there."""
import numpy as np
import pytest
import torch

from oracle import spsvm as O
from paper_1404_1066_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

EPS32 = float(np.finfo(np.float32).eps)
CASES = {
    "mixture_n500k_d128_J4096": dict(make=lambda: synth.gaussian_mixture(
        n=500_000, d=128, budget=4096, seed=1003), queries=100_000),
    "sparse_teacher_n100k_d784_J1024": dict(make=lambda: synth.sparse_teacher(
        n=100_000, d=784, budget=1024, seed=1002), queries=20_000),
}


@pytest.fixture(scope="module")
def sp():
    import paper_1404_1066_gb300 as sp
    sp.load()
    return sp


@pytest.fixture(scope="module", params=list(CASES))
def fitted(request, sp):
    case = CASES[request.param]
    p = case["make"]()
    Xq = synth.queries_like(p, case["queries"], seed=77)
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    m = sp.spsvm_fit(X, y, p.gamma, p.lam, p.budget, 1e-6, precision="bf16split",
                     candidates=256, add_per_round=64, seed=1)
    f = sp.spsvm_predict(m, torch.from_numpy(Xq).cuda()).cpu().numpy().astype(np.float64)
    J, beta = m.basis_and_beta()
    o = m.outputs(p.X.shape[0]).astype(np.float64)
    info = m.info()
    del X, y
    torch.cuda.empty_cache()
    return dict(p=p, Xq=Xq, J=J, beta=beta, o=o, f=f, info=info, name=request.param)


def _bf16split_bound(Xs, XJ, K, beta, gamma):
    nx = np.sum(Xs.astype(np.float64) ** 2, axis=1)[:, None]
    nz = np.sum(XJ.astype(np.float64) ** 2, axis=1)[None, :]
    dK = 6e-5 * gamma * (nx + nz) + 1e-5 * K + 2e-6
    return dK @ np.abs(beta) + 1e-5 * (np.abs(K) @ np.abs(beta))


def test_fit_reaches_budget(fitted):
    info, p = fitted["info"], fitted["p"]
    assert info["status"] == 0, info
    assert info["n_basis"] == p.budget
    assert len(np.unique(fitted["J"])) == p.budget


def test_sampled_training_outputs(fitted):
    p, J, beta = fitted["p"], fitted["J"], fitted["beta"]
    rows = np.sort(np.random.default_rng(5).choice(p.X.shape[0], 1000, replace=False))
    K = O.rbf_kernel(p.X[rows], p.X[J], p.gamma)
    ref = K @ beta
    bound = _bf16split_bound(p.X[rows], p.X[J], K, beta, p.gamma)
    err = np.abs(fitted["o"][rows] - ref)
    print(fitted["name"], "outputs: max err/bound", np.max(err / bound))
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3g}"


def test_sampled_decision_values(fitted):
    p, J, beta, Xq = fitted["p"], fitted["J"], fitted["beta"], fitted["Xq"]
    rows = np.sort(np.random.default_rng(6).choice(Xq.shape[0], 1000, replace=False))
    K = O.rbf_kernel(Xq[rows], p.X[J], p.gamma)
    ref = K @ beta
    nx = np.sum(Xq[rows].astype(np.float64) ** 2, axis=1)[:, None]
    nz = np.sum(p.X[J].astype(np.float64) ** 2, axis=1)[None, :]
    bound = (2e-6 + 4 * EPS32 * p.gamma * (nx + nz)) @ np.abs(beta) + 1e-5 * (K @ np.abs(beta))
    err = np.abs(fitted["f"][rows] - ref)
    print(fitted["name"], "decisions: max err/bound", np.max(err / bound))
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3g}"
    # labels agree wherever the decision value is outside its error bound
    sure = np.abs(ref) > bound
    np.testing.assert_array_equal(O.labels(fitted["f"][rows][sure]), O.labels(ref[sure]))


def test_objective_with_oracle_quadratic_term(fitted):
    p, J, beta, o = fitted["p"], fitted["J"], fitted["beta"], fitted["o"]
    KJJ = O.rbf_kernel(p.X[J], p.X[J], p.gamma)
    quad = 0.5 * p.lam * beta @ (KJJ @ beta)
    xi = np.maximum(0.0, 1.0 - p.y.astype(np.float64) * o)
    f_ref = quad + 0.5 * np.sum(xi * xi)
    # the quadratic term's BF16SPLIT kernel errors relative to |beta|^T |K_JJ| |beta|
    tol = 1e-4 * (0.5 * p.lam * np.abs(beta) @ (KJJ @ np.abs(beta))) + 1e-6 * f_ref
    print(fitted["name"], "objective: err/tol", abs(fitted["info"]["objective"] - f_ref) / tol)
    assert abs(fitted["info"]["objective"] - f_ref) <= tol, (fitted["info"]["objective"], f_ref)


def test_sampled_gradient_coordinates_vanish(fitted):
    p, J, beta, o = fitted["p"], fitted["J"], fitted["beta"], fitted["o"]
    y = p.y.astype(np.float64)
    S = y * o < 1.0
    cols = np.sort(np.random.default_rng(7).choice(len(J), 24, replace=False))
    KJc = O.rbf_kernel(p.X[J], p.X[J[cols]], p.gamma)        # |J| x 24
    res = np.where(S, o - y, 0.0)
    g = p.lam * (KJc.T @ beta)
    mag = p.lam * (KJc.T @ np.abs(beta))
    XS = p.X[S]
    rS = res[S]
    for r0 in range(0, XS.shape[0], 20000):
        Kc = O.rbf_kernel(XS[r0:r0 + 20000], p.X[J[cols]], p.gamma)
        g += Kc.T @ rS[r0:r0 + 20000]
        mag += Kc.T @ (np.abs(rS[r0:r0 + 20000]) + 1.0)
    ratio = np.abs(g) / mag
    print(fitted["name"], "gradient: max |g_j|/magnitude", np.max(ratio))
    assert np.all(ratio <= 1e-4), f"max |g_j| / magnitude {np.max(ratio):.3g}"
