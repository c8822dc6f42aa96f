"""Low-rank correction of the Newton solve (Section 4 reoptimisation): when
the active set changes by k points between Newton steps, the Newton matrix
changes by the rank-k term W^T Sigma W of their kernel rows, and the factor
in hand is corrected by the Sherman-Morrison-Woodbury identity instead of
being recomputed.  Checked against the oracle's Cholesky solve of the new
Newton matrix, and over whole fits against the oracle's replay and against
fits that factor afresh at every change of the active set."""
import numpy as np
import pytest
import torch

from oracle import spsvm as O
from paper_1404_1066_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    import paper_1404_1066_gb300 as sp
    sp.load()
    return sp


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _newton_pair(m, n_in, n_out, seed, n=6000, d=10, lam=1e-2, gamma=0.5):
    """Kernel rows (FP32) of n points on m basis points, two active sets
    S_a and S differing by n_in entering and n_out leaving points, and the
    Newton matrices lambda K_JJ + K_S^T K_S of both (FP64 from the FP32
    values; condition numbers ~1e4..1e5, where an FP32 factor refines to
    FP64 accuracy)."""
    g = np.random.default_rng(seed)
    X = g.standard_normal((n, d)).astype(np.float32)
    J = np.sort(g.choice(n, m, replace=False))
    K = O.rbf_kernel(X, X[J], gamma).astype(np.float32).astype(np.float64)
    Sa = g.random(n) < 0.4
    inside, outside = np.flatnonzero(Sa), np.flatnonzero(~Sa)
    S = Sa.copy()
    S[g.choice(outside, n_in, replace=False)] = True
    S[g.choice(inside, n_out, replace=False)] = False
    KJJ = 0.5 * (K[J] + K[J].T)
    Ha = lam * KJJ + K[Sa].T @ K[Sa]
    H = lam * KJJ + K[S].T @ K[S]
    return K, Sa, S, Ha, H


def _kmat(sp, K):
    """K (n x m) stored basis-major in FP32."""
    n, m = K.shape
    km = sp.kmat_empty(n, m, "fp32")
    km.buf.view(-1)[: m * km.ld].view(m, km.ld)[:, :n] = _t(K.T.astype(np.float32))
    return km


@pytest.mark.parametrize("m,n_in,n_out", [(600, 5, 3), (1000, 40, 0), (1000, 0, 40),
                                          (1500, 60, 68), (777, 1, 0), (2048, 64, 64)])
def test_lowrank_solve_matches_oracle(sp, m, n_in, n_out):
    K, Sa, S, Ha, H = _newton_pair(m, n_in, n_out, seed=m + n_in)
    km = _kmat(sp, K)
    k, Wt, sign = sp.spsvm_active_diff(km, _t(S.astype(np.uint8)), _t(Sa.astype(np.uint8)), 128)
    D = np.flatnonzero(S != Sa)
    assert k == len(D) == n_in + n_out
    # the changed points in increasing order, their kernel rows and signs
    np.testing.assert_array_equal(Wt.cpu().numpy(), K[D].T.astype(np.float32))
    np.testing.assert_array_equal(sign.cpu().numpy(), np.where(S[D], 1.0, -1.0))
    # H = Ha + W^T Sigma W in exact arithmetic
    g = np.random.default_rng(1)
    b, b2 = g.standard_normal(m), g.standard_normal(m)
    fi, ci, st, x, its, be, xs = sp.spsvm_solve_lowrank(_t(Ha), _t(H), Wt, sign, _t(b),
                                                        extra_rhs=(_t(b2),))
    assert fi == 0
    if ci != 0:
        # a rejected capacitance C = Sigma + V^T V must be ill-conditioned
        # (the pivot test of its FP32 inverse: a pivot below 1e-3 of max |C|)
        Lr, _ = O.jittered_cholesky(Ha)
        Vr = np.linalg.solve(Lr, K[D].T)
        Cr = np.diag(np.where(S[D], 1.0, -1.0)) + Vr.T @ Vr
        assert np.linalg.cond(Cr) > 1e2, np.linalg.cond(Cr)
        return
    assert st == 0, (fi, ci, st, its, be)
    for rhs, xg in ((b, x), (b2, xs[0])):
        xg = xg.cpu().numpy()
        r = rhs - H @ xg
        bw = np.max(np.abs(r)) / (np.max(np.abs(H).sum(1)) * np.max(np.abs(xg)) + np.max(np.abs(rhs)))
        assert bw <= 1e-13, bw
        xr, lv = O.newton_solve(H, rhs)
        assert lv == -1
        cond = np.linalg.cond(H)
        assert np.linalg.norm(xg - xr) <= 1e-12 * cond * np.linalg.norm(xr), (cond, np.linalg.norm(xg - xr))
    # as fast as a fresh factor: the correction is exact up to FP32 rounding
    assert its <= 8, its


def test_lowrank_diff_over_kmax_and_empty(sp):
    K, Sa, S, _, _ = _newton_pair(600, 70, 70, seed=3)
    km = _kmat(sp, K)
    k, Wt, sign = sp.spsvm_active_diff(km, _t(S.astype(np.uint8)), _t(Sa.astype(np.uint8)), 100)
    assert k == 140 and Wt.shape[1] == 100   # counted, rows not gathered past kmax
    k0, _, _ = sp.spsvm_active_diff(km, _t(Sa.astype(np.uint8)), _t(Sa.astype(np.uint8)), 100)
    assert k0 == 0


def test_lowrank_wrong_correction_never_claims_convergence(sp):
    """With the signs flipped the correction describes another matrix: the
    refinement against the true H either still reaches FP64 backward error
    (the result is then right) or reports NO_CONVERGE; never a wrong answer."""
    K, Sa, S, Ha, H = _newton_pair(800, 30, 30, seed=11)
    km = _kmat(sp, K)
    k, Wt, sign = sp.spsvm_active_diff(km, _t(S.astype(np.uint8)), _t(Sa.astype(np.uint8)), 128)
    b = np.random.default_rng(2).standard_normal(800)
    fi, ci, st, x, its, be, _ = sp.spsvm_solve_lowrank(_t(Ha), _t(H), Wt, -sign, _t(b))
    if fi == 0 and ci == 0 and st == 0:
        xg = x.cpu().numpy()
        r = b - H @ xg
        assert np.max(np.abs(r)) <= 1e-13 * (np.max(np.abs(H).sum(1)) * np.max(np.abs(xg)) + np.max(np.abs(b)))
    else:
        assert ci != 0 or st == -4


@pytest.mark.parametrize("prec", ["fp32", "bf16split"])
def test_fit_lowrank_steps_against_oracle_and_refactoring(sp, prec):
    """A growth run to |J| = 1024 on the benchmark workload's generator
    (mixture, d = 128, gamma = 1/d) at n = 20,000: Newton steps past
    |J| = 512 whose active set changed correct the factor in hand (points
    entering and leaving); the fit takes the same steps and basis as one that
    factors afresh at every change, and the oracle's replay holds it to the
    1e-4 bar on beta and decision values."""
    p = synth.gaussian_mixture(n=20000, d=128, budget=1024, seed=1201, lam=1e-3)
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    kw = dict(precision=prec, candidates=256, add_per_round=64, seed=23, record=True)
    m = sp.spsvm_fit(X, y, p.gamma, p.lam, 1024, 1e-8, lowrank=True, **kw)
    mf = sp.spsvm_fit(X, y, p.gamma, p.lam, 1024, 1e-8, **kw)
    h = m.history()
    lr = [s for s in h if s["solve"] == 3]
    assert len(lr) >= 3, [(s["basis"], s["solve"], s["changed"]) for s in h]
    assert all(s["basis"] >= 512 for s in lr)
    assert all(s["solve"] != 3 for s in mf.history())
    fac = sum(1 for s in h if s["solve"] == 1)
    assert fac < sum(1 for s in mf.history() if s["solve"] == 1)
    J, beta = m.basis_and_beta()
    Jf, _ = mf.basis_and_beta()
    np.testing.assert_array_equal(J, Jf)
    Xq = synth.queries_like(p, 3000, seed=6)
    f = m.predict(torch.from_numpy(Xq).cuda()).cpu().numpy().astype(np.float64)
    ff = mf.predict(torch.from_numpy(Xq).cuda()).cpu().numpy().astype(np.float64)
    assert np.max(np.abs(f - ff) / np.maximum(1.0, np.abs(ff))) <= 1e-4
    info = m.info()
    rep = [dict(candidates=c, chosen=ch) for c, ch in (m.round(k) for k in range(info["rounds"]))]
    r = O.fit(p.X, p.y, p.gamma, p.lam, 1024, tol=1e-10, kappa=256, q=64, seed=23, replay=rep,
              replay_rtol=1e-3)
    np.testing.assert_array_equal(J, r.J)
    assert np.linalg.norm(beta - r.beta) <= 1e-4 * np.linalg.norm(r.beta)
    fr = O.predict(Xq, p.X[J], r.beta, p.gamma)
    assert np.max(np.abs(f - fr) / np.maximum(1.0, np.abs(fr))) <= 1e-4
