"""Whole-fit parity of the CUDA path against the float64 oracle.

Decision values must agree within 1e-4 relative (|f_gpu - f_orc| <=
1e-4 max(1, |f_orc|)); active sets must agree except for points whose
oracle margin lies within the tie band |1 - y_i o_i| <= 1e-5 (FP32 outputs
carry ~1e-6 relative error); growth runs use the replay protocol (the
oracle checks each GPU choice against its own scores and adopts it)."""
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


def _cmp_decisions(f_gpu, f_orc, rtol=1e-4):
    err = np.abs(np.asarray(f_gpu, dtype=np.float64) - f_orc)
    bound = rtol * np.maximum(1.0, np.abs(f_orc))
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3g}"


def _cmp_active(o_gpu, o_orc, y, band=1e-5):
    Sg = y * o_gpu < 1
    So = y * o_orc < 1
    tie = np.abs(1 - y * o_orc) <= band
    assert np.all((Sg == So) | tie), int(np.sum((Sg != So) & ~tie))


@pytest.mark.parametrize("prec", ["fp32"])
def test_fixed_basis_two_gaussians(sp, prec):
    p = synth.two_gaussians()
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    m = sp.spsvm_fit(X, y, p.gamma, p.lam, p.budget, 1e-8, precision=prec,
                     initial_basis=p.initial_basis, fixed_basis=True)
    assert m.status == 0
    r = O.fit(p.X, p.y, p.gamma, p.lam, p.budget, tol=1e-8, initial_basis=p.initial_basis,
              grow=False)
    J, beta = m.basis_and_beta()
    np.testing.assert_array_equal(J, p.initial_basis)
    o = m.outputs(len(p.y))
    yd = p.y.astype(np.float64)
    _cmp_decisions(o, r.o)
    _cmp_active(o.astype(np.float64), r.o, yd)
    assert np.linalg.norm(beta - r.beta) <= 1e-4 * np.linalg.norm(r.beta)
    Xq = synth.queries_like(p, 3000, seed=5)
    f = m.predict(torch.from_numpy(Xq).cuda()).cpu().numpy()
    _cmp_decisions(f, O.predict(Xq, p.X[J], r.beta, p.gamma))
    info = m.info()
    assert abs(info["objective"] - O.objective(r.beta, O.rbf_kernel(p.X, p.X[J], p.gamma),
                                               O.rbf_kernel(p.X[J], p.X[J], p.gamma), yd,
                                               p.lam)) <= 1e-5 * abs(info["objective"])
    hist = m.history()
    losses = [h["loss"] for h in hist if h["t"] > 0]
    assert len(losses) >= 2


@pytest.mark.parametrize("prec", ["fp32"])
def test_growth_replay_mixture(sp, prec):
    p = synth.gaussian_mixture(n=3000, d=16, budget=192, seed=11, lam=1e-3)
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    m = sp.spsvm_fit(X, y, p.gamma, p.lam, 192, 1e-8, precision=prec, candidates=128,
                     add_per_round=64, seed=77, record=True)
    info = m.info()
    assert info["rounds"] == 3 and info["n_basis"] == 192
    rep = []
    for k in range(info["rounds"]):
        cand, chosen = m.round(k)
        rep.append(dict(candidates=cand, chosen=chosen))
    r = O.fit(p.X, p.y, p.gamma, p.lam, 192, tol=1e-10, kappa=128, q=64, seed=77, replay=rep,
              replay_rtol=1e-4)
    J, beta = m.basis_and_beta()
    np.testing.assert_array_equal(J, r.J)
    o = m.outputs(len(p.y))
    _cmp_decisions(o, r.o)
    _cmp_active(o.astype(np.float64), r.o, p.y.astype(np.float64))


def test_fit_argument_errors(sp):
    X = torch.zeros((10, 3), device="cuda")
    y = torch.ones(10, device="cuda")
    with pytest.raises(sp.SpsvmError):
        sp.spsvm_fit(X, y, -1.0, 1e-3, 5)
    with pytest.raises(sp.SpsvmError):
        sp.spsvm_fit(X, y, 1.0, 1e-3, 11)
    with pytest.raises(sp.SpsvmError):
        sp.spsvm_fit(X, y, 1.0, 1e-3, 5, initial_basis=[1, 1], fixed_basis=True)
