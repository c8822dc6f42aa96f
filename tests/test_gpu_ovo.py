"""One-vs-one multiclass on the GPU (Section 5 trains its multiclass sets
one against one) against the oracle's pairs and voting."""
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


@pytest.fixture(scope="module")
def fitted(sp):
    p = synth.gaussian_mixture(n=1600, d=8, components=4, seed=21, lam=1e-3, budget=64)
    cls = p.meta["components"].astype(np.int64)
    X = torch.from_numpy(p.X).cuda()
    kw = dict(precision="fp32", candidates=64, add_per_round=32, seed=5)
    models, st = sp.spsvm_fit_ovo(X, cls, 4, p.gamma, p.lam, 64, 1e-8, workers=3, **kw)
    return dict(p=p, cls=cls, X=X, models=models, st=st, kw=kw)


def test_pairs_are_the_class_pairs(sp, fitted):
    """Pair (a, b) is the binary problem on the rows of classes a (+1) and b
    (-1) in X order: the batch's model equals a fit of exactly that problem
    alone (the batch reproduces a lone fit bit for bit)."""
    p, cls, models = fitted["p"], fitted["cls"], fitted["models"]
    assert fitted["st"] == [0] * 6 and len(models) == 6
    for k in (0, 5):
        a, b = O.ovo_pairs(4)[k]
        rows = np.flatnonzero((cls == a) | (cls == b))
        y = np.where(cls[rows] == a, 1.0, -1.0).astype(np.float32)
        alone = sp.spsvm_fit(torch.from_numpy(p.X[rows]).cuda(), torch.from_numpy(y).cuda(),
                             p.gamma, p.lam, 64, 1e-8, **fitted["kw"])
        Ja, ba = alone.basis_and_beta()
        Jb, bb = models[k].basis_and_beta()
        np.testing.assert_array_equal(Ja, Jb)
        np.testing.assert_array_equal(ba, bb)


def test_votes_match_oracle(sp, fitted):
    """Three checks.  (1) Every pair's GPU decision value has the oracle's
    sign (float64, direct differences, from the GPU model's basis and
    coefficients) wherever the oracle value is outside the FP32 prediction
    error, 1e-5 of sum |beta|; in one-vs-one many values are near 0 (a query
    far from both classes of a pair).  (2) The GPU's vote counts and labels
    are exactly the oracle's voting rule applied to the GPU's own pair
    decisions.  (3) Labels equal the all-oracle labels wherever the votes of
    the unsure pairs cannot change the winner."""
    p, cls, models = fitted["p"], fitted["cls"], fitted["models"]
    Xq = synth.queries_like(p, 500, seed=3)
    Xqd = torch.from_numpy(Xq).cuda()
    lab, votes = sp.spsvm_predict_ovo(models, 4, Xqd, votes=True)
    lab, votes = lab.cpu().numpy(), votes.cpu().numpy()
    dec_gpu, dec_ref = [], []
    unsure = np.zeros(len(Xq), dtype=np.int64)
    for k, (a, b) in enumerate(O.ovo_pairs(4)):
        rows = np.flatnonzero((cls == a) | (cls == b))
        J, beta = models[k].basis_and_beta()
        f = O.predict(Xq, p.X[rows][J], beta, p.gamma)
        g = sp.spsvm_predict(models[k], Xqd).cpu().numpy().astype(np.float64)
        sure = np.abs(f) > 1e-5 * np.abs(beta).sum()
        np.testing.assert_array_equal(g[sure] >= 0, f[sure] >= 0)
        unsure += ~sure
        dec_gpu.append(g)
        dec_ref.append(f)
    gl, gv = O.ovo_vote(np.stack(dec_gpu), 4)
    np.testing.assert_array_equal(votes, gv)
    np.testing.assert_array_equal(lab, gl)
    rl, rv = O.ovo_vote(np.stack(dec_ref), 4)
    top2 = np.sort(rv, axis=1)[:, -2:]
    robust = (top2[:, 1] - top2[:, 0]) > 2 * unsure
    assert robust.mean() > 0.9
    np.testing.assert_array_equal(lab[robust], rl[robust])


def test_ovo_argument_errors(sp):
    X = torch.zeros((6, 2), device="cuda")
    with pytest.raises(sp.SpsvmError):
        sp.spsvm_fit_ovo(X, [0, 0, 1, 1, 2, 2], 1, 1.0, 1e-3, 2)
    with pytest.raises(sp.SpsvmError):   # class 2 absent
        sp.spsvm_fit_ovo(X, [0, 0, 1, 1, 1, 1], 3, 1.0, 1e-3, 2)
    with pytest.raises(sp.SpsvmError):   # label out of range
        sp.spsvm_fit_ovo(X, [0, 0, 1, 1, 5, 1], 3, 1.0, 1e-3, 2)
