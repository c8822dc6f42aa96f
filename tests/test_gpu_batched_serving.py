"""Batched fits and the serving loop: every result must be the same as the
same problem fitted alone (fixed reduction order, no cross-problem
arithmetic), whatever else runs beside it; admission by HBM footprint."""
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


def _grid(n=8000, d=32, count=6, seed=21):
    g = np.random.default_rng(seed)
    base = synth.gaussian_mixture(n=n, d=d, budget=64, seed=seed)
    comp = base.meta["components"]
    probs = []
    for k in range(count):
        ns = int(g.integers(1500, 4000))
        rows = np.sort(g.choice(n, size=ns, replace=False)).astype(np.int64)
        y = np.where(comp[rows] == k % 10, 1.0, -1.0).astype(np.float32)
        probs.append(dict(rows=rows, y=y, gamma=[0.5, 1.0, 2.0][k % 3] / d,
                          lam=[1e-3, 1e-4][k % 2], budget=64 * int(g.integers(1, 4)),
                          tol=1e-6, seed=100 + k))
    return base.X, probs


@pytest.mark.parametrize("prec", ["fp32", "bf16split"])
def test_batched_equals_alone(sp, prec):
    X, probs = _grid()
    Xd = torch.from_numpy(X).cuda()
    opts = dict(precision=prec, candidates=128, add_per_round=64)
    models, st = sp.spsvm_fit_batched(Xd, probs, workers=3, **opts)
    # OK, or the Newton step limit (the model is still returned)
    assert all(s in (0, -4) for s in st), st
    Xq = torch.from_numpy(X[:1000].copy()).cuda()
    for p, m in zip(probs, models):
        Xs = torch.from_numpy(X[p["rows"]].copy()).cuda()
        ys = torch.from_numpy(p["y"]).cuda()
        alone = sp.spsvm_fit(Xs, ys, p["gamma"], p["lam"], p["budget"], p["tol"], seed=p["seed"],
                             **opts)
        assert alone.status == m.status
        Ja, ba = alone.basis_and_beta()
        Jb, bb = m.basis_and_beta()
        np.testing.assert_array_equal(Ja, Jb)
        np.testing.assert_array_equal(ba, bb)
        np.testing.assert_array_equal(alone.predict(Xq).cpu().numpy(), m.predict(Xq).cpu().numpy())


def test_batched_problem_matches_oracle(sp):
    X, probs = _grid(count=2)
    p = probs[1]
    Xd = torch.from_numpy(X).cuda()
    models, st = sp.spsvm_fit_batched(Xd, [p], workers=1, precision="fp32", candidates=128,
                                      add_per_round=64, record=True)
    m = models[0]
    info = m.info()
    rep = [dict(zip(("candidates", "chosen"), m.round(k))) for k in range(info["rounds"])]
    Xs = X[p["rows"]]
    r = O.fit(Xs, p["y"], p["gamma"], p["lam"], p["budget"], tol=1e-10, kappa=128, q=64,
              seed=p["seed"], replay=rep, replay_rtol=1e-4)
    Xq = Xs[:500]
    f = m.predict(torch.from_numpy(Xq.copy()).cuda()).cpu().numpy().astype(np.float64)
    J, _ = m.basis_and_beta()
    ref = O.predict(Xq, Xs[J], r.beta, p["gamma"])
    assert np.max(np.abs(f - ref) / np.maximum(1, np.abs(ref))) <= 1e-4


def test_server_mix_equals_alone(sp):
    X, probs = _grid(count=4, seed=33)
    # budget fits about two of these requests at a time, so the rest queue
    one = sp.spsvm_fit_workspace_bytes(4000, 32, 192, sp.make_options(candidates=128)[0])
    srv = sp.Server(hbm_budget_bytes=int(2.2 * one), workers=3)
    Xq = X[:700].copy()
    fit_ids, pred_ids = [], []
    for p in probs:
        fid = srv.submit_fit(X[p["rows"]], p["y"], p["gamma"], p["lam"], p["budget"], p["tol"],
                             candidates=128, add_per_round=64, seed=p["seed"])
        fit_ids.append(fid)
        pred_ids.append(srv.submit_predict(fid, Xq))
    lat = []
    for fid, pid in zip(fit_ids, pred_ids):
        st, l1 = srv.wait(fid, 120.0)
        assert st == 0
        st, l2 = srv.wait(pid, 120.0)
        assert st == 0
        lat += [l1, l2]
    assert all(v > 0 for v in lat)
    s = srv.stats()
    assert s["done"] == 8 and s["queued"] == 0
    # the budget held while the workers kept their buffers and the models
    # stayed resident; the models' bytes are counted until released
    assert s["hbm_peak"] <= int(2.2 * one)
    mb = [srv.model(f).device_bytes() for f in fit_ids]
    assert all(b > 0 for b in mb)
    assert s["hbm_in_use"] >= sum(mb)
    for f in fit_ids:
        srv.release(f)
    assert srv.stats()["hbm_in_use"] == s["hbm_in_use"] - sum(mb)
    for p, pid in zip(probs, pred_ids):
        Xs = torch.from_numpy(X[p["rows"]].copy()).cuda()
        ys = torch.from_numpy(p["y"]).cuda()
        alone = sp.spsvm_fit(Xs, ys, p["gamma"], p["lam"], p["budget"], p["tol"], seed=p["seed"],
                             candidates=128, add_per_round=64)
        ref = alone.predict(torch.from_numpy(Xq).cuda()).cpu().numpy()
        np.testing.assert_array_equal(srv.decision(pid), ref)
    srv.close()


def test_server_budget_holds_with_resident_models(sp):
    """A budget that admits one fit at a time: six fits run one after
    another on two workers, every model stays resident and counted, the peak
    never passes the budget, and a released model gives its bytes back."""
    X, probs = _grid(count=6, seed=35)
    one = sp.spsvm_fit_workspace_bytes(4000, 32, 192, sp.make_options(candidates=128)[0])
    budget = int(1.6 * one)
    srv = sp.Server(hbm_budget_bytes=budget, workers=2)
    ids = [srv.submit_fit(X[p["rows"]], p["y"], p["gamma"], p["lam"], p["budget"], p["tol"],
                          candidates=128, add_per_round=64, seed=p["seed"]) for p in probs]
    for f in ids:
        assert srv.wait(f, 120.0)[0] == 0
    s = srv.stats()
    assert s["hbm_peak"] <= budget
    mb = [srv.model(f).device_bytes() for f in ids]
    assert s["hbm_in_use"] >= sum(mb)
    srv.release(ids[0])
    assert srv.stats()["hbm_in_use"] == s["hbm_in_use"] - mb[0]
    with pytest.raises(sp.SpsvmError):   # its model is gone
        srv.submit_predict(ids[0], X[:10])
    pid = srv.submit_predict(ids[1], X[:10])
    assert srv.wait(pid, 60.0)[0] == 0
    srv.close()


def test_server_rejects_request_over_budget(sp):
    X, probs = _grid(count=1)
    p = probs[0]
    srv = sp.Server(hbm_budget_bytes=1 << 20, workers=1)
    with pytest.raises(sp.SpsvmError) as e:
        srv.submit_fit(X[p["rows"]], p["y"], p["gamma"], p["lam"], p["budget"])
    assert e.value.code == -2
    srv.close()
