"""Row-sharded fit (Section 4, Eq. 4 over W processes): every sum over points
is a per-rank partial reduced by all-reduce.  Two gloo ranks on the CPU, an
uneven split of the rows, per-rank partials computed by the float64 oracle
over each rank's own rows; the reduced Newton system, gradient, right-hand
side, line-search step and selection scores, and a whole fit of three growth
rounds, must equal the single-process oracle."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import spsvm as O
from paper_1404_1066_gb300 import sharded as SH

N, D, LAM, GAMMA = 301, 6, 1e-3, 0.4
BASIS = [3, 17, 40, 41, 99, 150, 151, 152, 200, 233, 260, 299, 300, 5, 77, 123]


def _data():
    g = np.random.default_rng(41)
    X = g.standard_normal((N, D))
    y = np.where(X[:, 0] - 0.5 * X[:, 1] + 0.3 * g.standard_normal(N) > 0, 1.0, -1.0)
    beta = 0.3 * g.standard_normal(len(BASIS))
    return X, y, beta


class OracleShard:
    """The Shard protocol over rows [lo, hi), every sum from the oracle's
    float64 arithmetic on those rows only."""

    def __init__(self, X, y, lo, hi):
        self.X, self.y, self.lo, self.hi = X[lo:hi], y[lo:hi], lo, hi
        self.K = np.zeros((hi - lo, 0))

    def rows(self, idx):
        return self.X[np.asarray(idx) - self.lo]

    def kernel(self, A, B):
        return O.rbf_kernel(A, B, GAMMA)

    def extend(self, XJ_new):
        self.K = np.hstack([self.K, O.rbf_kernel(self.X, XJ_new, GAMMA)])

    def outputs(self, beta):
        return self.K @ beta

    def image(self, d):
        return self.K @ d

    def newton_parts(self, o):
        S = O.active_set(self.y, o)
        KS = self.K[S]
        return KS.T @ KS, KS.T @ (o[S] - self.y[S]), KS.T @ self.y[S]

    def score_parts(self, Xc, o):
        S = O.active_set(self.y, o)
        Kc = O.rbf_kernel(self.X, Xc, GAMMA)
        return Kc.T @ np.where(S, o - self.y, 0.0), np.sum(Kc[S] ** 2, axis=0)

    def factor(self, H, level):
        L, lv = O.jittered_cholesky(H, level)
        return (lambda b: O.cholesky_solve(L, b)), lv

    def draw(self, n, J, kappa, seed, round_index):
        return O.draw_candidates(n, J, kappa, seed, round_index)


def _steps(comm, X, y, beta):
    """One rank's side of the step-level checks."""
    lo, hi = SH.row_range(N, comm.world, comm.rank)
    sh = OracleShard(X, y, lo, hi)
    XJ = SH.gather_rows(comm, sh, BASIS, D)
    sh.extend(XJ)
    KJJ = O.rbf_kernel(XJ, XJ, GAMMA)
    o = sh.outputs(beta)
    H, g, r, nS = SH.newton_system(comm, sh, o, beta, KJJ, LAM)
    d = O.newton_solve(H, r)[0] - beta
    u = sh.image(d)
    t = SH.line_search(comm, LAM * d @ (KJJ @ beta), LAM * d @ (KJJ @ d), 1.0 - sh.y * o, sh.y * u)
    cand = O.draw_candidates(N, BASIS, 40, 7, 0)
    Xc = SH.gather_rows(comm, sh, cand, D)
    delta, gc, hc = SH.score(comm, sh, Xc, o, O.rbf_kernel(Xc, XJ, GAMMA) @ beta,
                             np.ones(len(cand)), LAM)
    return dict(lo=lo, hi=hi, XJ=XJ, H=H, g=g, r=r, nS=nS, d=d, t=t, cand=cand, delta=delta,
                gc=gc, hc=hc)


def _whole_fit(comm, X, y):
    lo, hi = SH.row_range(N, comm.world, comm.rank)
    J, beta, o, st = SH.fit(comm, OracleShard(X, y, lo, hi), N, D, LAM, budget=48, tol=1e-10,
                            kappa=64, q=16, max_newton=50, seed=11)
    return dict(J=J, beta=beta, o=o, status=st)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, y, beta = _data()
        comm = SH.Comm()
        out.put((rank, _steps(comm, X, y, beta), _whole_fit(comm, X, y)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.fixture(scope="module")
def two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(2)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) /
                 max(1.0, float(np.max(np.abs(np.asarray(b))))))


def test_row_range_partition():
    for n, w in [(301, 2), (10, 3), (7, 7), (5, 8), (0, 2)]:
        rs = [SH.row_range(n, w, r) for r in range(w)]
        assert rs[0][0] == 0 and rs[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        sizes = [hi - lo for lo, hi in rs]
        assert max(sizes) - min(sizes) <= 1


def test_reduced_newton_system_equals_one_process(two_ranks):
    X, y, beta = _data()
    (_, s0, _), (_, s1, _) = two_ranks
    assert (s0["lo"], s0["hi"], s1["lo"], s1["hi"]) == (0, 151, 151, 301)
    for k in ("H", "g", "r", "d", "XJ"):
        assert np.array_equal(s0[k], s1[k]), k     # replicated: identical on the ranks
    KnJ = O.rbf_kernel(X, X[BASIS], GAMMA)
    KJJ = KnJ[BASIS]
    o = KnJ @ beta
    S = O.active_set(y, o)
    assert np.array_equal(s0["XJ"], X[BASIS])
    assert _rel(s0["H"], O.hessian(beta, KnJ, KJJ, y, LAM)) <= 1e-13
    assert _rel(s0["g"], O.gradient(beta, KnJ, KJJ, y, LAM)) <= 1e-13
    assert _rel(s0["r"], KnJ[S].T @ y[S]) <= 1e-13
    assert s0["nS"] == int(S.sum())


def test_reduced_line_search_and_scores_equal_one_process(two_ranks):
    X, y, beta = _data()
    (_, s0, _), (_, s1, _) = two_ranks
    KnJ = O.rbf_kernel(X, X[BASIS], GAMMA)
    KJJ = KnJ[BASIS]
    o = KnJ @ beta
    d = s0["d"]
    t_ref = O.line_search(beta, d, o, KnJ @ d, y, KJJ, LAM)
    assert s0["t"] == s1["t"]
    assert s0["t"] == pytest.approx(t_ref, rel=1e-12, abs=1e-15)
    assert np.array_equal(s0["cand"], s1["cand"])
    dref, gref, href = O.score_candidates(X, y, BASIS, beta, o, s0["cand"], GAMMA, LAM)
    assert _rel(s0["gc"], gref) <= 1e-13 and _rel(s0["hc"], href) <= 1e-13
    assert np.allclose(s0["delta"], dref, rtol=1e-12, atol=0)
    assert np.array_equal(SH.select_top(s0["delta"], s0["cand"], 8),
                          O.select_top(dref, s0["cand"], 8))


def test_sharded_fit_equals_one_process(two_ranks):
    X, y, _ = _data()
    (_, _, f0), (_, _, f1) = two_ranks
    assert np.array_equal(f0["J"], f1["J"]) and np.array_equal(f0["beta"], f1["beta"])
    ref = O.fit(X, y, GAMMA, LAM, 48, tol=1e-10, kappa=64, q=16, max_newton=50, seed=11)
    assert np.array_equal(f0["J"], ref.J)
    assert np.linalg.norm(f0["beta"] - ref.beta) <= 1e-9 * np.linalg.norm(ref.beta)
    o = np.concatenate([f0["o"], f1["o"]])
    assert _rel(o, ref.o) <= 1e-9
    assert f0["status"] == f1["status"] == ref.status


@pytest.mark.parametrize("ties", [False, True])
def test_line_search_brackets_like_the_breakpoint_walk(ties):
    """The grid bracketing (one process) against the oracle's sorted walk
    over the breakpoints, on terms with many pieces, and with groups of
    equal breakpoints."""
    g = np.random.default_rng(5 + ties)
    n = 4000
    y = np.where(g.random(n) < 0.5, 1.0, -1.0)
    o = y * (1.0 + 0.8 * g.standard_normal(n))   # about 40% active at t = 0
    # mostly descending margins (v = y u > 0 for 80%): the root lies past
    # hundreds of breakpoints, inside (0, 1)
    u = y * np.where(g.random(n) < 0.8, 1.0, -1.0) * np.abs(g.standard_normal(n))
    if ties:   # blocks of points with the same (o, u): equal breakpoints
        o = np.repeat(o[: n // 8], 8)
        u = np.repeat(u[: n // 8], 8)
        y = np.repeat(y[: n // 8], 8)
    KJJ = np.eye(1)
    for b, dd in [(0.7, -2.0), (-0.2, 0.5), (0.0, 1.0)]:
        beta, d = np.array([b]), np.array([dd])
        t_ref = O.line_search(beta, d, o, u, y, KJJ, LAM)
        t = SH.line_search(SH.Comm(), LAM * dd * b, LAM * dd * dd, 1.0 - y * o, y * u)
        assert 0.0 < t_ref < 1.0
        assert t == pytest.approx(t_ref, rel=1e-12, abs=1e-15)
