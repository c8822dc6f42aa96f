"""Pins for the float64 oracle, against facts that do not come from the
oracle itself: hand-derived closed forms, published generator outputs,
library routines used as independent routes, finite differences and brute
force on tiny inputs.  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize
import scipy.spatial.distance

import oracle
from oracle import spsvm as O


def _blobs(n, d, seed, sep=1.0):
    g = np.random.default_rng(seed)
    y = np.where(g.random(n) < 0.5, 1.0, -1.0)
    X = g.standard_normal((n, d)) + sep * 0.5 * y[:, None]
    return X, y


# ---------------------------------------------------------------- kernel
def test_rbf_hand_values():
    # ||(0,0) - (3,4)||^2 = 25, gamma = 0.1 -> exp(-2.5)
    K = O.rbf_kernel(np.array([[0.0, 0.0]]), np.array([[3.0, 4.0], [0.0, 0.0]]), 0.1)
    assert K[0, 0] == pytest.approx(math.exp(-2.5), rel=1e-15)
    assert K[0, 1] == 1.0


def test_rbf_properties_and_library_route():
    g = np.random.default_rng(0)
    A = g.standard_normal((37, 9))
    K = O.rbf_kernel(A, A, 0.3)
    assert np.all(np.diag(K) == 1.0)
    np.testing.assert_allclose(K, K.T, rtol=0, atol=0)
    ref = np.exp(-0.3 * scipy.spatial.distance.cdist(A, A, "sqeuclidean"))
    np.testing.assert_allclose(K, ref, rtol=1e-13, atol=1e-15)
    # gamma -> 0: every entry -> 1
    np.testing.assert_allclose(O.rbf_kernel(A, A, 1e-12), 1.0, atol=1e-9)
    # positive semidefinite
    assert np.linalg.eigvalsh(K).min() > -1e-10


# ---------------------------------------------------------------- RNG
def test_splitmix64_published_vectors():
    # splitmix64 started from state 0 (Steele, Lea, Flood 2014; Vigna's
    # reference implementation): first three outputs.
    assert O.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert O.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert O.splitmix64(0, 2) == 0x06C45D188009454F


def test_draw_candidates_valid_and_deterministic():
    n = 1000
    J = [3, 17, 999, 0, 500]
    c = O.draw_candidates(n, J, 256, seed=42, round_index=3)
    assert len(c) == 256 and len(set(c.tolist())) == 256
    assert not (set(c.tolist()) & set(J))
    assert c.min() >= 0 and c.max() < n
    np.testing.assert_array_equal(c, O.draw_candidates(n, J, 256, 42, 3))
    assert not np.array_equal(c, O.draw_candidates(n, J, 256, 42, 4))
    # fewer points left than kappa: all of them
    c2 = O.draw_candidates(10, list(range(7)), 256, 1, 0)
    assert sorted(c2.tolist()) == [7, 8, 9]


def test_draw_candidates_uniform():
    # each of the n - |J| points equally likely to be drawn: chi-square
    n, kappa, R = 64, 8, 4000
    counts = np.zeros(n)
    for r in range(R):
        counts[O.draw_candidates(n, [5, 6], kappa, 7, r)] += 1
    assert counts[5] == 0 and counts[6] == 0
    cnt = np.delete(counts, [5, 6])
    exp = R * kappa / (n - 2)
    chi2 = np.sum((cnt - exp) ** 2 / exp)
    # 61 dof: 99.9% quantile ~ 100
    assert chi2 < 100


def test_select_top_ties_to_smaller_index():
    cand = np.array([40, 7, 12, 3])
    delta = np.array([1.0, 2.0, 2.0, 0.5])
    np.testing.assert_array_equal(O.select_top(delta, cand, 3), [7, 12, 40])


# ------------------------------------------------- objective derivatives
def _setup(n=60, d=4, m=9, seed=1, lam=0.05, gamma=0.4, scale=1.0):
    X, y = _blobs(n, d, seed)
    J = np.arange(0, n, n // m)[:m]
    KnJ = O.rbf_kernel(X, X[J], gamma)
    KJJ = KnJ[J]
    beta = scale * np.random.default_rng(seed + 1).standard_normal(m)
    return X, y, J, KnJ, KJJ, beta, lam, gamma


def test_gradient_matches_central_differences():
    X, y, J, KnJ, KJJ, beta, lam, _ = _setup()
    o = KnJ @ beta
    assert np.min(np.abs(1 - y * o)) > 1e-3   # no point on the kink
    g = O.gradient(beta, KnJ, KJJ, y, lam)
    h = 1e-6
    fd = np.array([(O.objective(beta + h * e, KnJ, KJJ, y, lam)
                    - O.objective(beta - h * e, KnJ, KJJ, y, lam)) / (2 * h)
                   for e in np.eye(len(beta))])
    np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-8)


def test_hessian_matches_differences_of_gradient():
    X, y, J, KnJ, KJJ, beta, lam, _ = _setup(seed=3)
    H = O.hessian(beta, KnJ, KJJ, y, lam)
    h = 1e-7
    fd = np.array([(O.gradient(beta + h * e, KnJ, KJJ, y, lam)
                    - O.gradient(beta - h * e, KnJ, KJJ, y, lam)) / (2 * h)
                   for e in np.eye(len(beta))]).T
    np.testing.assert_allclose(H, fd, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(H, H.T, atol=0)


# ------------------------------------------------- Newton closed form
def test_all_active_newton_step_is_regularised_least_squares():
    # lambda large keeps |o| small, so every point stays active (y o < 1):
    # f is then the quadratic lambda/2 b'K_JJ b + 1/2||K_nJ b - y||^2 and one
    # Newton step from 0 lands on (lambda K_JJ + K^T K)^{-1} K^T y.
    X, y, J, KnJ, KJJ, _, _, _ = _setup(n=80, m=12, seed=5)
    lam = 50.0
    hist = []
    beta, o, status = O.newton(KnJ, KJJ, y, lam, np.zeros(len(J)), 1e-12, 5, hist)
    assert np.all(y * o < 1)
    # independent route: least squares on [K_nJ; sqrt(lam) K_JJ^{1/2}] by SVD
    w, V = np.linalg.eigh(KJJ)
    root = (V * np.sqrt(np.maximum(w, 0))) @ V.T
    A = np.vstack([KnJ, math.sqrt(lam) * root])
    b = np.concatenate([y, np.zeros(len(J))])
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    np.testing.assert_allclose(beta, ref, rtol=1e-9, atol=1e-11)
    assert hist[0]["t"] == 1.0


def test_two_point_closed_form():
    # x1=(0,0) y=+1, x2=(1,0) y=-1, gamma=1: K = [[1,k],[k,1]], k = e^-1.
    # By symmetry beta = (b,-b); f = lam b^2 (1-k) + (1 - b(1-k))^2, whose
    # minimiser is b = 1/(lam + 1 - k).
    X = np.array([[0.0, 0.0], [1.0, 0.0]])
    y = np.array([1.0, -1.0])
    lam = 0.5
    r = O.fit(X, y, 1.0, lam, 2, tol=1e-14, initial_basis=[0, 1], grow=False)
    b = 1.0 / (lam + 1.0 - math.exp(-1.0))
    np.testing.assert_allclose(r.beta, [b, -b], rtol=1e-13)


# ------------------------------------------------- optimum with J = all
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_full_basis_matches_bruteforce_dual(seed):
    X, y = _blobs(10, 2, seed, sep=0.8)
    gamma, lam = 0.7, 0.05
    r = O.fit(X, y, gamma, lam, 10, tol=1e-13, initial_basis=list(range(10)),
              grow=False, max_newton=100)
    K = O.rbf_kernel(X, X, gamma)
    alpha, beta_dual = oracle.squared_hinge_dual_bruteforce(K, y, lam)
    scale = np.abs(beta_dual).max()
    np.testing.assert_allclose(r.beta, beta_dual, rtol=1e-8, atol=1e-10 * scale)
    np.testing.assert_allclose(K @ r.beta, K @ beta_dual, atol=1e-10)
    # KKT fixed point of the primal: lam beta_i = y_i max(0, 1 - y_i o_i)
    o = K @ r.beta
    np.testing.assert_allclose(lam * r.beta, y * np.maximum(0, 1 - y * o), atol=1e-10 * max(1, lam * scale))


def test_golden_xor_dual():
    # Stored brute-force dual solution of a 4-point XOR problem; written by
    # tests/golden/make_golden.py (calls only the oracle's dual route).
    import json, os
    path = os.path.join(os.path.dirname(__file__), "golden", "xor4.json")
    G = json.load(open(path))
    X = np.array(G["X"]); y = np.array(G["y"])
    r = O.fit(X, y, G["gamma"], G["lam"], 4, tol=1e-14, initial_basis=[0, 1, 2, 3],
              grow=False)
    np.testing.assert_allclose(r.beta, G["beta"], rtol=1e-12)
    # XOR symmetry: all |beta_i| equal, signs follow the labels
    np.testing.assert_allclose(np.abs(r.beta), abs(r.beta[0]), rtol=1e-12)
    np.testing.assert_array_equal(np.sign(r.beta), y)


# ------------------------------------------------- line search
@pytest.mark.parametrize("seed", range(5))
def test_line_search_is_exact_minimiser(seed):
    X, y, J, KnJ, KJJ, beta, lam, _ = _setup(n=120, m=10, seed=10 + seed, lam=0.01)
    g = np.random.default_rng(seed)
    d = g.standard_normal(len(J)) * 2.0
    o = KnJ @ beta
    u = KnJ @ d
    if O.line_search_derivative(0.0, beta, d, o, u, y, KJJ, lam) > 0:
        d, u = -d, -u
    t = O.line_search(beta, d, o, u, y, KJJ, lam)
    phi = lambda s: O.objective(beta + s * d, KnJ, KJJ, y, lam)
    # derivative vanishes at t (phi is C^1)
    dt = O.line_search_derivative(t, beta, d, o, u, y, KJJ, lam)
    scale = abs(O.line_search_derivative(0.0, beta, d, o, u, y, KJJ, lam))
    assert abs(dt) <= 1e-9 * scale
    # brute force: dense grid then bounded scalar minimisation
    grid = np.linspace(0, 4 * max(t, 1.0), 4001)
    k = int(np.argmin([phi(s) for s in grid]))
    lo, hi = grid[max(0, k - 1)], grid[min(len(grid) - 1, k + 1)]
    ref = scipy.optimize.minimize_scalar(phi, bounds=(lo, hi), method="bounded",
                                         options=dict(xatol=1e-12)).x
    assert phi(t) <= phi(ref) + 1e-12 * abs(phi(ref))
    assert t == pytest.approx(ref, rel=1e-5, abs=1e-8)


def test_line_search_full_step_on_quadratic_piece():
    X, y, J, KnJ, KJJ, _, _, _ = _setup(n=80, m=12, seed=5)
    lam = 50.0
    beta = np.zeros(len(J))
    o = KnJ @ beta
    H = lam * KJJ + KnJ.T @ KnJ
    d = np.linalg.solve(H, KnJ.T @ y)
    t = O.line_search(beta, d, o, KnJ @ d, y, KJJ, lam)
    assert t == 1.0


# ------------------------------------------------- basis-vector score
def test_score_derivatives_and_exact_decrease():
    # g_c, h_c are df/dbeta_c and d2f/dbeta_c^2 at beta_c = 0; when no
    # point crosses the margin along the 1-D path, f is quadratic in beta_c
    # and the best decrease is exactly g_c^2 / (2 h_c).
    X, y = _blobs(50, 3, 8)
    gamma, lam = 0.5, 40.0
    J = [0, 5, 9]
    KnJ = O.rbf_kernel(X, X[J], gamma)
    beta, o, _ = O.newton(KnJ, KnJ[J], y, lam, np.zeros(3), 1e-12, 20)
    cand = np.array([11, 23, 37])
    delta, g, h = O.score_candidates(X, y, J, beta, o, cand, gamma, lam)
    for k, c in enumerate(cand):
        Jc = J + [int(c)]
        Kc = O.rbf_kernel(X, X[Jc], gamma)
        f1 = lambda b: O.objective(np.concatenate([beta, [b]]), Kc, Kc[Jc], y, lam)
        e = 1e-5
        assert g[k] == pytest.approx((f1(e) - f1(-e)) / (2 * e), rel=1e-6, abs=1e-9)
        assert h[k] == pytest.approx((f1(e) - 2 * f1(0) + f1(-e)) / e ** 2, rel=1e-4)
        bstar = -g[k] / h[k]
        oc = Kc @ np.concatenate([beta, [bstar]])
        assert np.all(y * oc < 1) and np.all(y * o < 1)
        assert f1(0) - f1(bstar) == pytest.approx(delta[k], rel=1e-9)
        res = scipy.optimize.minimize_scalar(f1, bracket=(-1, 1), tol=1e-12)
        assert f1(0) - res.fun == pytest.approx(delta[k], rel=1e-7)


# ------------------------------------------------- whole fit
def test_fit_monotone_and_converged_fixed_basis():
    X, y = _blobs(300, 5, 21, sep=1.0)
    r = O.fit(X, y, 0.2, 1e-3, 40, tol=1e-10, initial_basis=list(range(0, 300, 7))[:40],
              grow=False, max_newton=100)
    objs = [h["objective"] for h in r.history if h["step"]]
    assert len(objs) >= 2
    for a, b in zip(objs, objs[1:]):
        assert b <= a * (1 + 1e-12)
    KnJ = O.rbf_kernel(X, X[r.J], 0.2)
    assert np.linalg.norm(O.gradient(r.beta, KnJ, KnJ[r.J], y, 1e-3)) <= 1e-9
    assert r.status in ("tol", "repeat")


def test_fit_growth_rounds():
    X, y = _blobs(400, 4, 22, sep=1.2)
    r = O.fit(X, y, 0.25, 1e-3, 48, tol=1e-10, kappa=32, q=16, seed=9)
    assert len(r.J) == 48 and len(set(r.J.tolist())) == 48
    assert len(r.rounds) == 3
    # each round's chosen points are the top-q of its candidates by score
    for rd in r.rounds:
        d = rd["delta"]
        chosen_scores = [d[list(rd["candidates"]).index(c)] for c in rd["chosen"]]
        assert min(chosen_scores) >= np.sort(d)[::-1][len(rd["chosen"]) - 1]
    # objective at the end of every round decreases as the basis grows
    ends = []
    last = None
    for h in r.history:
        if last is not None and h["basis"] != last["basis"]:
            ends.append(last["objective"])
        last = h
    ends.append(last["objective"])
    assert all(b <= a * (1 + 1e-12) for a, b in zip(ends, ends[1:]))
    # training accuracy well above chance on separable-ish blobs
    assert np.mean(O.labels(r.o) == y) > 0.8


def test_growth_stop_rule():
    """Section 4's growth stop: after each round, stop when the drop in the
    training error rate divided by the number of vectors added falls below
    epsilon.  The rate starts at 1 (at beta = 0 every y_i o_i = 0 counts as
    an error).  A run to budget fixes the per-round rates; for each epsilon
    the stopped run must end at the first round whose drop per vector is
    below it, with the budget run's basis up to there."""
    X, y = _blobs(400, 4, 22, sep=1.2)
    full = O.fit(X, y, 0.25, 1e-3, 96, tol=1e-10, kappa=32, q=16, seed=9)
    E = [1.0] + [rd["error_rate"] for rd in full.rounds]
    # the last recorded rate is the training error of the final decision values
    dec_vals = O.predict(X, X[full.J], full.beta, 0.25)
    assert E[-1] == np.mean(y * dec_vals <= 0)
    drop = [(E[k] - E[k + 1]) / 16 for k in range(len(full.rounds))]
    stops = set()
    for eps in (1.0, 1e-3, 5e-4, 1e-9):
        want = next((k + 1 for k, d in enumerate(drop) if d < eps), len(drop))
        stops.add(want)
        r = O.fit(X, y, 0.25, 1e-3, 96, tol=1e-10, kappa=32, q=16, seed=9, growth_tol=eps)
        assert len(r.rounds) == want
        np.testing.assert_array_equal(r.J, full.J[:16 * want])
    assert len(stops) >= 3   # the epsilons exercise different rounds


def _score_case(seed, n=60, d=3, m=5, lam=1e-2, gamma=0.4):
    X, y = _blobs(n, d, seed, sep=0.8)
    g = np.random.default_rng(seed)
    J = list(g.choice(n, m, replace=False))
    KnJ = O.rbf_kernel(X, X[J], gamma)
    beta = 0.3 * g.standard_normal(m)
    o = KnJ @ beta
    cand = np.array([c for c in range(n) if c not in J][:12])
    return X, y, J, beta, o, cand, gamma, lam


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_exact_score_is_the_one_dimensional_minimum(seed):
    """Delta_c of the exact score equals f(beta) minus the minimum of f over a
    fine grid of the new coefficient (brute force, refined around the best
    grid point), and is never below the heuristic's prediction evaluated on
    the true objective at the heuristic's step -g_c / h_c."""
    X, y, J, beta, o, cand, gamma, lam = _score_case(seed)
    dex, tex = O.score_candidates_exact(X, y, J, beta, o, cand, gamma, lam)
    _, g, h = O.score_candidates(X, y, J, beta, o, cand, gamma, lam)
    for k, c in enumerate(cand):
        Ja = J + [int(c)]
        KnJa = O.rbf_kernel(X, X[Ja], gamma)
        KJJa = KnJa[Ja]
        ba = np.concatenate([beta, [0.0]])

        def f(t):
            b = ba.copy()
            b[-1] = t
            return O.objective(b, KnJa, KJJa, y, lam)

        f0 = f(0.0)
        grid = np.linspace(-20.0, 20.0, 4001)
        vals = np.array([f(t) for t in grid])
        t0 = grid[np.argmin(vals)]
        fine = np.linspace(t0 - 0.01, t0 + 0.01, 2001)
        best = min(f(t) for t in fine)
        assert dex[k] >= -1e-14
        assert abs((f0 - best) - dex[k]) <= 1e-9 * max(1.0, f0)
        assert abs(f(tex[k]) - best) <= 1e-9 * max(1.0, f0)
        assert dex[k] >= f0 - f(-g[k] / h[k]) - 1e-12 * max(1.0, f0)


def test_exact_score_with_bias_is_the_one_dimensional_minimum():
    """With a bias b carried by o the exact score's decrease equals f(beta, b)
    minus the minimum over the new coefficient of the bias-aware objective
    lambda/2 beta^T K_JJ beta + 1/2 sum max(0, 1 - y (K beta + b))^2 (brute
    force on a grid refined around its best point)."""
    X, y, J, beta, o, cand, gamma, lam = _score_case(5)
    b = 0.37
    o = o + b
    dex, tex = O.score_candidates_exact(X, y, J, beta, o, cand, gamma, lam)
    for k, c in enumerate(cand[:6]):
        Ja = J + [int(c)]
        KnJa = O.rbf_kernel(X, X[Ja], gamma)
        KJJa = KnJa[Ja]

        def f(t):
            ba = np.concatenate([beta, [t]])
            oo = KnJa @ ba + b
            return 0.5 * lam * ba @ (KJJa @ ba) + 0.5 * np.sum(np.maximum(0.0, 1.0 - y * oo) ** 2)

        grid = np.linspace(-20.0, 20.0, 4001)
        t0 = grid[np.argmin([f(t) for t in grid])]
        best = min(f(t) for t in np.linspace(t0 - 0.01, t0 + 0.01, 2001))
        assert abs((f(0.0) - best) - dex[k]) <= 1e-9 * max(1.0, f(0.0))
        assert abs(f(tex[k]) - best) <= 1e-9 * max(1.0, f(0.0))


def test_exact_score_equals_heuristic_without_margin_crossings():
    """With every point inside the margin before and after the step (a large
    lambda keeps the outputs near 0, so y o < 1 throughout), f along the new
    coefficient is one quadratic piece and its exact decrease is the
    heuristic's g^2 / (2 h)."""
    X, y, J, beta, o, cand, gamma, lam = _score_case(4, lam=5.0)
    beta = 0.01 * beta
    o = O.rbf_kernel(X, X[J], gamma) @ beta
    dex, tex = O.score_candidates_exact(X, y, J, beta, o, cand, gamma, lam)
    dh, g, h = O.score_candidates(X, y, J, beta, o, cand, gamma, lam)
    for k, c in enumerate(cand):
        after = o + tex[k] * O.rbf_kernel(X, X[[int(c)]], gamma)[:, 0]
        assert np.all(y * o < 1) and np.all(y * after < 1)
    np.testing.assert_allclose(dex, dh, rtol=1e-10, atol=1e-15)
    np.testing.assert_allclose(tex, -g / h, rtol=1e-9, atol=1e-15)


def test_bias_first_step_is_regularised_least_squares_with_intercept():
    """Eq. 4 with its bias b on a fixed basis J = all points, lambda large enough
    that every point stays active: one Newton step from (beta, b) = 0 is the
    minimiser of lambda/2 beta^T K beta + 1/2 ||K beta + b 1 - y||^2, here
    found independently as the least-squares solution of the stacked system
    [K 1; sqrt(lambda) R 0] z = [y; 0] with K = R^T R (SVD-based lstsq)."""
    X, y = _blobs(40, 3, 31, sep=0.3)
    gamma, lam = 0.5, 50.0
    K = O.rbf_kernel(X, X, gamma)
    r = O.fit(X, y, gamma, lam, 40, tol=1e-12, initial_basis=list(range(40)), grow=False,
              max_newton=1, bias=True)
    o = K @ r.beta + r.bias
    assert np.all(y * o < 1)   # still all active: the one step is the minimiser
    R = np.linalg.cholesky(K + 1e-12 * np.eye(40)).T
    A = np.block([[K, np.ones((40, 1))], [np.sqrt(lam) * R, np.zeros((40, 1))]])
    z = np.linalg.lstsq(A, np.concatenate([y, np.zeros(40)]), rcond=None)[0]
    np.testing.assert_allclose(r.beta, z[:40], rtol=1e-6, atol=1e-9)
    assert abs(r.bias - z[40]) <= 1e-8


def test_bias_kkt_at_the_optimum():
    """At a fitted optimum with bias the gradient of Eq. 4 vanishes in both
    parts: lambda K_JJ beta + K_SJ^T (o_S - y_S) = 0 and sum_{i in S} (o_i - y_i)
    = 0 (b is not regularised); and with labels all +1 and a huge lambda,
    beta -> 0 and b -> 1 (each max(0, 1 - b)^2 is minimised at b = 1)."""
    X, y = _blobs(150, 3, 32, sep=1.0)
    y = np.where(np.arange(150) % 3 == 0, -y, y)   # unbalanced, overlapping
    r = O.fit(X, y, 0.4, 1e-2, 24, tol=1e-12, kappa=32, q=8, seed=5, bias=True)
    KnJ = O.rbf_kernel(X, X[r.J], 0.4)
    o = KnJ @ r.beta + r.bias
    np.testing.assert_allclose(o, r.o, rtol=1e-10, atol=1e-12)
    S = y * o < 1
    gb = np.sum(o[S] - y[S])
    gbeta = 1e-2 * (KnJ[r.J] @ r.beta) + KnJ[S].T @ (o[S] - y[S])
    assert abs(gb) <= 1e-9 * S.sum() and np.linalg.norm(gbeta) <= 1e-9 * S.sum()
    assert abs(r.bias) > 1e-3   # the bias is used on unbalanced labels
    r1 = O.fit(X, np.ones(150), 0.4, 1e6, 8, tol=1e-14, kappa=16, q=8, seed=1, bias=True)
    assert np.max(np.abs(r1.beta)) <= 1e-5 and abs(r1.bias - 1.0) <= 1e-5


def test_ovo_pairs_and_hand_counted_votes():
    """One-vs-one voting on decision values counted by hand: three classes,
    pairs (0,1), (0,2), (1,2).  Query 0: 0 beats 1, 2 beats 0, 1 beats 2 --
    one vote each, the tie goes to class 0.  Query 1: 1, 2, 2 -> class 2.
    Query 2: 0, 0, 1 -> class 0 with two votes.  A decision of exactly 0
    votes for the first class of the pair."""
    assert O.ovo_pairs(3) == [(0, 1), (0, 2), (1, 2)]
    assert len(O.ovo_pairs(10)) == 45 and O.ovo_pairs(4)[3] == (1, 2)
    dec = np.array([[+1.0, -1.0, +0.5],
                    [-1.0, -1.0, +2.0],
                    [+1.0, -0.5, 0.0]])
    lab, votes = O.ovo_vote(dec, 3)
    np.testing.assert_array_equal(votes, [[1, 1, 1], [0, 1, 2], [2, 1, 0]])
    np.testing.assert_array_equal(lab, [0, 2, 0])


def test_ovo_two_classes_is_the_binary_machine():
    # with two classes one-vs-one is the binary SP-SVM: class 0 where f >= 0
    X, y = _blobs(120, 3, 40, sep=1.0)
    cls = np.where(y > 0, 0, 1)
    fitted = O.fit_ovo(X, cls, 2, 0.3, 1e-3, 16, tol=1e-10, kappa=24, q=8, seed=3)
    rows, r = fitted[0]
    np.testing.assert_array_equal(rows, np.arange(len(y)))
    Xq = X[:50] + 0.1
    lab, _ = O.predict_ovo(X, fitted, 2, Xq, 0.3)
    f = O.predict(Xq, X[r.J], r.beta, 0.3)
    np.testing.assert_array_equal(lab, np.where(f >= 0, 0, 1))


def test_ovo_separates_far_apart_classes():
    # three tight clusters far apart: every training point gets its class
    g = np.random.default_rng(8)
    centres = np.array([[0.0, 0.0], [6.0, 0.0], [0.0, 6.0]])
    cls = np.repeat(np.arange(3), 30)
    X = centres[cls] + 0.3 * g.standard_normal((90, 2))
    fitted = O.fit_ovo(X, cls, 3, 0.5, 1e-3, 12, tol=1e-10, kappa=20, q=6, seed=2)
    assert [len(rows) for rows, _ in fitted] == [60, 60, 60]
    lab, votes = O.predict_ovo(X, fitted, 3, X, 0.5)
    np.testing.assert_array_equal(lab, cls)
    assert np.all(votes.sum(axis=1) == 3)


def test_replay_adopts_other_choice_and_rejects_bad_one():
    X, y = _blobs(200, 3, 30)
    r = O.fit(X, y, 0.3, 1e-3, 32, tol=1e-10, kappa=24, q=16, seed=4)
    rep = [dict(candidates=rd["candidates"], chosen=rd["chosen"]) for rd in r.rounds]
    r2 = O.fit(X, y, 0.3, 1e-3, 32, tol=1e-10, kappa=24, q=16, seed=4, replay=rep)
    np.testing.assert_array_equal(r.J, r2.J)
    bad = [dict(candidates=rep[0]["candidates"],
                chosen=np.array(sorted(rep[0]["candidates"],
                                       key=lambda c: r.rounds[0]["delta"][list(rep[0]["candidates"]).index(c)])[:16]))]
    with pytest.raises(AssertionError):
        O.fit(X, y, 0.3, 1e-3, 16, tol=1e-10, kappa=24, q=16, seed=4, replay=bad)


def test_predict_and_sign_convention():
    X, y = _blobs(30, 2, 40)
    J = np.array([1, 4, 9])
    beta = np.array([0.5, -1.0, 2.0])
    Xq = np.random.default_rng(1).standard_normal((7, 2))
    f = O.predict(Xq, X[J], beta, 0.6)
    ref = np.exp(-0.6 * scipy.spatial.distance.cdist(Xq, X[J], "sqeuclidean")) @ beta
    np.testing.assert_allclose(f, ref, rtol=1e-13)
    np.testing.assert_array_equal(O.labels(np.array([0.0, -0.0, -1e-300, 2.0])), [1, 1, -1, 1])


def test_newton_solve_against_lu_and_breakdown():
    g = np.random.default_rng(3)
    A = g.standard_normal((20, 20))
    H = A @ A.T + 1e-3 * np.eye(20)
    r = g.standard_normal(20)
    x, lv = O.newton_solve(H, r)
    assert lv == -1
    np.testing.assert_allclose(x, scipy.linalg.solve(H, r), rtol=1e-8)
    with pytest.raises(O.NotPositiveDefinite):
        O.newton_solve(-np.eye(3), np.ones(3))


def test_newton_solve_jitter_levels_against_eigendecomposition():
    """A symmetric matrix with one eigenvalue at -3e-8 tr(H)/|J|: levels -1
    (none), 0, 1, 2 (shift 1e-8 tr/|J|) leave it indefinite, level 3 (1e-7)
    is the first that factorises; the solve must equal Q diag(1/(e + shift))
    Q^T r from the eigendecomposition.  A start level above the needed one
    is kept (the level never goes down within a fit)."""
    g = np.random.default_rng(11)
    m = 20
    Q, _ = np.linalg.qr(g.standard_normal((m, m)))
    e = np.arange(1.0, m + 1.0)
    e[-1] = 0.0
    e[-1] = -3e-8 * e.sum() / m
    H = (Q * e) @ Q.T
    H = 0.5 * (H + H.T)
    r = g.standard_normal(m)
    tr = np.trace(H)
    x, lv = O.newton_solve(H, r)
    assert lv == 3
    shift = 1e-7 * tr / m
    np.testing.assert_allclose(x, Q @ ((Q.T @ r) / (e + shift)), rtol=1e-6)
    x5, lv5 = O.newton_solve(H, r, 5)
    assert lv5 == 5
    np.testing.assert_allclose(x5, Q @ ((Q.T @ r) / (e + 1e-5 * tr / m)), rtol=1e-8)
    # a level beyond the last one is a breakdown
    with pytest.raises(O.NotPositiveDefinite):
        O.newton_solve(H - 1e-1 * tr / m * np.eye(m), r)


def test_newton_no_descent_raises_jitter(monkeypatch):
    """When the line search finds no descent (t = 0) along the Newton step,
    the jitter goes up one level and the step becomes the regularised Newton
    step -(H + 1e-10 tr(H)/|J| I)^{-1} grad f; the level is kept."""
    g = np.random.default_rng(17)
    X = g.standard_normal((60, 3))
    y = np.where(X[:, 0] + 0.3 * g.standard_normal(60) > 0, 1.0, -1.0)
    J = [0, 5, 9, 20]
    lam, gamma = 1e-2, 0.5
    KnJ = O.rbf_kernel(X, X[J], gamma)
    KJJ = KnJ[J]
    beta0 = np.zeros(len(J))
    real = O.line_search
    calls = []

    def first_fails(*a):
        calls.append(1)
        return 0.0 if len(calls) == 1 else real(*a)

    monkeypatch.setattr(O, "line_search", first_fails)
    hist, jit = [], [-1]
    beta1, _, _ = O.newton(KnJ, KJJ, y, lam, beta0, 1e-12, 1, hist, jit)
    assert jit == [0] and hist[0]["jitter"] == 0 and len(calls) == 2
    S = y * (KnJ @ beta0) < 1
    H = lam * KJJ + KnJ[S].T @ KnJ[S]
    grad = lam * KJJ @ beta0 + KnJ[S].T @ (KnJ[S] @ beta0 - y[S])
    d = -np.linalg.solve(H + 1e-10 * np.trace(H) / len(J) * np.eye(len(J)), grad)
    t = real(beta0, d, KnJ @ beta0, KnJ @ d, y, KJJ, lam)
    np.testing.assert_allclose(beta1, beta0 + t * d, rtol=1e-9)
