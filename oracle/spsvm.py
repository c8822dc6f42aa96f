"""Plain float64 SP-SVM, step by step, for checking the CUDA library.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.

Problem (Section 4, Eq. 4, with the bias dropped as Section 2 does and the
objective divided by C, lambda = 1/C, which leaves the minimiser unchanged):

    f(beta) = lambda/2 * beta^T K_JJ beta + 1/2 * sum_i max(0, 1 - y_i o_i)^2,
    o = K_nJ beta,   k(x, z) = exp(-gamma ||x - z||^2)   (Section 2, RBF).

J grows by the two-stage cycle of Section 4 ("Sparse primal optimization"):
basis-vector selection from a random candidate subset, scored by the
estimated loss reduction, then reoptimisation of Eq. 4 on the grown basis.

The paper does not print the score, the Newton step or a line search.  The
readings used here (all listed with the other readings in the design notes):
  * score of candidate c: the one-coordinate Newton estimate of the decrease
    in f from adding c with beta_c = 0, Delta_c = g_c^2 / (2 h_c), with
    g_c = lambda k_cJ beta + sum_{i in S} (o_i - y_i) K_ic and
    h_c = lambda K_cc + sum_{i in S} K_ic^2;
  * Newton step of the squared-hinge primal (Section 4, "Primal
    optimization": second-order method): on the active set
    S = {i : y_i o_i < 1}, beta_bar = (lambda K_JJ + K_SJ^T K_SJ)^{-1} K_SJ^T y_S;
  * exact line search along d = beta_bar - beta (f is convex and piecewise
    quadratic along any line), so f never increases;
  * candidate draw: kappa indices without replacement from the points not
    in J, by a partial Fisher-Yates shuffle driven by the counter-based
    splitmix64 generator (Steele, Lea, Flood 2014);
  * growth stop of Section 4: (change in training error rate) / (number of
    basis vectors added) < epsilon; zero epsilon runs to the budget.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

MASK64 = (1 << 64) - 1
SPLITMIX_GAMMA = 0x9E3779B97F4A7C15


class NotPositiveDefinite(RuntimeError):
    pass


# --------------------------------------------------------------------------
# Kernel (Section 2: k(x_i, x_j) = exp(-gamma ||x_i - x_j||^2))
# --------------------------------------------------------------------------
def rbf_kernel(A, B, gamma):
    """K[i, j] = exp(-gamma * sum_k (A[i,k] - B[j,k])^2), from direct
    differences in float64 (no norm expansion)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    n, m = A.shape[0], B.shape[0]
    K = np.empty((n, m))
    if n == 0 or m == 0:
        return K
    rows = max(1, int(4_000_000 // max(1, m * A.shape[1])))
    for r0 in range(0, n, rows):
        diff = A[r0:r0 + rows, None, :] - B[None, :, :]
        K[r0:r0 + rows] = np.exp(-gamma * np.sum(diff * diff, axis=2))
    return K


# --------------------------------------------------------------------------
# Objective, gradient, Hessian of Eq. 4 (divided by C)
# --------------------------------------------------------------------------
def objective(beta, KnJ, KJJ, y, lam):
    """f(beta) = lambda/2 beta^T K_JJ beta + 1/2 sum_i max(0, 1 - y_i o_i)^2."""
    o = KnJ @ beta
    xi = np.maximum(0.0, 1.0 - y * o)
    return 0.5 * lam * beta @ (KJJ @ beta) + 0.5 * np.sum(xi * xi)


def active_set(y, o):
    """S = {i : y_i o_i < 1} (strict inequality)."""
    return y * o < 1.0


def gradient(beta, KnJ, KJJ, y, lam):
    """grad f = lambda K_JJ beta + K_SJ^T (o_S - y_S)   (y_i^2 = 1)."""
    o = KnJ @ beta
    S = active_set(y, o)
    return lam * (KJJ @ beta) + KnJ[S].T @ (o[S] - y[S])


def hessian(beta, KnJ, KJJ, y, lam):
    """Generalised Hessian H = lambda K_JJ + K_SJ^T K_SJ on the current S."""
    o = KnJ @ beta
    S = active_set(y, o)
    KS = KnJ[S]
    return lam * KJJ + KS.T @ KS


# --------------------------------------------------------------------------
# Newton system (Cholesky in float64)
# --------------------------------------------------------------------------
JITTER_MAX_LEVEL = 8


def jitter_shift(trace, m, level):
    """Diagonal jitter of level l >= 0: 10^(l-10) tr(H)/|J|; level -1 is none."""
    return 0.0 if level < 0 else 10.0 ** (level - 10) * trace / m


def jittered_cholesky(H, level=-1):
    """Cholesky factor of H + jitter_shift(tr H, |J|, l) I for the first
    l = level, level + 1, ..., JITTER_MAX_LEVEL that factorises (level -1:
    H itself).  H is positive definite in exact arithmetic (lambda > 0,
    distinct basis points), but a computed H of a smooth kernel can lose that
    at rounding level.  Returns (L, l); raises NotPositiveDefinite when every
    level breaks down."""
    m = H.shape[0]
    tr = float(np.trace(H))
    for lv in range(level, JITTER_MAX_LEVEL + 1):
        try:
            return scipy.linalg.cholesky(H + jitter_shift(tr, m, lv) * np.eye(m), lower=True), lv
        except np.linalg.LinAlgError:
            continue
    raise NotPositiveDefinite(f"no jitter level up to {JITTER_MAX_LEVEL} factorises H")


def cholesky_solve(L, b):
    """(L L^T)^{-1} b by two triangular solves."""
    z = scipy.linalg.solve_triangular(L, b, lower=True)
    return scipy.linalg.solve_triangular(L.T, z, lower=False)


def newton_solve(H, r, level=-1):
    """beta_bar = (H + shift I)^{-1} r with the jitter of jittered_cholesky
    (shift 0 when H itself factorises).  Returns (beta_bar, l)."""
    if H.shape[0] == 0:
        return np.zeros(0), level
    L, lv = jittered_cholesky(H, level)
    return cholesky_solve(L, r), lv


# --------------------------------------------------------------------------
# Exact line search along d
# --------------------------------------------------------------------------
def _line_terms(beta, d, o, u, y, KJJ, lam):
    """phi'(t) = a0 + a1 t - sum_i v_i max(0, m_i - t v_i), with
    a0 = lambda d^T K_JJ beta, a1 = lambda d^T K_JJ d, m_i = 1 - y_i o_i,
    v_i = y_i u_i, u = K_nJ d."""
    a0 = lam * d @ (KJJ @ beta)
    a1 = lam * d @ (KJJ @ d)
    return a0, a1, 1.0 - y * o, y * u


def line_search_derivative(t, beta, d, o, u, y, KJJ, lam):
    a0, a1, m, v = _line_terms(beta, d, o, u, y, KJJ, lam)
    return a0 + a1 * t - np.sum(v * np.maximum(0.0, m - t * v))


def line_search(beta, d, o, u, y, KJJ, lam):
    """t* = argmin_{t >= 0} phi(t), phi(t) = f(beta + t d).

    phi' is piecewise linear and nondecreasing; its pieces change where a
    point crosses the margin, at t_i = m_i / v_i.  Walk the breakpoints in
    increasing order, keeping phi' = c0 + c1 t on the current piece, and
    return the root in the first piece where phi' reaches zero.  If
    |phi'(1)| <= 1e-12 |phi'(0)| the full step t = 1 is taken."""
    a0, a1, m, v = _line_terms(beta, d, o, u, y, KJJ, lam)

    def dphi(t):
        return a0 + a1 * t - np.sum(v * np.maximum(0.0, m - t * v))

    d0 = dphi(0.0)
    if d0 >= 0.0:
        return 0.0
    if abs(dphi(1.0)) <= 1e-12 * abs(d0):
        return 1.0
    # active just after t = 0
    act = (m > 0) | ((m == 0) & (v < 0))
    c0 = a0 - np.sum(v[act] * m[act])
    c1 = a1 + np.sum(v[act] ** 2)
    nz = v != 0
    bp = np.full(m.shape, np.inf)
    bp[nz] = m[nz] / v[nz]
    ev = np.nonzero(nz & (bp > 0))[0]
    ev = ev[np.argsort(bp[ev], kind="stable")]
    k = 0
    while k < len(ev):
        tb = bp[ev[k]]
        if c0 + c1 * tb >= 0.0:
            return -c0 / c1
        # every point with this breakpoint toggles here
        while k < len(ev) and bp[ev[k]] == tb:
            i = ev[k]
            if v[i] > 0:       # leaves the active set
                c0 += v[i] * m[i]
                c1 -= v[i] * v[i]
            else:              # enters the active set
                c0 -= v[i] * m[i]
                c1 += v[i] * v[i]
            k += 1
    if c1 <= 0.0:
        raise RuntimeError("line search: phi is unbounded below")
    return -c0 / c1


# --------------------------------------------------------------------------
# Basis-vector selection (Section 4, "Basis vector selection")
# --------------------------------------------------------------------------
def splitmix64(seed, counter):
    """Counter-based splitmix64: the finaliser applied to
    seed + (counter + 1) * 0x9E3779B97F4A7C15 (mod 2^64).  With seed 0 and
    counters 0, 1, 2 this is the published sequence of splitmix64 started
    from state 0."""
    z = (seed + (counter + 1) * SPLITMIX_GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def draw_candidates(n, J, kappa, seed, round_index):
    """kappa distinct indices from {0..n-1} minus J: the pool in increasing
    order, then a partial Fisher-Yates shuffle whose k-th swap partner is
    k + R mod (m - k), R = splitmix64(seed, round_index * 2^32 + k)."""
    pool = np.setdiff1d(np.arange(n, dtype=np.int64),
                        np.asarray(J, dtype=np.int64), assume_unique=False)
    m = len(pool)
    kk = min(kappa, m)
    for k in range(kk):
        r = splitmix64(seed, ((round_index & 0xFFFFFFFF) << 32) | k)
        j = k + int(r % (m - k))
        pool[k], pool[j] = pool[j], pool[k]
    return pool[:kk].copy()


def score_candidates(X, y, J, beta, o, cand, gamma, lam):
    """Delta_c = g_c^2 / (2 h_c) for each candidate c, where g_c and h_c are
    the first and second derivatives of f with respect to a new coefficient
    beta_c at beta_c = 0, on the current active set:
        g_c = lambda k(x_c, X_J) beta + sum_{i in S} (o_i - y_i) K_ic
        h_c = lambda k(x_c, x_c) + sum_{i in S} K_ic^2.
    Returns (Delta, g, h)."""
    X = np.asarray(X, dtype=np.float64)
    KnC = rbf_kernel(X, X[cand], gamma)
    S = active_set(y, o)
    res = np.where(S, o - y, 0.0)
    if len(J):
        KCJ = rbf_kernel(X[cand], X[np.asarray(J)], gamma)
        reg = KCJ @ beta
    else:
        reg = np.zeros(len(cand))
    Kcc = np.array([rbf_kernel(X[c:c + 1], X[c:c + 1], gamma)[0, 0] for c in cand])
    g = lam * reg + KnC.T @ res
    h = lam * Kcc + np.sum(KnC[S] ** 2, axis=0)
    return g * g / (2.0 * h), g, h


def score_candidates_exact(X, y, J, beta, o, cand, gamma, lam):
    """Exact one-dimensional variant of the selection score: f restricted to
    a new coefficient beta_c (every other coefficient fixed) is convex and
    piecewise quadratic in beta_c, and Delta_c is its exact decrease,
    f(beta) - min_t f(beta + t e_c).  The minimiser is found by the exact
    line search on the basis J + [c] along -sign(g_c) e_c (g_c the first
    derivative, as in score_candidates), which covers both signs of the new
    coefficient.  Returns (Delta, t) with t the signed minimiser."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    _, g, _ = score_candidates(X, y, J, beta, o, cand, gamma, lam)
    deltas, ts = [], []
    for k, c in enumerate(cand):
        Ja = [int(j) for j in J] + [int(c)]
        KnJa = rbf_kernel(X, X[Ja], gamma)
        KJJa = KnJa[Ja]
        ba = np.concatenate([np.asarray(beta, dtype=np.float64), [0.0]])
        if g[k] == 0.0:
            deltas.append(0.0)
            ts.append(0.0)
            continue
        sgn = -1.0 if g[k] > 0 else 1.0
        d = np.zeros(len(Ja))
        d[-1] = sgn
        t = line_search(ba, d, o, KnJa @ d, y, KJJa, lam)
        # f(beta + x e_c) - f(beta) written out from o (which carries any bias):
        # lambda x k_cJ beta + lambda/2 x^2 k_cc + 1/2 sum [xi(x)^2 - xi(0)^2]
        x = sgn * t
        kc = KnJa[:, -1]
        reg = lam * x * (KJJa[-1, :-1] @ np.asarray(beta, dtype=np.float64)) + 0.5 * lam * x * x * KJJa[-1, -1]
        loss = 0.5 * np.sum(np.maximum(0.0, 1.0 - y * (o + x * kc)) ** 2 - np.maximum(0.0, 1.0 - y * o) ** 2)
        deltas.append(-(reg + loss))
        ts.append(x)
    return np.asarray(deltas), np.asarray(ts)


def select_top(delta, cand, q):
    """The q candidates with the largest Delta, in decreasing Delta; equal
    scores go to the smaller point index first."""
    order = sorted(range(len(cand)), key=lambda k: (-delta[k], int(cand[k])))
    return np.asarray([cand[k] for k in order[:q]], dtype=np.int64)


# --------------------------------------------------------------------------
# Reoptimisation of Eq. 4 on a fixed basis
# --------------------------------------------------------------------------
def newton(KnJ, KJJ, y, lam, beta, tol, max_newton, history=None, jitter=None):
    """Newton iterations with exact line search on a fixed J.

    Stops when ||grad f|| <= tol, when the active set repeats after a full
    unjittered step (t = 1; the quadratic piece's minimiser is then
    stationary), when no jitter level gives descent, or after max_newton
    steps.  Returns (beta, o, status) with status one of 'tol', 'repeat',
    'stall', 'max'.  jitter: a one-element list holding the jitter level that
    factorised the previous Newton matrix of this fit (-1 at the start); each
    factorisation starts from that level and stores its own."""
    if jitter is None:
        jitter = [-1]
    o = KnJ @ beta
    status = "max"
    for _ in range(max_newton):
        S = active_set(y, o)
        g = lam * (KJJ @ beta) + KnJ[S].T @ (o[S] - y[S])
        gn = float(np.linalg.norm(g))
        if gn <= tol:
            status = "tol"
            if history is not None:
                history.append(dict(objective=objective(beta, KnJ, KJJ, y, lam),
                                    gnorm=gn, active=int(S.sum()), t=0.0,
                                    basis=len(beta), step=False, jitter=jitter[0]))
            break
        KS = KnJ[S]
        H = lam * KJJ + KS.T @ KS
        r = KS.T @ y[S]
        # Section 4's step d = beta_bar - beta, beta_bar = H^{-1} K_SJ^T y_S.
        # With a jitter the step is the regularised Newton step
        # d = -(H + shift I)^{-1} grad f (the same at shift 0); when the line
        # search finds no descent along d the jitter goes up one level.
        Lc, lv = jittered_cholesky(H, jitter[0])
        d = cholesky_solve(Lc, r) - beta if lv < 0 else -cholesky_solve(Lc, g)
        u = KnJ @ d
        t = line_search(beta, d, o, u, y, KJJ, lam)
        while t == 0.0 and lv < JITTER_MAX_LEVEL:
            Lc, lv = jittered_cholesky(H, lv + 1)
            d = -cholesky_solve(Lc, g)
            u = KnJ @ d
            t = line_search(beta, d, o, u, y, KJJ, lam)
        jitter[0] = lv
        if t == 0.0:
            status = "stall"
            if history is not None:
                history.append(dict(objective=objective(beta, KnJ, KJJ, y, lam),
                                    gnorm=gn, active=int(S.sum()), t=0.0,
                                    basis=len(beta), step=False, jitter=lv))
            break
        beta = beta + t * d
        o = KnJ @ beta
        S_new = active_set(y, o)
        if history is not None:
            history.append(dict(objective=objective(beta, KnJ, KJJ, y, lam),
                                gnorm=gn, active=int(S.sum()), t=float(t),
                                basis=len(beta), step=True, jitter=jitter[0]))
        if t == 1.0 and np.array_equal(S_new, S) and lv < 0:
            status = "repeat"
            break
    return beta, o, status


@dataclass
class FitResult:
    J: np.ndarray
    beta: np.ndarray
    o: np.ndarray
    history: list = field(default_factory=list)
    rounds: list = field(default_factory=list)
    status: str = ""
    bias: float = 0.0

    def decision(self, X, Xq, gamma):
        return predict(Xq, np.asarray(X)[self.J], self.beta, gamma, self.bias)


def fit(X, y, gamma, lam, budget, tol=1e-8, kappa=256, q=64, max_newton=50,
        initial_basis=None, grow=True, seed=0, growth_tol=0.0, replay=None,
        replay_rtol=1e-6, score="heuristic", bias=False):
    """SP-SVM (Section 4): alternate basis-vector selection and
    reoptimisation until |J| = budget or the growth stop fires.

    `replay`, if given, is a list with one dict per growth round holding the
    other implementation's 'candidates' and 'chosen'.  The oracle then checks
    that its own draw gives the same candidates and that every chosen point
    scores at least (q-th best oracle score) * (1 - replay_rtol), and adopts
    the chosen list, so that near-ties cannot make the two runs diverge.

    bias=True adds Eq. 4's bias b as an unregularised coordinate: the Newton
    iteration runs on the basis extended by a column of ones whose row and
    column of the regulariser are zero, and the model is f(x) = k(x, X_J)
    beta + b.  The scores see b through o alone."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = X.shape[0]
    J = [] if initial_basis is None else [int(j) for j in initial_basis]
    KnJ = rbf_kernel(X, X[J], gamma) if J else np.zeros((n, 0))
    beta = np.zeros(len(J))
    b = 0.0
    res = FitResult(J=np.asarray(J, dtype=np.int64), beta=beta, o=np.zeros(n))
    status = ""
    jitter = [-1]

    def reoptimise(beta, b):
        if not bias:
            beta, o, st = newton(KnJ, KnJ[J], y, lam, beta, tol, max_newton, res.history, jitter)
            return beta, 0.0, o, st
        m = KnJ.shape[1]
        KJJa = np.zeros((m + 1, m + 1))
        KJJa[1:, 1:] = KnJ[J]
        ba, o, st = newton(np.hstack([np.ones((n, 1)), KnJ]), KJJa, y, lam,
                           np.concatenate([[b], beta]), tol, max_newton, res.history, jitter)
        return ba[1:], ba[0], o, st

    if J or bias:
        beta, b, o, status = reoptimise(beta, b)
    else:
        o = np.zeros(n)
    E_prev = float(np.mean(y * o <= 0))
    rnd = 0
    while grow and len(J) < budget:
        cand = draw_candidates(n, J, kappa, seed, rnd)
        if len(cand) == 0:
            break
        if score == "exact":
            delta, _ = score_candidates_exact(X, y, J, beta, o, cand, gamma, lam)
        else:
            delta, _, _ = score_candidates(X, y, J, beta, o, cand, gamma, lam)
        qq = min(q, budget - len(J), len(cand))
        chosen = select_top(delta, cand, qq)
        info = dict(candidates=cand, delta=delta, chosen=chosen)
        if replay is not None:
            other = replay[rnd]
            oc = np.asarray(other["candidates"], dtype=np.int64)
            if not np.array_equal(oc, cand):
                raise AssertionError(f"round {rnd}: candidate draws differ")
            ochosen = np.asarray(other["chosen"], dtype=np.int64)
            pos = {int(c): k for k, c in enumerate(cand)}
            qth = np.sort(delta)[::-1][qq - 1]
            for c in ochosen:
                if delta[pos[int(c)]] < qth * (1.0 - replay_rtol):
                    raise AssertionError(
                        f"round {rnd}: chosen point {int(c)} scores "
                        f"{delta[pos[int(c)]]:.17g} < q-th best {qth:.17g}")
            info["oracle_chosen"] = chosen
            chosen = ochosen
        res.rounds.append(info)
        J = J + [int(c) for c in chosen]
        KnJ = np.hstack([KnJ, rbf_kernel(X, X[chosen], gamma)])
        beta = np.concatenate([beta, np.zeros(len(chosen))])
        beta, b, o, status = reoptimise(beta, b)
        rnd += 1
        E = float(np.mean(y * o <= 0))
        res.rounds[-1]["error_rate"] = E
        if growth_tol > 0 and (E_prev - E) / len(chosen) < growth_tol:
            break
        E_prev = E
    res.J = np.asarray(J, dtype=np.int64)
    res.beta = beta
    res.bias = float(b)
    res.o = o
    res.status = status
    return res


def predict(Xq, XJ, beta, gamma, bias=0.0):
    """Decision values f(x) = sum_{j in J} beta_j k(x, x_j) + b (Section 4,
    h(x) = w^T phi(x) with w restricted to the basis; b = 0 unless fitted)."""
    return rbf_kernel(Xq, XJ, gamma) @ beta + bias


def ovo_pairs(classes):
    """The one-vs-one binary problems (a, b), a < b, in the order (0, 1),
    (0, 2), ..., (0, C-1), (1, 2), ... (Section 5 trains its multiclass
    sets one-vs-one)."""
    return [(a, b) for a in range(classes) for b in range(a + 1, classes)]


def ovo_vote(decisions, classes):
    """Labels from one-vs-one decision values: decisions[p][i], the value of
    pair p = (a, b) of ovo_pairs(classes) at query i, is a vote for a when
    it is >= 0 and for b otherwise; the class with the most votes wins, a
    tie going to the smaller class (a reading: the paper names no rule).
    Returns (labels, votes)."""
    decisions = np.asarray(decisions)
    nq = decisions.shape[1]
    votes = np.zeros((nq, classes), dtype=np.int64)
    for p, (a, b) in enumerate(ovo_pairs(classes)):
        for i in range(nq):
            if decisions[p, i] >= 0:
                votes[i, a] += 1
            else:
                votes[i, b] += 1
    out = np.zeros(nq, dtype=np.int64)
    for i in range(nq):
        best = 0
        for c in range(1, classes):
            if votes[i, c] > votes[i, best]:
                best = c
        out[i] = best
    return out, votes


def fit_ovo(X, class_labels, classes, gamma, lam, budget, replay=None, **kw):
    """One binary SP-SVM per pair (a, b) on the points of class a (y = +1)
    and class b (y = -1), the budget capped at the pair's point count.
    Returns [(rows, FitResult)] in ovo_pairs order; replay, if given, holds
    one replay list per pair."""
    X = np.asarray(X, dtype=np.float64)
    class_labels = np.asarray(class_labels)
    out = []
    for p, (a, b) in enumerate(ovo_pairs(classes)):
        rows = np.flatnonzero((class_labels == a) | (class_labels == b))
        y = np.where(class_labels[rows] == a, 1.0, -1.0)
        r = fit(X[rows], y, gamma, lam, min(budget, len(rows)),
                replay=None if replay is None else replay[p], **kw)
        out.append((rows, r))
    return out


def predict_ovo(X, fitted, classes, Xq, gamma):
    """Labels (and votes) of the queries Xq by one-vs-one voting over the
    pair models of fit_ovo (basis rows taken from X through each pair's
    rows)."""
    X = np.asarray(X, dtype=np.float64)
    dec = np.stack([predict(Xq, X[rows][r.J], r.beta, gamma) for rows, r in fitted])
    return ovo_vote(dec, classes)


def labels(decision):
    """sign with sign(0) = +1."""
    return np.where(np.asarray(decision) >= 0, 1.0, -1.0)
