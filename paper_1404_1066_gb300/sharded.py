"""Row-sharded form of one SP-SVM fit (Section 4, Eq. 4) over W processes.

Every sum over points in the method splits by rows.  Rank r holds a
contiguous range of the n points: its rows of X, y, K_nJ, o = K_nJ beta and
u = K_nJ d.  The basis rows X_J, beta, K_JJ and the |J| x |J| Newton system
are replicated: every rank solves the same system with the same
deterministic arithmetic, so the ranks stay identical without a broadcast.
Per Newton step the ranks exchange, by all-reduce (sum, FP64):

  * the data parts of the Newton system, of the gradient and of the
    right-hand side, packed into one reduce: K_{S_r J}^T K_{S_r J},
    K_{S_r J}^T (o - y)_{S_r}, K_{S_r J}^T y_{S_r} and |S_r|;
  * for the exact line search, phi'(t) on a 33-point grid together with the
    number of breakpoints in each grid cell (one reduce per bracketing pass,
    usually one or two), then the two coefficients of the linear piece that
    holds the root;
  * the number of points whose active flag changed (the stopping rule);

and per growth round:

  * the rows of the candidates and of the chosen points (each rank fills the
    rows it owns, zeros elsewhere, so the sum is the gather);
  * the data parts of the selection score, sum_{S_r} (o_i - y_i) K_ic and
    sum_{S_r} K_ic^2.

The per-rank arithmetic comes from a provider object (the `Shard` protocol
below) that computes sums over its own rows only.  This module holds the
partition, the collective schedule and the assembly of the reduced parts.
It is exercised with two gloo ranks on the CPU; one fit spread over several
GPUs has not been measured.
"""
from __future__ import annotations

from typing import Callable, Protocol, Sequence, Tuple

import numpy as np
import torch
import torch.distributed as dist


def row_range(n: int, world: int, rank: int) -> Tuple[int, int]:
    """Rows [lo, hi) of rank `rank`: n split into `world` contiguous ranges
    whose sizes differ by at most one (the first n mod world ranks hold one
    more)."""
    base, extra = divmod(int(n), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


class Comm:
    """Reductions over the default process group in FP64 (a process without
    a group is a world of one and reduces nothing).  `device` is where the
    packed buffer lives for the collective: "cpu" for gloo, a CUDA device
    for NCCL."""

    def __init__(self, device="cpu", group=None):
        self.group = group
        self.device = device
        on = dist.is_available() and dist.is_initialized()
        self.world = dist.get_world_size(group) if on else 1
        self.rank = dist.get_rank(group) if on else 0

    def _reduce(self, arrays, op):
        flat = [np.asarray(a, dtype=np.float64) for a in arrays]
        if self.world == 1:
            return [f.copy() for f in flat]
        buf = torch.from_numpy(np.concatenate([f.ravel() for f in flat])).to(self.device)
        dist.all_reduce(buf, op=op, group=self.group)
        buf = buf.cpu().numpy()
        out, k = [], 0
        for f in flat:
            out.append(buf[k:k + f.size].reshape(f.shape))
            k += f.size
        return out

    def sum(self, *arrays):
        """Element-wise sums over the ranks, one collective for all arrays."""
        return self._reduce(arrays, dist.ReduceOp.SUM if self.world > 1 else None)

    def min(self, *arrays):
        return self._reduce(arrays, dist.ReduceOp.MIN if self.world > 1 else None)


class Shard(Protocol):
    """Per-rank arithmetic over rows [lo, hi) of the points.

    lo, hi: the row range; y: its labels (FP64).
    rows(idx): the rows of X at global indices idx, all in [lo, hi).
    kernel(A, B): k(a, b) for rows A, B (replicated small blocks).
    extend(XJ_new): append the columns k(x_i, z) for the new basis rows z.
    outputs(beta): K_{rJ} beta over the rank's rows.
    image(d): K_{rJ} d.
    newton_parts(o): (K_{S_r J}^T K_{S_r J}, K_{S_r J}^T (o - y)_{S_r},
        K_{S_r J}^T y_{S_r}) with S_r = {i in [lo, hi) : y_i o_i < 1}.
    score_parts(Xc, o): (sum_{S_r} (o_i - y_i) k(x_i, x_c), sum_{S_r} k(x_i, x_c)^2).
    factor(H, level): (solve, level used) of the first jitter level from
        `level` whose factor of H + shift I exists; solve(b) applies its inverse.
    draw(n, J, kappa, seed, round_index): the round's candidates (the same
        on every rank: a counter-based generator).
    """

    lo: int
    hi: int
    y: np.ndarray

    def rows(self, idx: np.ndarray) -> np.ndarray: ...
    def kernel(self, A: np.ndarray, B: np.ndarray) -> np.ndarray: ...
    def extend(self, XJ_new: np.ndarray) -> None: ...
    def outputs(self, beta: np.ndarray) -> np.ndarray: ...
    def image(self, d: np.ndarray) -> np.ndarray: ...
    def newton_parts(self, o: np.ndarray) -> Tuple[np.ndarray, np.ndarray, np.ndarray]: ...
    def score_parts(self, Xc: np.ndarray, o: np.ndarray) -> Tuple[np.ndarray, np.ndarray]: ...
    def factor(self, H: np.ndarray, level: int) -> Tuple[Callable, int]: ...
    def draw(self, n: int, J: Sequence[int], kappa: int, seed: int, round_index: int) -> np.ndarray: ...


def gather_rows(comm: Comm, shard: Shard, idx, d: int) -> np.ndarray:
    """Rows idx of X on every rank: the owner of each row contributes it,
    the others zeros, and the sum is exact."""
    idx = np.asarray(idx, dtype=np.int64)
    out = np.zeros((len(idx), d))
    mine = (idx >= shard.lo) & (idx < shard.hi)
    if mine.any():
        out[mine] = shard.rows(idx[mine])
    return comm.sum(out)[0]


def newton_system(comm: Comm, shard: Shard, o, beta, KJJ, lam):
    """The Newton system of Eq. 4 on the active set from one reduce:
    H = lambda K_JJ + K_SJ^T K_SJ, g = lambda K_JJ beta + K_SJ^T (o - y)_S,
    r = K_SJ^T y_S, |S|."""
    HS, gS, rS = shard.newton_parts(o)
    nS = np.array([np.count_nonzero(shard.y * o < 1.0)], dtype=np.float64)
    HS, gS, rS, nS = comm.sum(HS, gS, rS, nS)
    H = lam * KJJ + HS
    g = lam * (KJJ @ beta) + gS
    return H, g, rS, int(nS[0])


def line_search(comm: Comm, a0: float, a1: float, m: np.ndarray, v: np.ndarray,
                grid: int = 33, max_pass: int = 80) -> float:
    """Exact minimiser t >= 0 of phi(t) = f(beta + t d) from the ranks' terms.

    phi'(t) = a0 + a1 t - sum_i v_i max(0, m_i - t v_i) is piecewise linear
    and nondecreasing, with breakpoints t_i = m_i / v_i (m_i = 1 - y_i o_i,
    v_i = y_i u_i; a0 = lambda d^T K_JJ beta and a1 = lambda d^T K_JJ d are
    replicated).  The root is bracketed on a grid of `grid` points, one
    reduce per pass (phi' at the grid points and the count of breakpoints
    strictly inside each cell), until the cell holding the root holds no
    breakpoint; there phi' = c0 + c1 t exactly, with c0, c1 reduced over the
    points active inside the cell, and t = -c0 / c1.  t = 1 when
    |phi'(1)| <= 1e-12 |phi'(0)|; t = 0 when phi'(0) >= 0."""
    m = np.asarray(m, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)

    def sums(ts):
        ts = np.asarray(ts, dtype=np.float64)
        return np.array([np.sum(v * np.maximum(0.0, m - t * v)) for t in ts])

    s0, s1 = comm.sum(sums([0.0, 1.0]))[0]
    d0, d1 = a0 - s0, a0 + a1 - s1
    if d0 >= 0.0:
        return 0.0
    if abs(d1) <= 1e-12 * abs(d0):
        return 1.0
    nz = v != 0.0
    bp = np.full(m.shape, np.inf)
    bp[nz] = m[nz] / v[nz]
    tl, th = 0.0, 1.0
    dh = d1
    for _ in range(1100):   # phi' grows without bound unless c1 <= 0 at large t
        if dh >= 0.0:
            break
        tl, th = th, 2.0 * th
        dh = a0 + a1 * th - comm.sum(sums([th]))[0][0]
    else:
        raise RuntimeError("line search: phi is unbounded below")

    def piece(a, b):
        tm = 0.5 * (a + b)
        act = m - tm * v > 0.0
        C0, C1 = comm.sum(np.array([np.sum(v[act] * m[act]), np.sum(v[act] ** 2)]))[0]
        c0, c1 = a0 - C0, a1 + C1
        if c1 <= 0.0:
            raise RuntimeError("line search: phi is unbounded below")
        return -c0 / c1

    for _ in range(max_pass):
        ts = tl + (th - tl) * np.arange(grid) / (grid - 1)
        ts[-1] = th
        inside = np.array([np.count_nonzero((bp > ts[k]) & (bp < ts[k + 1]))
                           for k in range(grid - 1)], dtype=np.float64)
        S, cnt = comm.sum(sums(ts), inside)
        dp = a0 + a1 * ts - S
        k = int(np.argmax(dp >= 0.0)) if np.any(dp >= 0.0) else grid - 1
        k = max(k, 1)
        a, b = ts[k - 1], ts[k]
        if cnt[k - 1] == 0:
            return piece(a, b)
        # the breakpoints inside: when they are all one value tb, phi' is
        # linear on either side of it
        sel = (bp > a) & (bp < b)
        lo_hi = np.array([bp[sel].min() if sel.any() else np.inf,
                          -bp[sel].max() if sel.any() else np.inf])
        bmin, nbmax = comm.min(lo_hi)[0]
        if bmin == -nbmax:
            tb = bmin
            dtb = a0 + a1 * tb - comm.sum(sums([tb]))[0][0]
            return piece(a, tb) if dtb >= 0.0 else piece(tb, b)
        tl, th = a, b
    return piece(tl, th)


def score(comm: Comm, shard: Shard, Xc, o, reg, Kcc, lam):
    """Selection score of Section 4 for candidates with rows Xc:
    g_c = lambda k_cJ beta + sum_S (o_i - y_i) K_ic, h_c = lambda K_cc +
    sum_S K_ic^2, Delta_c = g_c^2 / (2 h_c); reg = k_cJ beta and Kcc are
    replicated, the sums are one reduce."""
    G, Hc = shard.score_parts(Xc, o)
    G, Hc = comm.sum(G, Hc)
    g = lam * np.asarray(reg) + G
    h = lam * np.asarray(Kcc) + Hc
    return g * g / (2.0 * h), g, h


def select_top(delta, cand, q):
    """The q candidates with the largest Delta, in decreasing Delta; equal
    scores go to the smaller point index first."""
    order = sorted(range(len(cand)), key=lambda k: (-float(delta[k]), int(cand[k])))
    return np.asarray([cand[k] for k in order[:q]], dtype=np.int64)


JITTER_MAX_LEVEL = 8


def newton(comm: Comm, shard: Shard, KJJ, lam, beta, tol, max_newton, jitter=None):
    """Newton iterations of Eq. 4 with the exact line search on a fixed basis,
    row-sharded.  Same rules as the single-process fit: stop when
    ||grad f|| <= tol, when a full unjittered step leaves the active set
    unchanged, when no jitter level gives descent, or after max_newton
    steps.  Returns (beta, o over the rank's rows, status)."""
    if jitter is None:
        jitter = [-1]
    beta = np.asarray(beta, dtype=np.float64)
    o = shard.outputs(beta)
    status = "max"
    for _ in range(max_newton):
        S = shard.y * o < 1.0
        H, g, r, _ = newton_system(comm, shard, o, beta, KJJ, lam)
        if float(np.linalg.norm(g)) <= tol:
            status = "tol"
            break
        solve, lv = shard.factor(H, jitter[0])
        d = solve(r) - beta if lv < 0 else -solve(g)

        def search(d):
            u = shard.image(d)
            return line_search(comm, lam * d @ (KJJ @ beta), lam * d @ (KJJ @ d),
                               1.0 - shard.y * o, shard.y * u)

        t = search(d)
        while t == 0.0 and lv < JITTER_MAX_LEVEL:
            solve, lv = shard.factor(H, lv + 1)
            d = -solve(g)
            t = search(d)
        jitter[0] = lv
        if t == 0.0:
            status = "stall"
            break
        beta = beta + t * d
        o = shard.outputs(beta)
        changed = comm.sum(np.array([np.count_nonzero((shard.y * o < 1.0) != S)], dtype=np.float64))[0][0]
        if t == 1.0 and changed == 0 and lv < 0:
            status = "repeat"
            break
    return beta, o, status


def fit(comm: Comm, shard: Shard, n: int, d: int, lam: float, budget: int, tol: float = 1e-8,
        kappa: int = 256, q: int = 64, max_newton: int = 50, seed: int = 0):
    """Row-sharded SP-SVM fit (Section 4): rounds of candidate draw, score,
    top-q selection and reoptimisation until |J| = budget.  Returns
    (J, beta, o over the rank's rows, status); J and beta are the same on
    every rank."""
    J: list = []
    XJ = np.zeros((0, d))
    beta = np.zeros(0)
    o = np.zeros(shard.hi - shard.lo)
    status = ""
    jitter = [-1]
    rnd = 0
    while len(J) < budget:
        cand = np.asarray(shard.draw(n, J, kappa, seed, rnd), dtype=np.int64)
        if len(cand) == 0:
            break
        Xc = gather_rows(comm, shard, cand, d)
        reg = shard.kernel(Xc, XJ) @ beta if len(J) else np.zeros(len(cand))
        Kcc = np.array([shard.kernel(Xc[k:k + 1], Xc[k:k + 1])[0, 0] for k in range(len(cand))])
        delta, _, _ = score(comm, shard, Xc, o, reg, Kcc, lam)
        qq = min(q, budget - len(J), len(cand))
        chosen = select_top(delta, cand, qq)
        Xn = gather_rows(comm, shard, chosen, d)
        J += [int(c) for c in chosen]
        XJ = np.vstack([XJ, Xn])
        shard.extend(Xn)
        KJJ = shard.kernel(XJ, XJ)
        beta = np.concatenate([beta, np.zeros(len(chosen))])
        beta, o, status = newton(comm, shard, KJJ, lam, beta, tol, max_newton, jitter)
        rnd += 1
    return np.asarray(J, dtype=np.int64), beta, o, status
