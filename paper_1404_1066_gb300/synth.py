"""Seeded synthetic inputs for the SP-SVM workloads.

This module only draws data: feature matrices, labels, fixed random bases,
subsample index lists and arrival streams.  It holds none of the SP-SVM
arithmetic (no kernel block, objective, Newton step or basis score), so the
oracle and the CUDA path can both be fed from it without sharing method code.

The paper's datasets (Adult, Covertype, KDDCup99, MITFaces, Epsilon, FD,
MNIST8M; Section 5) are not available, so these generators stand in for them
with the same shapes and value ranges: features scaled to [0, 1] with many
zeros for the MNIST-like case (Section 5, "Datasets"), dense Gaussian
mixtures for the Covertype / KDDCup-scale cases.

Every generator returns float32 features (the storage precision of X) and
float32 labels in {-1, +1}.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Problem:
    """One binary SP-SVM training problem (Eq. 4 with lambda = 1/C)."""
    X: np.ndarray            # n x d float32, row-major
    y: np.ndarray            # n float32 in {-1, +1}
    gamma: float             # RBF width, k(x,z) = exp(-gamma ||x-z||^2)
    lam: float               # lambda = 1/C
    budget: int              # final |J|
    initial_basis: np.ndarray | None = None   # int64 indices (fixed basis)
    grow: bool = True
    candidates: int = 256    # kappa, candidates drawn per growth round
    add_per_round: int = 64  # q, basis vectors added per round
    tol: float = 1e-8
    seed: int = 0
    name: str = ""
    meta: dict = field(default_factory=dict)


def two_gaussians(n=2000, d=20, flip=0.05, seed=1001, basis=100, lam=1e-3):
    """Binary workload: two Gaussian components with means +-0.5*1 and unit
    covariance; labels by component with a fraction `flip` flipped; gamma =
    1/d; a fixed random basis of `basis` points (drawn here, as an input)."""
    g = _rng(seed)
    comp = g.integers(0, 2, size=n)
    mean = np.where(comp[:, None] == 1, 0.5, -0.5)
    X = (mean + g.standard_normal((n, d))).astype(np.float32)
    y = np.where(comp == 1, 1.0, -1.0)
    flips = g.random(n) < flip
    y[flips] = -y[flips]
    J0 = np.sort(g.choice(n, size=min(basis, n), replace=False)).astype(np.int64)
    return Problem(X=X, y=y.astype(np.float32), gamma=1.0 / d, lam=lam,
                   budget=len(J0), initial_basis=J0, grow=False, tol=1e-8,
                   seed=seed, name=f"two_gaussians_n{n}_d{d}")


def _sparse_unit(g, n, d, p_zero):
    v = g.random((n, d))
    keep = g.random((n, d)) >= p_zero
    # Uniform(0,1]: 1 - U[0,1) lies in (0,1].
    return np.where(keep, 1.0 - v, 0.0)


def sparse_teacher(n=100_000, d=784, p_zero=0.8, centers=50, seed=1002,
                   budget=1024, lam=1e-4, kappa=256, q=64):
    """MNIST-like workload: each feature is 0 with probability p_zero, else
    Uniform(0,1]; labels are the sign of a random RBF expansion over
    `centers` teacher centres drawn from the same distribution with N(0,1)
    weights; gamma = 1/(d * var) with var the population variance of all
    entries of X.  The teacher is part of the data recipe, evaluated here in
    float64 from direct differences."""
    g = _rng(seed)
    X64 = _sparse_unit(g, n, d, p_zero)
    X = X64.astype(np.float32)
    var = float(np.var(X.astype(np.float64)))
    gamma = 1.0 / (d * var)
    T = _sparse_unit(g, centers, d, p_zero).astype(np.float32).astype(np.float64)
    a = g.standard_normal(centers)
    Xd = X.astype(np.float64)
    score = np.zeros(n)
    for c0 in range(0, n, 8192):
        blk = Xd[c0:c0 + 8192]
        d2 = ((blk[:, None, :] - T[None, :, :]) ** 2).sum(-1)
        score[c0:c0 + 8192] = np.exp(-gamma * d2) @ a
    y = np.where(score >= 0, 1.0, -1.0).astype(np.float32)
    return Problem(X=X, y=y, gamma=gamma, lam=lam, budget=budget,
                   candidates=kappa, add_per_round=q, tol=1e-6, seed=seed,
                   name=f"sparse_teacher_n{n}_d{d}",
                   meta={"var": var})


def gaussian_mixture(n=500_000, d=128, components=10, sigma_m=1.0,
                     seed=1003, budget=4096, lam=1e-4, gamma=None,
                     kappa=256, q=64, label_class=None):
    """Dense mixture workload: `components` Gaussian components with means
    drawn from N(0, sigma_m^2 I) and isotropic scales s_c ~ U[0.5, 2];
    x = mu_c + s_c * N(0, I).  Binary labels by component parity (+1 for an
    even component), or one-vs-rest against `label_class` when given.
    gamma defaults to 1/d."""
    g = _rng(seed)
    mu = g.standard_normal((components, d)) * sigma_m
    s = g.uniform(0.5, 2.0, size=components)
    comp = g.integers(0, components, size=n)
    X = np.empty((n, d), dtype=np.float32)
    for c0 in range(0, n, 65536):
        c1 = min(n, c0 + 65536)
        cc = comp[c0:c1]
        X[c0:c1] = (mu[cc] + s[cc, None] * g.standard_normal((c1 - c0, d))).astype(np.float32)
    if label_class is None:
        y = np.where(comp % 2 == 0, 1.0, -1.0)
    else:
        y = np.where(comp == label_class, 1.0, -1.0)
    return Problem(X=X, y=y.astype(np.float32),
                   gamma=(1.0 / d) if gamma is None else gamma, lam=lam,
                   budget=budget, candidates=kappa, add_per_round=q, tol=1e-6,
                   seed=seed, name=f"gaussian_mixture_n{n}_d{d}",
                   meta={"components": comp.astype(np.int32), "means": mu, "scales": s,
                         "label_class": label_class})


def mixture_holdout(problem: Problem, m: int, seed: int, components=False):
    """Labelled held-out points (float32 X, +-1 y) drawn afresh from the
    same mixture as a gaussian_mixture problem (its component means and
    scales), labelled the same way; with components=True the component
    index (the multiclass label) instead of y."""
    mu, s = problem.meta["means"], problem.meta["scales"]
    g = _rng(seed)
    comp = g.integers(0, mu.shape[0], size=m)
    X = (mu[comp] + s[comp, None] * g.standard_normal((m, mu.shape[1]))).astype(np.float32)
    if components:
        return X, comp.astype(np.int64)
    lc = problem.meta["label_class"]
    y = np.where(comp % 2 == 0, 1.0, -1.0) if lc is None else np.where(comp == lc, 1.0, -1.0)
    return X, y.astype(np.float32)


@dataclass
class GridSolve:
    """One solve of the one-vs-rest x (gamma, lambda) grid on a shared X."""
    solve_id: int
    label_class: int
    gamma: float
    lam: float
    rows: np.ndarray          # int64 indices into the shared X (sorted)
    budget: int


def ovr_grid(n=60_000, d=256, classes=10, seed=1004, n_min=5_000,
             n_max=60_000, j_min=256, j_max=2048, gammas=(0.25, 0.5, 1.0, 2.0),
             lams=(1e-3, 1e-4, 1e-5)):
    """Batched workload: a shared 10-class mixture X (as gaussian_mixture),
    one-vs-rest classes x gamma in {0.25,0.5,1,2}/d x lambda in
    {1e-3,1e-4,1e-5}; each solve on a seeded subsample with n_s ~ U[n_min,
    n_max] and |J|_s ~ U[j_min, j_max] rounded to a multiple of 64."""
    base = gaussian_mixture(n=n, d=d, components=classes, seed=seed)
    comp = base.meta["components"]
    solves = []
    sid = 0
    for c in range(classes):
        for gm in gammas:
            for lm in lams:
                g = _rng(seed * 1_000_003 + sid)
                ns = int(g.integers(n_min, n_max + 1))
                rows = np.sort(g.choice(n, size=ns, replace=False)).astype(np.int64)
                jb = int(g.integers(j_min, j_max + 1))
                jb = max(64, min(j_max, 64 * int(round(jb / 64))))
                jb = min(jb, ns)
                solves.append(GridSolve(sid, c, gm / d, lm, rows, jb))
                sid += 1
    return base.X, comp, solves


def ovr_labels(comp: np.ndarray, label_class: int) -> np.ndarray:
    return np.where(comp == label_class, 1.0, -1.0).astype(np.float32)


@dataclass
class Request:
    t_arrival: float
    kind: str                 # "fit" or "predict"
    n: int
    d: int
    budget: int
    seed: int
    target: int = -1          # for predict: index of the fit request it uses


def arrival_stream(count=2000, rate=20.0, seed=1005, n_lo=1_000, n_hi=200_000,
                   dims=(32, 128, 784), budgets=tuple(128 * k for k in range(1, 17)),
                   predict_frac=0.5, m_lo=1_000, m_hi=100_000):
    """Serving workload: Poisson arrivals (exponential gaps, mean rate `rate`
    per second) of fit requests with n log-uniform in [n_lo, n_hi], d from
    `dims` and |J| from `budgets`, interleaved with predict requests of
    m_lo..m_hi points against an earlier fit."""
    g = _rng(seed)
    t = 0.0
    out = []
    fits = []
    for k in range(count):
        t += float(g.exponential(1.0 / rate))
        if fits and g.random() < predict_frac:
            m = int(math.exp(g.uniform(math.log(m_lo), math.log(m_hi))))
            tgt = int(fits[int(g.integers(0, len(fits)))])
            out.append(Request(t, "predict", m, out[tgt].d, 0, seed * 7919 + k, tgt))
        else:
            n = int(math.exp(g.uniform(math.log(n_lo), math.log(n_hi))))
            dd = int(dims[int(g.integers(0, len(dims)))])
            jb = int(budgets[int(g.integers(0, len(budgets)))])
            jb = min(jb, n)
            fits.append(k)
            out.append(Request(t, "fit", n, dd, jb, seed * 7919 + k))
    return out


def queries_like(problem: Problem, m: int, seed: int) -> np.ndarray:
    """Held-out query points from the same distribution family (resampled
    rows with small jitter), float32."""
    g = _rng(seed)
    idx = g.integers(0, problem.X.shape[0], size=m)
    Xq = problem.X[idx].astype(np.float64) + 0.05 * g.standard_normal((m, problem.X.shape[1]))
    return Xq.astype(np.float32)
