"""Brute-force dual of the squared-hinge kernel SVM, for tiny problems.

TEST INFRASTRUCTURE ONLY (see the package header).

With J = all points, Eq. 4 is Chapelle's primal (Section 4, Eq. 3, bias
dropped).  Multiplying f by C = 1/lambda gives 1/2 ||w||^2 + C/2 sum xi_i^2,
whose Lagrange dual is the squared-hinge form of Eq. 2 (Section 2):

    max_{alpha >= 0}  sum_i alpha_i - 1/2 alpha^T (Q + lambda I) alpha,
    Q_ij = y_i y_j k(x_i, x_j),

with w = sum_i alpha_i y_i phi(x_i), i.e. beta = alpha * y.  The dual is a
strictly concave QP, so its optimum is the unique point satisfying the KKT
conditions; for n <= ~14 it is found by enumerating every support pattern A,
solving (Q_AA + lambda I) alpha_A = 1 and keeping the pattern whose alpha
is nonnegative and whose dual gradient is nonpositive off A.
"""
from __future__ import annotations

import itertools

import numpy as np


def squared_hinge_dual_bruteforce(K, y, lam, feas_tol=1e-12):
    """Returns (alpha, beta) for the squared-hinge dual with Gram matrix K."""
    K = np.asarray(K, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    if n > 16:
        raise ValueError("brute force is for tiny problems only")
    M = (y[:, None] * y[None, :]) * K + lam * np.eye(n)
    best = None
    for size in range(n + 1):
        for A in itertools.combinations(range(n), size):
            A = list(A)
            alpha = np.zeros(n)
            if A:
                alpha[A] = np.linalg.solve(M[np.ix_(A, A)], np.ones(len(A)))
            if np.any(alpha[A] < -feas_tol):
                continue
            grad = 1.0 - M @ alpha
            off = [i for i in range(n) if i not in A]
            if off and np.any(grad[off] > feas_tol):
                continue
            val = alpha.sum() - 0.5 * alpha @ M @ alpha
            if best is None or val > best[0]:
                best = (val, alpha)
    if best is None:
        raise RuntimeError("no KKT point found")
    alpha = best[1]
    return alpha, alpha * y
