"""Writes the stored expected values under tests/golden/.

Calls only the oracle (its brute-force dual route), never the CUDA library.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import rbf_kernel, squared_hinge_dual_bruteforce  # noqa: E402


def xor4():
    # XOR on the unit square, squared-hinge dual of Eq. 2 (Section 2) with
    # J = all points (Eq. 3 of Section 4 without bias).
    X = np.array([[0.0, 0.0], [1.0, 1.0], [0.0, 1.0], [1.0, 0.0]])
    y = np.array([1.0, 1.0, -1.0, -1.0])
    gamma, lam = 1.0, 0.1
    K = rbf_kernel(X, X, gamma)
    alpha, beta = squared_hinge_dual_bruteforce(K, y, lam)
    return dict(
        cite="Section 2 Eq. 2 (squared-hinge dual) and Section 4 Eq. 3/4 with J = all; "
             "RBF kernel of Section 2",
        X=X.tolist(), y=y.tolist(), gamma=gamma, lam=lam,
        alpha=alpha.tolist(), beta=beta.tolist())


if __name__ == "__main__":
    with open(os.path.join(HERE, "xor4.json"), "w") as f:
        json.dump(xor4(), f, indent=1)
    print("wrote xor4.json")
