"""Pins of the oracle's backward error, shared by tests/test_oracle.py and the
mutation test.  The values are worked out by hand below, independently of
the oracle's code.

A = [[4, 1, 0], [1, 3, 1], [0, 1, 2]] (SPD; leading minors 4, 11, 18),
||A||_inf = max row sum of |a_ij| = max(5, 5, 3) = 5.

Column 1: x* = (1, -1, 2), b = A x* = (3, 0, 3).  With x = x* + (0, 0.5, 0):
A x = (3.5, 1.5, 3.5), r = b - A x = (-0.5, -1.5, -0.5), ||r|| = 1.5,
||x|| = 2, ||b|| = 3, berr = 1.5 / (5 * 2 + 3) = 1.5 / 13.

Column 2: x* = (0, 1, 0), b = (1, 3, 1).  With x = (0.25, 1, 0):
A x = (2, 3.25, 1), r = (-1, -0.25, 0), ||r|| = 1, ||x|| = 1, ||b|| = 3,
berr = 1 / (5 * 1 + 3) = 1 / 8.

The oracle's berr is the maximum over the columns: 1 / 8.  Exact solutions
give 0 exactly (integer data), and scaling x and b together leaves berr
unchanged.
"""
import numpy as np

# A in CSR, columns of each row deliberately unsorted
RP = np.array([0, 2, 5, 7], dtype=np.int64)
CI = np.array([1, 0, 2, 0, 1, 2, 1], dtype=np.int32)
VX = np.array([1.0, 4.0, 1.0, 1.0, 3.0, 2.0, 1.0])
B = np.array([[3.0, 1.0], [0.0, 3.0], [3.0, 1.0]])
X_EXACT = np.array([[1.0, 0.0], [-1.0, 1.0], [2.0, 0.0]])
X_PERT = np.array([[1.0, 0.25], [-0.5, 1.0], [2.0, 0.0]])


def failures(berr):
    """Names of the hand-computed pins that `berr` (signature of
    oracle.berr) fails."""
    bad = set()

    def check(name, ok):
        if not ok:
            bad.add(name)

    try:
        check("exact solution", berr(RP, CI, VX, X_EXACT, B) == 0.0)
        check("column 1", abs(berr(RP, CI, VX, X_PERT[:, 0], B[:, 0]) - 1.5 / 13) <= 1e-16)
        check("column 2", abs(berr(RP, CI, VX, X_PERT[:, 1], B[:, 1]) - 1.0 / 8) <= 1e-16)
        check("max over columns", abs(berr(RP, CI, VX, X_PERT, B) - 1.0 / 8) <= 1e-16)
        check("scale invariance",
              abs(berr(RP, CI, VX, 3.0 * X_PERT, 3.0 * B) - 1.0 / 8) <= 1e-16)
    except Exception:
        bad.add("raised")
    return bad
