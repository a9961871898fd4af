"""Brute-force solution of Eq. (prob1) for tiny n by support and sign enumeration.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For a sign pattern z in {-1, 0, +1}^n with support T, a minimiser with that pattern
satisfies the restricted stationarity system of Sec. 3.2 (Eq. bd9 and the line after it),
A_T^T A_T x_T = A_T^T b - tau z_T, together with sign(x_T) = z_T and
|A_{T^c}^T (b - A_T x_T)| <= tau.  Every pattern is tried; the feasible candidate with the
smallest objective is returned.  3^n systems, so n <= 10.
"""

import itertools

import numpy as np


def brute_force(A, b, tau, slack=1e-9):
    """Minimiser of Eq. (prob1) and its objective, by enumeration of all sign patterns."""
    A = np.asarray(A.todense() if hasattr(A, "todense") else A, dtype=np.float64)
    m, n = A.shape
    if n > 12:
        raise ValueError("brute force is limited to n <= 12")
    best_x, best_f = None, np.inf
    for pattern in itertools.product((-1, 0, 1), repeat=n):
        z = np.array(pattern, dtype=np.float64)
        T = np.flatnonzero(z)
        x = np.zeros(n)
        if len(T):
            AT = A[:, T]
            M = AT.T @ AT
            if np.linalg.matrix_rank(M) < len(T):
                continue
            xT = np.linalg.solve(M, AT.T @ b - tau * z[T])
            if np.any(np.sign(xT) != z[T]):
                continue
            x[T] = xT
        atr = A.T @ (b - A @ x)
        off = np.setdiff1d(np.arange(n), T)
        if len(off) and np.any(np.abs(atr[off]) > tau * (1.0 + slack)):
            continue
        f = tau * np.abs(x).sum() + 0.5 * float((A @ x - b) @ (A @ x - b))
        if f < best_f:
            best_x, best_f = x, f
    return best_x, best_f
