"""Textbook bidiagonalizations used to pin the oracle (test infrastructure).

Both routines are independent of the Givens update: they bidiagonalize a
dense matrix from scratch.  When the right transformations never touch the
first column (Householder, Sec. 2.2: right reflectors start at column k+1)
or the Lanczos start vector is e_1 (GKB, Sec. 2.3), the bidiagonal of
X = A+ P is unique up to signs whenever it is unreduced, so |alpha|, |beta|
must agree with the oracle's |d+|, |e+|.
"""
import numpy as np


def _reflector(x):
    """y, tau with (I - tau y y^T) x = -sign(x0) ||x|| e_1 (Eq. house)."""
    y = np.array(x, dtype=np.float64, copy=True)
    nx = np.linalg.norm(y)
    if nx == 0.0:
        return y, 0.0
    y[0] += np.copysign(nx, y[0])
    return y, 2.0 / np.dot(y, y)


def householder_bidiag(X):
    """Alternating left/right Householder bidiagonalization of X (m >= n).

    Returns (alpha, beta): the diagonal and superdiagonal of the upper
    bidiagonal B with X = Q B P^T, where P e_1 = e_1 (Sec. 2.2,
    Eq. housesparse).
    """
    A = np.array(X, dtype=np.float64, copy=True)
    m, n = A.shape
    for k in range(n):
        y, tau = _reflector(A[k:, k])
        A[k:, k:] -= tau * np.outer(y, y @ A[k:, k:])
        if k < n - 2:
            y, tau = _reflector(A[k, k + 1:])
            A[k:, k + 1:] -= tau * np.outer(A[k:, k + 1:] @ y, y)
    return np.diag(A)[:n].copy(), np.diag(A, 1)[: n - 1].copy()


def gkb_full_reorth(X, p1, steps=None):
    """Golub-Kahan bidiagonalization (Eqs. recp, recq) from the unit vector p1,
    with full reorthogonalization of both bases.  Returns (alpha, beta)."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    steps = n if steps is None else steps
    Qb = np.zeros((m, steps)); Pb = np.zeros((n, steps))
    alpha = np.zeros(steps); beta = np.zeros(max(steps - 1, 0))
    p = np.asarray(p1, dtype=np.float64) / np.linalg.norm(p1)
    Pb[:, 0] = p
    q_prev = np.zeros(m)
    for k in range(steps):
        w = X @ Pb[:, k] - (beta[k - 1] * q_prev if k > 0 else 0.0)
        for _ in range(2):
            w -= Qb[:, :k] @ (Qb[:, :k].T @ w)
        alpha[k] = np.linalg.norm(w)
        Qb[:, k] = w / alpha[k]
        q_prev = Qb[:, k]
        if k + 1 < steps:
            z = X.T @ Qb[:, k] - alpha[k] * Pb[:, k]
            for _ in range(2):
                z -= Pb[:, : k + 1] @ (Pb[:, : k + 1].T @ z)
            beta[k] = np.linalg.norm(z)
            Pb[:, k + 1] = z / beta[k]
    return alpha, beta
