"""BHU, the bidiagonal Householder update: a plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.

What BHU computes (Sec. 3.3, Algorithm 1, Theorem 1).  The update
A + b c^T = Q (B + u v^T) P^T, with u = Q^T b and v = P^T c (Eq. rk1), is
brought back to bidiagonal form by Householder reflectors applied alternately
from the left and from the right of the m x n matrix B + u v^T (m >= n):

- left reflector k zeroes column k below the diagonal, built from that column's
  entries k..m as in Sec. 2.1 (Eq. house, the sign that avoids cancellation);
- right reflector k+1 zeroes row k right of the superdiagonal, built from that
  row's entries k+1..n, so no right reflector touches column 1.

Algorithm 1 keeps the transformed matrix in the factored form of Theorem 1
(Eq. comp: B minus a rank-(2k+1) term built from the normalized reflector
vectors Y_k, W_k and the triangular T_k, R_k of Eq. TR) instead of forming it.
In exact arithmetic its reflectors and its bidiagonal are those of the dense
process, so this oracle is the dense process written out: A is formed once,
each reflector is computed from the current column or row and applied to the
whole matrix, one at a time, in the order of Algorithm 1.  Nothing is blocked,
fused or reordered.

Readings (listed with the others in the design notes):

- Algorithm 1 builds w_{k+1} from the row it writes as e_{k+1}^T A_{k,k-1}.  The
  definition of the right reflectors in Sec. 2.1 (the k-th row, its entries
  k+1..n) and the pattern of Eq. housesparse need row k, which is what is used.
- The loop of Algorithm 1 runs k = 1..n-1 (left) and exits before the right
  reflector of k = n-1: n-1 left and n-2 right reflectors, the count for
  m = n.  For m > n column n still has entries below the diagonal, so a left
  reflector k = n is added (n left reflectors).  With m = n the last diagonal
  entry and the last superdiagonal entry are read off without a reflector.
- house(x) for x = 0 is the identity (y = 0, alpha = 0).  Otherwise it is
  y = x + sign(x_1) ||x|| e_1, normalized to ||y|| = 1 (Algorithm 1 assumes
  normalized vectors), with alpha = -sign(x_1) ||x||.  sign(x_1) is the sign
  bit of x_1, so -0.0 counts as negative.  A vector already of the form
  x_1 e_1 still gets its reflector, which flips its sign.
- A partial factorization after t iterations of the loop is the matrix after
  the first t left reflectors and the right reflectors that come with them
  (Sec. 3.3: stopping early gives a partial factorization).
- Direct rank-r absorption.  Sec. 3.2 takes rank r as r repeated rank-1 steps.
  Algorithm 1 needs only the products of A with a vector, so it runs just as
  well once on B + U V^T with the r projected columns U = Q^T B, V = P^T C
  (Theorem 1's first block grows from one column to r).  The result keeps
  P's first column, as r sequential sweeps do, so by the implicit-Q theorem
  the two bidiagonals agree up to the signs of their entries.

Functions
---------
house(x)                              Eq. house, normalized (alpha, y)
bhu(d, e, u, v, m, steps=None)        Algorithm 1 on B + u v^T (dense form)
factors(Y, W, m, n)                   Q_k, P_k as explicit products (Eq. QP)
theorem1(d, e, u, v, m, Y, W)         the factored form of Eq. comp
update(Q, d, e, P, Bm, Cm)            a rank-r update by r BHU steps (Eq. bidiagplus)
update_direct(Q, d, e, P, Bm, Cm)     a rank-r update by one BHU sweep on B + U V^T
"""
import numpy as np


def house(x):
    """Sec. 2.1, Eq. house: (alpha, y) with (I - 2 y y^T) x = alpha e_1, ||y|| = 1."""
    x = np.asarray(x, dtype=np.float64)
    sigma = float(np.sqrt(np.dot(x, x)))
    if sigma == 0.0:
        return 0.0, np.zeros_like(x)
    s = np.copysign(1.0, x[0])
    y = x.copy()
    y[0] += s * sigma
    y /= np.sqrt(np.dot(y, y))
    return -s * sigma, y


def bidiag_dense(d, e, m):
    """The m x n upper bidiagonal with diagonal d and superdiagonal e."""
    n = len(d)
    B = np.zeros((m, n))
    B[np.arange(n), np.arange(n)] = d
    if n > 1:
        B[np.arange(n - 1), np.arange(1, n)] = e
    return B


def counts(m, n):
    """(left, right) reflector counts of a complete run (Algorithm 1 with the
    m > n reading)."""
    return (n if m > n else n - 1), max(n - 2, 0)


def bhu(d, e, u, v, m, steps=None):
    """Algorithm 1 (Sec. 3.3) on A = B + u v^T, written out on the dense matrix
    (u, v may also be m x r and n x r: A = B + U V^T, direct rank-r absorption).

    Returns a dict with
      alpha (steps,), beta (min(steps, n-1),): the new diagonal / superdiagonal,
      Y (m x kl), W (n x kr): the normalized reflector vectors (y_k with zeros
          above row k, w_{k+1} with zeros in rows 1..k), as in Eq. YW,
      A: the dense matrix after those reflectors (A_{kk} of Eq. arec).
    """
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    n = len(d)
    assert m >= n >= 1
    t = n if steps is None else int(steps)
    assert 0 <= t <= n
    nl, nr = counts(m, n)
    U = np.asarray(u, dtype=np.float64).reshape(m, -1)
    V = np.asarray(v, dtype=np.float64).reshape(n, -1)
    A = bidiag_dense(d, e, m) + U @ V.T
    alpha = np.zeros(t)
    beta = np.zeros(min(t, n - 1))
    Y = np.zeros((m, min(t, nl)))
    W = np.zeros((n, min(t, nr)))
    for k in range(t):
        # left: column k, rows k..m-1
        if k < nl:
            alpha[k], y = house(A[k:, k])
            Y[k:, k] = y
            A[k:, :] -= 2.0 * np.outer(y, y @ A[k:, :])
        else:
            alpha[k] = A[k, k]
        if k > n - 2:
            continue
        # right: row k, columns k+1..n-1
        if k < nr:
            beta[k], w = house(A[k, k + 1:])
            W[k + 1:, k] = w
            A[:, k + 1:] -= 2.0 * np.outer(A[:, k + 1:] @ w, w)
        else:
            beta[k] = A[k, k + 1]
    return {"alpha": alpha, "beta": beta, "Y": Y, "W": W, "A": A}


def factors(Y, W, m, n):
    """Q_k = H_1 ... H_k and P_k = H_2 ... H_{k+1} as explicit matrices (Eq. QP,
    left side: the plain product of the reflectors)."""
    Qk = np.eye(m)
    for j in range(Y.shape[1]):
        y = Y[:, j]
        Qk -= 2.0 * np.outer(Qk @ y, y)
    Pk = np.eye(n)
    for j in range(W.shape[1]):
        w = W[:, j]
        Pk -= 2.0 * np.outer(Pk @ w, w)
    return Qk, Pk


def theorem1(d, e, u, v, m, Y, W):
    """B - U M^{-1} V^T of Theorem 1 (Eq. comp) for k = Y.shape[1] = W.shape[1]
    reflectors on each side, with T_k, R_k from Eq. TR."""
    n = len(d)
    k = Y.shape[1]
    assert W.shape[1] == k
    B = bidiag_dense(d, e, m)
    T = np.eye(k) + np.triu(2.0 * (Y.T @ Y), 1)
    R = np.eye(k) + np.triu(2.0 * (W.T @ W), 1)
    u = np.asarray(u, dtype=np.float64).reshape(m, 1)
    v = np.asarray(v, dtype=np.float64).reshape(n, 1)
    U = np.hstack([u, Y, B @ W])
    V = np.hstack([v, B.T @ Y, W])
    M = np.zeros((1 + 2 * k, 1 + 2 * k))
    M[0, 0] = -1.0
    M[0, 1 + k:] = (v.T @ W).ravel()
    M[1:1 + k, 0] = (Y.T @ u).ravel()
    M[1:1 + k, 1:1 + k] = 0.5 * T.T
    M[1:1 + k, 1 + k:] = Y.T @ B @ W
    M[1 + k:, 1 + k:] = 0.5 * R
    return B - U @ np.linalg.solve(M, V.T)


def update(Q, d, e, P, Bm, Cm):
    """Rank-r update A + Bm Cm^T by r BHU steps (Sec. 3.2, Eq. bidiagplus: rank r
    as r rank-1 steps): u = Q^T b, v = P^T c, Algorithm 1, then Q <- Q Q_k,
    P <- P P_k and (d, e) <- (alpha, beta)."""
    Q = np.array(Q, dtype=np.float64, copy=True)
    P = np.array(P, dtype=np.float64, copy=True)
    d = np.array(d, dtype=np.float64, copy=True)
    e = np.array(e, dtype=np.float64, copy=True)
    m, n = Q.shape[0], P.shape[0]
    Bm = np.asarray(Bm, dtype=np.float64).reshape(m, -1)
    Cm = np.asarray(Cm, dtype=np.float64).reshape(n, -1)
    for k in range(Bm.shape[1]):
        u = Q.T @ Bm[:, k]
        v = P.T @ Cm[:, k]
        r = bhu(d, e, u, v, m)
        Qk, Pk = factors(r["Y"], r["W"], m, n)
        Q = Q @ Qk
        P = P @ Pk
        d = r["alpha"]
        e = r["beta"]
    return Q, d, e, P


def update_direct(Q, d, e, P, Bm, Cm):
    """Rank-r update A + Bm Cm^T by one BHU sweep on B + U V^T with U = Q^T Bm,
    V = P^T Cm (direct rank-r absorption), then Q <- Q Q_k, P <- P P_k and
    (d, e) <- (alpha, beta)."""
    Q = np.array(Q, dtype=np.float64, copy=True)
    P = np.array(P, dtype=np.float64, copy=True)
    m, n = Q.shape[0], P.shape[0]
    U = Q.T @ np.asarray(Bm, dtype=np.float64).reshape(m, -1)
    V = P.T @ np.asarray(Cm, dtype=np.float64).reshape(n, -1)
    r = bhu(d, e, U, V, m)
    Qk, Pk = factors(r["Y"], r["W"], m, n)
    return Q @ Qk, r["alpha"], r["beta"], P @ Pk


# ---------------------------------------------------------------------------
# The symmetric variant (Sec. 6, future directions: the updating algorithms
# adapted to generate a tridiagonal).  A = Q T Q^T with T symmetric tridiagonal
# (diagonal a, off-diagonal b); A + rho c c^T = Q (T + rho u u^T) Q^T with
# u = Q^T c.  The same process as Algorithm 1 with one reflector per step
# applied on both sides: column k's entries k+1..n give reflector k (Eq. house),
# which acts on rows and columns k+1..n, so Q's first column is kept.  Readings:
# n-2 reflectors (k = 1..n-2); the last off-diagonal entry and the diagonal
# entries are read off the transformed matrix.
# ---------------------------------------------------------------------------

def tridiag_dense(a, b):
    """The symmetric tridiagonal with diagonal a and off-diagonal b."""
    n = len(a)
    T = np.diag(np.asarray(a, dtype=np.float64))
    if n > 1:
        T += np.diag(np.asarray(b, dtype=np.float64), 1) + np.diag(np.asarray(b, dtype=np.float64), -1)
    return T


def tri(a, b, u, rho, steps=None):
    """Householder tridiagonalization of T + rho u u^T, written out on the dense
    matrix.  Returns alpha (steps,), beta (min(steps, n-1),), Y (n x k, the
    normalized vectors, y_k with zeros in rows 1..k) and the transformed A."""
    a = np.asarray(a, dtype=np.float64)
    n = len(a)
    t = n if steps is None else int(steps)
    nt = max(n - 2, 0)
    u = np.asarray(u, dtype=np.float64)
    A = tridiag_dense(a, b) + rho * np.outer(u, u)
    alpha = np.zeros(t)
    beta = np.zeros(min(t, n - 1))
    Y = np.zeros((n, min(t, nt)))
    for k in range(t):
        alpha[k] = A[k, k]
        if k < nt:
            beta[k], y = house(A[k + 1:, k])
            Y[k + 1:, k] = y
            A[k + 1:, :] -= 2.0 * np.outer(y, y @ A[k + 1:, :])
            A[:, k + 1:] -= 2.0 * np.outer(A[:, k + 1:] @ y, y)
        elif k == n - 2:
            beta[k] = A[k + 1, k]
    return {"alpha": alpha, "beta": beta, "Y": Y, "A": A}


def tri_update(Q, a, b, rho, c):
    """A + rho c c^T for A = Q T Q^T: u = Q^T c, the tridiagonalization of
    T + rho u u^T, Q <- Q Q_k; returns (Q, alpha, beta)."""
    Q = np.asarray(Q, dtype=np.float64)
    n = Q.shape[0]
    r = tri(a, b, Q.T @ np.asarray(c, dtype=np.float64), rho)
    Qk, _ = factors(r["Y"], np.zeros((1, 0)), n, 1)
    return Q @ Qk, r["alpha"], r["beta"]
