"""Pins of the oracle's m < n form (A = Q L P^T with L lower bidiagonal,
updated through its transpose).  Sec. 1 states the factorization with an
upper bidiagonal and Algorithm 2 covers m >= n; for m < n the reading is the
transposed problem, and these checks hold it to the definition itself: the
reconstruction of A + B C^T, orthogonal factors, the singular values of A+,
the Frobenius identity, the rank-1 closed form from L = 0, and the vector
that no rotation touches."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import inputs as I


def _dense(Q, d, e, P):
    m, n = Q.shape[0], P.shape[0]
    return Q @ O.lower_bidiag_dense(d, e, m, n) @ P.T


@pytest.mark.parametrize("m,n,r", [(20, 35, 1), (31, 80, 3), (1, 5, 2), (2, 3, 1), (49, 50, 2)])
def test_lower_reconstruction_and_orthogonality(m, n, r):
    Q, d, e, P = I.factorization(m, n, config=0, which=5)
    assert len(d) == m and len(e) == m - 1
    B, C = I.dense_update(m, n, h=3, config=0, r=r)
    A = _dense(Q, d, e, P) + B @ C.T
    Q2, d2, e2, P2, cnt = O.update_lower(Q, d, e, P, B, C)
    assert len(d2) == m and len(e2) == m - 1
    assert np.linalg.norm(_dense(Q2, d2, e2, P2) - A) <= 1e-13 * np.linalg.norm(A)
    assert np.linalg.norm(Q2.T @ Q2 - np.eye(m)) <= 1e-13 * m
    assert np.linalg.norm(P2.T @ P2 - np.eye(n)) <= 1e-13 * n
    # the vector that no rotation touches is Q(:,1) in this form
    assert np.array_equal(Q2[:, 0], Q[:, 0])
    assert cnt["band_violations"] == 0 and cnt["zero_violations"] == 0


@pytest.mark.parametrize("m,n", [(12, 30), (40, 41)])
def test_lower_singular_values_are_those_of_a(m, n):
    Q, d, e, P = I.factorization(m, n, config=0, which=9)
    A = _dense(Q, d, e, P)
    for h in range(3):
        B, C = I.dense_update(m, n, h=h, config=0, r=2)
        A = A + B @ C.T
        Q, d, e, P, _ = O.update_lower(Q, d, e, P, B, C)
    sv = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(O.singular_values(d, e), sv, rtol=0, atol=1e-12 * sv[0])
    np.testing.assert_allclose(O.jacobi_sv(O.lower_bidiag_dense(d, e, m, n)), sv, rtol=0, atol=1e-12 * sv[0])


def test_lower_frobenius_identity():
    """||L+||_F^2 = ||L||_F^2 + 2 u^T L v + ||u||^2 ||v||^2, u = Q^T b, v = P^T c."""
    m, n = 33, 70
    Q, d, e, P = I.factorization(m, n, config=0, which=13)
    B, C = I.dense_update(m, n, h=7, config=0, r=1)
    u = Q.T @ B[:, 0]; v = P.T @ C[:, 0]
    L = O.lower_bidiag_dense(d, e, m, n)
    want = np.sum(d ** 2) + np.sum(e ** 2) + 2 * u @ L @ v + (u @ u) * (v @ v)
    _, d2, e2, _, _ = O.update_lower(Q, d, e, P, B, C)
    assert abs(np.sum(d2 ** 2) + np.sum(e2 ** 2) - want) < 1e-13 * want


def test_lower_zero_start_closed_form():
    """L = 0, rank 1: A+ = b c^T has sigma_1 = ||b|| ||c||, one nonzero pair
    (d_1, e_1) and P+(:,1) = +-c / ||c||; Q(:,1) is kept, so |d_1| = ||c|| |q_1^T b|."""
    m, n = 18, 40
    Q, _, _, P = I.factorization(m, n, config=0, which=21)
    d = np.zeros(m); e = np.zeros(m - 1)
    g = np.random.default_rng(5)
    b = g.standard_normal(m); c = g.standard_normal(n)
    Q2, d2, e2, P2, _ = O.update_lower(Q, d, e, P, b, c)
    nb, nc, qb = np.linalg.norm(b), np.linalg.norm(c), Q[:, 0] @ b
    assert abs(math.hypot(d2[0], e2[0]) - nb * nc) < 1e-13 * nb * nc
    assert abs(abs(d2[0]) - nc * abs(qb)) < 1e-13 * nb * nc
    assert abs(abs(e2[0]) - nc * math.sqrt(nb ** 2 - qb ** 2)) < 1e-13 * nb * nc
    assert np.all(d2[1:] == 0.0) and np.all(e2[1:] == 0.0)
    p1 = P2[:, 0] * np.sign(P2[:, 0] @ c)
    np.testing.assert_allclose(p1, c / nc, atol=1e-14)


def test_lower_pins_reject_the_upper_reading():
    """The reconstruction pin tells the lower band from an upper one: reading
    the same d, e as an m x n upper bidiagonal misses A + B C^T."""
    m, n = 15, 28
    Q, d, e, P = I.factorization(m, n, config=0, which=2)
    B, C = I.dense_update(m, n, h=1, config=0, r=1)
    A = _dense(Q, d, e, P) + B @ C.T
    Q2, d2, e2, P2, _ = O.update_lower(Q, d, e, P, B, C)
    U = np.zeros((m, n))
    U[np.arange(m), np.arange(m)] = d2
    U[np.arange(m - 1), np.arange(1, m)] = e2
    assert np.linalg.norm(Q2 @ U @ P2.T - A) > 1e-3 * np.linalg.norm(A)


def test_lower_rejects_m_at_least_n():
    Q, d, e, P = I.factorization(6, 4, config=0, which=1)
    with pytest.raises(ValueError):
        O.update_lower(Q, d, e, P, np.ones(6), np.ones(4))
