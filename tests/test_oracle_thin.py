"""Pins of the oracle's rank-k tracking step (Sec. 4, Eqs. lrup - bdlrup),
each checked against what the mathematics fixes rather than against the
oracle's own formulas: the untruncated factorization reproduces A + b c^T,
the truncation error it reports is the true Frobenius error, the factors stay
orthonormal (also when b lies in span(Q1)), and a stream that never exceeds
rank k is tracked exactly, with the singular values of the sum."""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import inputs as I


def _start(m, n, k, which, zero=False):
    g = np.random.default_rng(1000 + which)
    Q1 = I.householder_orthogonal(m, g)[:, :k]
    P1 = I.householder_orthogonal(n, g)[:, :k]
    d = np.zeros(k) if zero else g.uniform(1.0, 10.0, k)
    e = np.zeros(k - 1) if zero else g.standard_normal(k - 1)
    return Q1, d, e, P1, g


def _dense(Q1, d, e, P1):
    return Q1 @ O.bidiag_dense(d, e) @ P1.T


@pytest.mark.parametrize("m,n,k", [(60, 40, 8), (33, 90, 5), (20, 20, 1), (50, 50, 12)])
def test_untruncated_factorization_is_exact(m, n, k):
    Q1, d, e, P1, g = _start(m, n, k, 1)
    b = g.standard_normal(m); c = g.standard_normal(n)
    A = _dense(Q1, d, e, P1) + np.outer(b, c)
    *_, (Qf, df, ef, Pf) = O.thin_update(Q1, d, e, P1, b, c, full=True)
    assert Qf.shape == (m, k + 1) and Pf.shape == (n, k + 1)
    assert np.linalg.norm(Qf @ O.bidiag_dense(df, ef) @ Pf.T - A) <= 1e-13 * np.linalg.norm(A)
    assert np.linalg.norm(Qf.T @ Qf - np.eye(k + 1)) <= 1e-13 * k
    assert np.linalg.norm(Pf.T @ Pf - np.eye(k + 1)) <= 1e-13 * k


@pytest.mark.parametrize("m,n,k", [(60, 40, 8), (33, 90, 5), (70, 70, 3)])
def test_reported_error_is_the_frobenius_error(m, n, k):
    Q1, d, e, P1, g = _start(m, n, k, 2)
    A = _dense(Q1, d, e, P1)
    for h in range(6):
        b = g.standard_normal(m) * (1 + h); c = g.standard_normal(n)
        A = _dense(Q1, d, e, P1) + np.outer(b, c)
        Q1, d, e, P1, i, err2 = O.thin_update(Q1, d, e, P1, b, c)
        assert 0 <= i <= k and len(d) == k and len(e) == k - 1
        res = np.linalg.norm(A - _dense(Q1, d, e, P1)) ** 2
        assert abs(res - err2) <= 1e-12 * np.linalg.norm(A) ** 2
        assert np.linalg.norm(Q1.T @ Q1 - np.eye(k)) <= 1e-13 * k
        assert np.linalg.norm(P1.T @ P1 - np.eye(k)) <= 1e-13 * k


def test_stream_within_rank_k_is_tracked_exactly():
    """From B = 0, five rank-1 terms with k = 7: nothing is lost, and the
    singular values are those of the sum."""
    m, n, k = 45, 38, 7
    Q1, d, e, P1, g = _start(m, n, k, 3, zero=True)
    S = np.zeros((m, n))
    for h in range(5):
        b = g.standard_normal(m); c = g.standard_normal(n)
        S += np.outer(b, c)
        Q1, d, e, P1, i, err2 = O.thin_update(Q1, d, e, P1, b, c)
        assert err2 == 0.0
    assert np.linalg.norm(_dense(Q1, d, e, P1) - S) <= 1e-13 * np.linalg.norm(S)
    sv = np.linalg.svd(S, compute_uv=False)[:k]
    np.testing.assert_allclose(O.singular_values(d, e), sv, rtol=0, atol=1e-13 * sv[0])


def test_update_inside_the_subspace():
    """b = Q1 x (delta = 0) and c = P1 y (gamma = 0): the fill direction keeps
    the factors orthonormal and the error identity holds."""
    m, n, k = 40, 30, 6
    Q1, d, e, P1, g = _start(m, n, k, 4)
    b = Q1 @ g.standard_normal(k); c = P1 @ g.standard_normal(k)
    A = _dense(Q1, d, e, P1) + np.outer(b, c)
    Q2, d2, e2, P2, i, err2 = O.thin_update(Q1, d, e, P1, b, c)
    assert np.linalg.norm(Q2.T @ Q2 - np.eye(k)) <= 1e-13 * k
    assert np.linalg.norm(P2.T @ P2 - np.eye(k)) <= 1e-13 * k
    assert abs(np.linalg.norm(A - _dense(Q2, d2, e2, P2)) ** 2 - err2) <= 1e-12 * np.linalg.norm(A) ** 2
    # A+ has rank <= k here; the column dropped is the one of the fill direction
    assert i == k and err2 <= 1e-24 * np.linalg.norm(A) ** 2


def test_fill_vector_is_orthogonalizable():
    z = O.fill_vector(1000)
    assert np.all(np.abs(z) <= 0.5) and abs(z.mean()) < 0.01
    assert z[0] == -0.5 and z[1] == O.GOLDEN - 0.5


def test_hand_derived_rank_one_step():
    """k = 1, m = n = 2, Q1 = P1 = e1, B = [alpha], b = beta e2, c = e1:
    A+ = (alpha e1 + beta e2) e1^T has sigma = hypot(alpha, beta), so one
    tracking step loses nothing and gives Q1+ = +-(alpha, beta) / sigma,
    P1+ = +-e1 (c lies in span(P1): gamma = 0)."""
    alpha, beta = 3.0, -4.0
    Q1 = np.array([[1.0], [0.0]]); P1 = np.array([[1.0], [0.0]])
    Q2, d2, e2, P2, i, err2 = O.thin_update(Q1, [alpha], [], P1, [0.0, beta], [1.0, 0.0])
    assert abs(abs(d2[0]) - 5.0) <= 1e-15 * 5.0 and len(e2) == 0
    assert err2 == 0.0 and i == 1
    q = Q2[:, 0] * np.sign(Q2[0, 0])
    np.testing.assert_allclose(q, [0.6, -0.8], rtol=0, atol=1e-15)
    np.testing.assert_allclose(np.abs(P2[:, 0]), [1.0, 0.0], rtol=0, atol=1e-15)
