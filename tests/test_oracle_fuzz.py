"""Randomized small problems with structured exact zeros (zero entries of d
and e, sparse or zero columns of B and C, m > n spikes, m < n, ranks above 1),
each held to the definition: the factorization reproduces A + B C^T, the
factors stay orthogonal, the vector no rotation may touch is unchanged, and
the oracle's own band and exact-zero checks stay silent (it raises otherwise).
Seeded, so every run draws the same cases."""
import numpy as np

import oracle as O
from paper_2509_02840_gb300 import inputs as I


def _case(rng):
    n = int(rng.integers(1, 9))
    m = n + int(rng.integers(0, 5))
    r = int(rng.integers(1, 4))
    Q = I.householder_orthogonal(m, rng)
    P = I.householder_orthogonal(n, rng)
    d = rng.standard_normal(n) * (rng.random(n) > 0.3)
    e = rng.standard_normal(max(n - 1, 0)) * (rng.random(max(n - 1, 0)) > 0.3)
    B = rng.standard_normal((m, r)) * (rng.random((m, r)) > 0.5)
    C = rng.standard_normal((n, r)) * (rng.random((n, r)) > 0.5)
    if rng.random() < 0.1:
        B[:] = 0.0
    if rng.random() < 0.1:
        C[:] = 0.0
    return Q, d, e, P, B, C


def test_upper_form_with_structured_zeros():
    rng = np.random.default_rng(20250902)
    for _ in range(600):
        Q, d, e, P, B, C = _case(rng)
        m, n = Q.shape[0], P.shape[0]
        A = Q @ O.bidiag_dense(d, e, m) @ P.T + B @ C.T
        Q2, d2, e2, P2, _ = O.update(Q, d, e, P, B, C)
        R = Q2 @ O.bidiag_dense(d2, e2, m) @ P2.T
        assert np.linalg.norm(R - A) <= 1e-13 * max(np.linalg.norm(A), 1e-300)
        assert np.linalg.norm(Q2.T @ Q2 - np.eye(m)) <= 1e-13
        assert np.linalg.norm(P2.T @ P2 - np.eye(n)) <= 1e-13
        assert np.array_equal(P2[:, 0], P[:, 0])


def test_lower_form_with_structured_zeros():
    rng = np.random.default_rng(20250903)
    for _ in range(300):
        Qt, d, e, Pt, Bt, Ct = _case(rng)
        if Qt.shape[0] == Pt.shape[0]:
            continue
        # the transposed shapes: m < n
        Q, P, B, C = Pt, Qt, Ct, Bt
        m, n = Q.shape[0], P.shape[0]
        A = Q @ O.lower_bidiag_dense(d, e, m, n) @ P.T + B @ C.T
        Q2, d2, e2, P2, _ = O.update_lower(Q, d, e, P, B, C)
        R = Q2 @ O.lower_bidiag_dense(d2, e2, m, n) @ P2.T
        assert np.linalg.norm(R - A) <= 1e-13 * max(np.linalg.norm(A), 1e-300)
        assert np.array_equal(Q2[:, 0], Q[:, 0])


def test_rank_k_tracking_error_identity():
    rng = np.random.default_rng(20250904)
    for _ in range(150):
        k = int(rng.integers(1, 6))
        m = k + 1 + int(rng.integers(0, 8))
        n = k + 1 + int(rng.integers(0, 8))
        Q1 = np.linalg.qr(rng.standard_normal((m, k)))[0]
        P1 = np.linalg.qr(rng.standard_normal((n, k)))[0]
        d = rng.standard_normal(k) * (rng.random(k) > 0.3)
        e = rng.standard_normal(k - 1) * (rng.random(k - 1) > 0.3)
        b = rng.standard_normal(m) * (rng.random(m) > 0.4)
        c = rng.standard_normal(n) * (rng.random(n) > 0.4)
        if rng.random() < 0.2:
            b = Q1 @ rng.standard_normal(k)
        A = Q1 @ O.bidiag_dense(d, e) @ P1.T + np.outer(b, c)
        Q2, d2, e2, P2, i, err2 = O.thin_update(Q1, d, e, P1, b, c)
        res = np.linalg.norm(A - Q2 @ O.bidiag_dense(d2, e2) @ P2.T) ** 2
        assert abs(res - err2) <= 1e-12 * max(np.linalg.norm(A) ** 2, 1e-300)
        assert np.linalg.norm(Q2.T @ Q2 - np.eye(k)) <= 1e-12
        assert np.linalg.norm(P2.T @ P2 - np.eye(k)) <= 1e-12
