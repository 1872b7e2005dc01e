"""The mixed form on the whole benchmark stream, checked against the plain
definition of the result.

m = n = 4096, the recommender stream (rank-1 "set item column" updates
A + b e_j^T, b a 2 % ratings column), 200 updates in the overlapped mixed
form with the library's default re-orthogonalization cadence: the form and
workload that the benchmark times.  The reference is independent of both the
GPU and the oracle's schedule: A+ = A0 + sum_h b_h e_{j_h}^T accumulated
densely in FP64 on the host, and its singular values from LAPACK.  Sec. 2
fixes sigma(Bd) = sigma(A) for orthogonal Q, P; the tolerances are the mixed
form's (singular values within 1e-5 of sigma_1, ||Q^T Q - I||_2 and
||P^T P - I||_2 at most 1e-5).
"""
import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse.linalg as sla

from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu

M = N = 4096
UPDATES = 200


def _bidiag_svals(d, e):
    """Singular values of the upper bidiagonal (d, e), descending: the
    nonnegative eigenvalues of its Golub-Kahan tridiagonal (zero diagonal,
    off-diagonal d1, e1, d2, ..., dn), from LAPACK."""
    n = d.size
    off = np.zeros(2 * n - 1)
    off[0::2] = d
    off[1::2] = e
    w = sl.eigvalsh_tridiagonal(np.zeros(2 * n), off, select="i", select_range=(n, 2 * n - 1))
    return np.sort(np.abs(w))[::-1]


def _ortho_err(X):
    """||X^T X - I||_2 in FP64 (Lanczos on the symmetric error matrix)."""
    G = X.T @ X
    G[np.diag_indices_from(G)] -= 1.0
    return float(abs(sla.eigsh(G, k=1, which="LM", return_eigenvectors=False, tol=1e-6)[0]))


def test_mixed_form_holds_its_tolerances_over_the_benchmark_stream():
    Q0, d0, e0, P0 = I.factorization(M, N, config=1)
    A = (Q0 * d0) @ P0.T
    A[:, :] += (Q0[:, :-1] * e0) @ P0[:, 1:].T
    probes = []
    with bdu.Factorization(Q0, d0, e0, P0, precision=bdu.MIXED, overlap=True) as F:
        for h in range(UPDATES):
            B, C = I.recommender_update(M, N, h, config=1)
            F.update(B, C)
            j = int(np.flatnonzero(C[:, 0])[0])
            A[:, j] += B[:, 0] * C[j, 0]
            if (h + 1) % 10 == 0:
                q_est, p_est = F.check_orthogonality()
                probes.append((h + 1, q_est, p_est))
        Q, d, e, P = F.read()
        st = F.stats()
    assert st["updates"] == UPDATES
    # the library's own estimate after every 10th update
    worst = max(max(q, p) for _, q, p in probes)
    assert worst <= 1e-5, probes
    # the same property from the factors read back, in FP64 on the host
    assert _ortho_err(Q) <= 1e-5
    assert _ortho_err(P) <= 1e-5
    # singular values: every one of the 4096, against LAPACK on the dense A+
    s_ref = np.linalg.svd(A, compute_uv=False)
    s_bd = _bidiag_svals(d, e)
    gap = np.max(np.abs(s_bd - s_ref)) / s_ref[0]
    assert gap <= 1e-5, gap
    # the relative residual ||A+ - Q Bd P^T||_F / ||A+||_F, reported; a loose
    # bound guards against a gross error that the spectrum alone could miss
    R = (Q * d) @ P.T + (Q[:, :-1] * e) @ P[:, 1:].T
    res = float(np.linalg.norm(A - R) / np.linalg.norm(A))
    print(f"\nmixed form, {UPDATES} updates at m = n = {M}: max |sigma(Bd) - sigma(A+)| / sigma_1 = {gap:.2e}, "
          f"relative residual {res:.2e}, probes (update, Q, P) {probes[-1]}")
    assert res <= 1e-3
