"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: each checks the oracle's result
against a definition (reconstruction of A + B C^T, orthogonality, exact band
zeros), a closed form, a hand-derived example, or an independent textbook
routine (Householder and Golub-Kahan bidiagonalization, one-sided Jacobi,
LAPACK SVD through numpy).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle.textbook import gkb_full_reorth, householder_bidiag
from paper_2509_02840_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_A(Q, d, e, P):
    return Q @ O.bidiag_dense(d, e, Q.shape[0]) @ P.T


def rel_resid(Aplus, Q, d, e, P):
    return np.linalg.norm(Aplus - dense_A(Q, d, e, P)) / np.linalg.norm(Aplus)


# --------------------------------------------------------------------------
# rotation generator (Eqs. giv, giv1 and the zero handling of Sec. 3.4)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("f,g", [(3.0, 4.0), (-3.0, 4.0), (3.0, -4.0), (1e300, 1e300),
                                 (1e-300, 3e-300), (-2.5e-170, 7e-170), (1.0, 1e-20)])
def test_rot_zeroes_second_component(f, g):
    ok, c, s, r = O.rot(f, g)
    assert ok
    assert abs(c * c + s * s - 1.0) < 4e-16
    assert math.isfinite(r) and r != 0.0
    assert math.copysign(1.0, r) == math.copysign(1.0, f) and c > 0
    scale = max(abs(f), abs(g))
    assert abs((c * f + s * g) - r) <= 4e-16 * scale
    assert abs(-s * f + c * g) <= 4e-16 * scale
    assert abs(abs(r) - math.hypot(f, g)) <= 4e-16 * math.hypot(f, g)


def test_rot_textbook_values():
    assert O.rot(3.0, 4.0)[1:] == pytest.approx((0.6, 0.8, 5.0), abs=1e-16)
    assert O.rot(-3.0, 4.0)[1:] == pytest.approx((0.6, -0.8, -5.0), abs=1e-16)
    # f == 0: the permutation case, c = 0, s = 1, r = g
    assert O.rot(0.0, -2.0) == (True, 0.0, 1.0, -2.0)
    # g == 0: no rotation
    assert O.rot(5.0, 0.0)[0] is False
    assert O.rot(0.0, 0.0)[0] is False


# --------------------------------------------------------------------------
# hand-derived worked examples (tests/golden)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["n2_worked_example.json", "n1_worked_example.json"])
def test_golden_worked_examples(name):
    fx = json.load(open(os.path.join(GOLDEN, name)))
    m, n = fx["m"], fx["n"]
    Q = np.array(fx["Q"]); P = np.array(fx["P"])
    d = np.array(fx["d"]); e = np.array(fx["e"]) if n > 1 else np.zeros(0)
    b = np.array(fx["b"]).reshape(m, 1); c = np.array(fx["c"]).reshape(n, 1)
    _, d2, e2, _, _ = O.update(Q, d, e, P, b, c)
    want_d = [eval(x, {"sqrt": math.sqrt}) for x in fx["abs_d"]]
    want_e = [eval(x, {"sqrt": math.sqrt}) for x in fx["abs_e"]]
    np.testing.assert_allclose(np.abs(d2), want_d, rtol=1e-15, atol=0)
    np.testing.assert_allclose(np.abs(e2), want_e, rtol=1e-15, atol=0)


# --------------------------------------------------------------------------
# the plain definition: Q+ Bd+ P+^T = A + B C^T, orthogonality, band zeros
# --------------------------------------------------------------------------
SHAPES = [(1, 1), (2, 1), (5, 1), (2, 2), (3, 2), (3, 3), (4, 3), (5, 4), (8, 8), (9, 8),
          (17, 5), (33, 33), (40, 39), (64, 16), (100, 100), (130, 97)]


@pytest.mark.parametrize("m,n", SHAPES)
@pytest.mark.parametrize("r", [1, 3])
def test_reconstruction_orthogonality(m, n, r):
    Q, d, e, P = I.factorization(m, n, config=0, which=m * 1000 + n)
    B, C = I.dense_update(m, n, h=r, config=0, r=r)
    Aplus = dense_A(Q, d, e, P) + B @ C.T
    Q2, d2, e2, P2, cnt = O.update(Q, d, e, P, B, C)
    assert cnt["band_violations"] == 0 and cnt["zero_violations"] == 0
    assert rel_resid(Aplus, Q2, d2, e2, P2) < 1e-14 * max(1, math.sqrt(n))
    assert np.linalg.norm(Q2.T @ Q2 - np.eye(m), 2) < 1e-13
    assert np.linalg.norm(P2.T @ P2 - np.eye(n), 2) < 1e-13
    # the schedule never rotates column 1 of P
    assert np.array_equal(P2[:, 0], P[:, 0])
    if m > n + 1:
        assert cnt["left"]["spike"] > 0


def test_stream_of_updates_config0_shape():
    """20 sequential rank-1 updates at m=256, n=128 against A accumulated exactly in FP64."""
    m, n = 256, 128
    Q, d, e, P = I.factorization(m, n, config=0)
    A = dense_A(Q, d, e, P)
    for h in range(20):
        B, C = I.dense_update(m, n, h, config=0)
        A = A + B @ C.T
        Q, d, e, P, cnt = O.update(Q, d, e, P, B, C)
        assert cnt["zero_violations"] == 0 and cnt["band_violations"] == 0
    assert rel_resid(A, Q, d, e, P) < 1e-13
    assert np.linalg.norm(Q.T @ Q - np.eye(m), 2) < 1e-12
    assert np.linalg.norm(P.T @ P - np.eye(n), 2) < 1e-12


# --------------------------------------------------------------------------
# independent textbook bidiagonalizations (uniqueness with P+(:,1) = P(:,1))
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,n", [(12, 12), (40, 25), (128, 128), (200, 150)])
def test_householder_and_gkb_agree(m, n):
    Q, d, e, P = I.factorization(m, n, config=0, which=7 + m)
    B, C = I.dense_update(m, n, h=3, config=0, r=2)
    Aplus = dense_A(Q, d, e, P) + B @ C.T
    _, d2, e2, _, _ = O.update(Q, d, e, P, B, C)
    scale = np.linalg.norm(Aplus, 2)
    ha, hb = householder_bidiag(Aplus @ P)
    np.testing.assert_allclose(np.abs(d2), np.abs(ha), rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(np.abs(e2), np.abs(hb), rtol=0, atol=1e-12 * scale)
    ga, gb = gkb_full_reorth(Aplus, P[:, 0])
    np.testing.assert_allclose(np.abs(d2), ga, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(np.abs(e2), gb, rtol=0, atol=1e-12 * scale)


def test_textbook_routines_themselves():
    """Both pins reproduce a known bidiagonal: X = Q0 Bd P0^T with P0 e1 = e1.

    The size is small and the off-diagonal comparable to the diagonal, so that
    the Krylov basis from e_1 is well conditioned: otherwise the trailing
    bidiagonal entries are ill-conditioned functions of X and rounding alone
    moves them, although every routine is backward stable."""
    g = np.random.default_rng(5)
    n = 10
    d = g.uniform(1, 2, n); e = g.uniform(1, 2, n - 1)
    Q0 = I.householder_orthogonal(n, g)
    P0 = np.eye(n); P0[1:, 1:] = I.householder_orthogonal(n - 1, g)
    X = Q0 @ O.bidiag_dense(d, e) @ P0.T
    ha, hb = householder_bidiag(X)
    np.testing.assert_allclose(np.abs(ha), d, rtol=1e-12)
    np.testing.assert_allclose(np.abs(hb), e, rtol=1e-12)
    ga, gb = gkb_full_reorth(X, np.eye(n)[:, 0])
    np.testing.assert_allclose(ga, d, rtol=1e-12)
    np.testing.assert_allclose(gb, e, rtol=1e-12)


# --------------------------------------------------------------------------
# singular values: one-sided Jacobi (tiny) and LAPACK through numpy
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,n", [(4, 4), (7, 5), (16, 16), (24, 10)])
def test_singular_values_jacobi(m, n):
    Q, d, e, P = I.factorization(m, n, config=0, which=99 + n)
    B, C = I.dense_update(m, n, h=5, config=0, r=1)
    Aplus = dense_A(Q, d, e, P) + B @ C.T
    _, d2, e2, _, _ = O.update(Q, d, e, P, B, C)
    sv_core = O.jacobi_sv(O.bidiag_dense(d2, e2))
    sv_A = O.jacobi_sv(Aplus)
    np.testing.assert_allclose(sv_core, sv_A[:n], rtol=1e-12, atol=1e-14 * sv_A[0])
    np.testing.assert_allclose(sv_core, np.linalg.svd(Aplus, compute_uv=False)[:n], rtol=1e-12,
                               atol=1e-14 * sv_A[0])


def test_jacobi_against_lapack():
    X = np.random.default_rng(3).standard_normal((9, 6))
    np.testing.assert_allclose(O.jacobi_sv(X), np.linalg.svd(X, compute_uv=False), rtol=1e-13)


# --------------------------------------------------------------------------
# invariants and closed forms
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,n", [(50, 50), (80, 31)])
def test_frobenius_identity(m, n):
    """||Bd+||_F^2 = ||Bd||_F^2 + 2 u^T Bd v + ||u||^2 ||v||^2 (orthogonal invariance)."""
    Q, d, e, P = I.factorization(m, n, config=0, which=3)
    B, C = I.dense_update(m, n, h=11, config=0, r=1)
    u = Q.T @ B[:, 0]; v = P.T @ C[:, 0]
    Bd = O.bidiag_dense(d, e, m)
    want = np.sum(d ** 2) + np.sum(e ** 2) + 2 * u @ Bd @ v + (u @ u) * (v @ v)
    _, d2, e2, _, _ = O.update(Q, d, e, P, B, C)
    assert abs(np.sum(d2 ** 2) + np.sum(e2 ** 2) - want) < 1e-13 * want


@pytest.mark.parametrize("m,n", [(30, 30), (45, 20)])
def test_zero_start_closed_form(m, n):
    """Bd = 0 (a stream that starts from zero, Eq. stream): rank-1 closed form."""
    Q, _, _, P = I.factorization(m, n, config=0, which=42)
    d = np.zeros(n); e = np.zeros(n - 1)
    g = np.random.default_rng(1)
    b = g.standard_normal(m); c = g.standard_normal(n)
    Q2, d2, e2, P2, _ = O.update(Q, d, e, P, b, c)
    nb, nc, pc = np.linalg.norm(b), np.linalg.norm(c), P[:, 0] @ c
    assert abs(abs(d2[0]) - nb * abs(pc)) < 1e-13 * nb * nc
    assert abs(abs(e2[0]) - nb * math.sqrt(nc ** 2 - pc ** 2)) < 1e-13 * nb * nc
    assert np.all(d2[1:] == 0.0) and np.all(e2[1:] == 0.0)
    assert abs(math.hypot(d2[0], e2[0]) - nb * nc) < 1e-13 * nb * nc  # sigma_1 = ||b|| ||c||
    q1 = Q2[:, 0] * np.sign(Q2[:, 0] @ b)
    np.testing.assert_allclose(q1, b / nb, atol=1e-14)


def test_already_bidiagonal_needs_no_rotation():
    """u in span(e1), v in span(e1, e2): Bd + u v^T is bidiagonal already."""
    n = 10
    d = np.arange(1.0, n + 1); e = np.full(n - 1, 0.5)
    b = np.zeros(n); b[0] = 2.0
    c = np.zeros(n); c[0] = 3.0; c[1] = -1.0
    Q2, d2, e2, P2, cnt = O.update(np.eye(n), d, e, np.eye(n), b, c)
    assert cnt["total"] == 0
    want_d = d.copy(); want_d[0] += 6.0
    want_e = e.copy(); want_e[0] += -2.0
    assert np.array_equal(d2, want_d) and np.array_equal(e2, want_e)
    assert np.array_equal(Q2, np.eye(n)) and np.array_equal(P2, np.eye(n))


def test_zero_b_is_a_no_op():
    Q, d, e, P = I.factorization(20, 12, config=0, which=5)
    Q2, d2, e2, P2, cnt = O.update(Q, d, e, P, np.zeros(20), np.ones(12))
    assert cnt["total"] == 0
    assert np.array_equal(d2, d) and np.array_equal(e2, e)
    assert np.array_equal(Q2, Q) and np.array_equal(P2, P)


def test_zero_c_keeps_the_factorization():
    """A+ = A and P+(:,1) = P(:,1).  The leading entries are well-conditioned
    functions of A (alpha_1 = ||A p_1||, Eq. recp with k = 1) and must stay,
    singular values must stay, and Q+ Bd+ P+^T must still reproduce A.  The
    trailing entries of Bd+ need not match Bd: for this distribution they are
    ill-conditioned functions of A (Krylov basis from p_1 nearly dependent)."""
    Q, d, e, P = I.factorization(40, 40, config=0, which=8)
    A = dense_A(Q, d, e, P)
    b = np.random.default_rng(2).standard_normal(40)
    Q2, d2, e2, P2, cnt = O.update(Q, d, e, P, b, np.zeros(40))
    assert cnt["total"] > 0
    assert abs(abs(d2[0]) - d[0]) < 1e-13 * d[0]
    assert abs(abs(e2[0]) - abs(e[0])) < 1e-13 * d[0]
    assert rel_resid(A, Q2, d2, e2, P2) < 1e-14
    np.testing.assert_allclose(np.linalg.svd(O.bidiag_dense(d2, e2), compute_uv=False),
                               np.linalg.svd(O.bidiag_dense(d, e), compute_uv=False), rtol=1e-13)


def test_spike_with_u_already_inside_the_core():
    """m > n with Q^T b having no component below row n+1: the spike is empty."""
    m, n = 30, 12
    d = np.linspace(1, 2, n); e = np.full(n - 1, 0.3)
    b = np.zeros(m); b[:n + 1] = np.random.default_rng(4).standard_normal(n + 1)
    c = np.random.default_rng(5).standard_normal(n)
    Aplus = O.bidiag_dense(d, e, m) + np.outer(b, c)
    Q2, d2, e2, P2, cnt = O.update(np.eye(m), d, e, np.eye(n), b, c)
    assert cnt["left"]["spike"] == 0
    assert rel_resid(Aplus, Q2, d2, e2, P2) < 1e-14


def test_rank_r_equals_sequential_rank_1():
    m, n, r = 60, 45, 4
    Q, d, e, P = I.factorization(m, n, config=0, which=12)
    B, C = I.dense_update(m, n, h=2, config=0, r=r)
    Qa, da, ea, Pa, _ = O.update(Q, d, e, P, B, C)
    Qb, db, eb, Pb = Q, d, e, P
    for k in range(r):
        Qb, db, eb, Pb, _ = O.update(Qb, db, eb, Pb, B[:, k], C[:, k])
    scale = np.linalg.norm(np.concatenate([da, ea]))
    np.testing.assert_allclose(da, db, atol=1e-13 * scale)
    np.testing.assert_allclose(ea, eb, atol=1e-13 * scale)
    np.testing.assert_allclose(Qa, Qb, atol=1e-13)
    np.testing.assert_allclose(Pa, Pb, atol=1e-13)


def test_rotation_count_is_quadratic():
    """About 1.5 n^2 rotations per rank-1 column (Sec. 3.4: O(n) bulges of O(n) rotations)."""
    for n in (64, 256):
        Q, d, e, P = I.factorization(n, n, config=0, which=n)
        B, C = I.dense_update(n, n, h=1, config=0)
        _, _, _, _, cnt = O.update(Q, d, e, P, B, C)
        assert 1.4 * n * n < cnt["total"] < 1.6 * n * n


def test_generate_and_apply_rows_match_update():
    """The sampled-row path used at full size equals the full update, bitwise."""
    m, n = 70, 50
    Q, d, e, P = I.factorization(m, n, config=0, which=77)
    B, C = I.dense_update(m, n, h=4, config=0, r=2)
    Qf, df, ef, Pf, _ = O.update(Q, d, e, P, B, C)
    U, V = O.project(Q, P, B, C)
    d2, e2, L, R, _ = O.generate(m, n, d, e, U, V)
    assert np.array_equal(d2, df) and np.array_equal(e2, ef)
    rows = np.array([0, 5, 33, 69])
    Qs = O.apply_rows(Q, rows, L)
    assert np.array_equal(Qs[rows], Qf[rows])
    Ps = O.apply_rows(P, np.array([1, 49]), R)
    assert np.array_equal(Ps[[1, 49]], Pf[[1, 49]])


# --------------------------------------------------------------------------
# the pins catch planted mistakes (mistakes are planted in inputs to the
# oracle's own building blocks, on the CPU)
# --------------------------------------------------------------------------
def test_pins_detect_a_transposed_projection():
    m, n = 40, 40
    Q, d, e, P = I.factorization(m, n, config=0, which=21)
    B, C = I.dense_update(m, n, h=9, config=0)
    Aplus = dense_A(Q, d, e, P) + B @ C.T
    U, V = O.project(Q.T, P, B, C)  # planted: Q instead of Q^T
    d2, e2, L, R, _ = O.generate(m, n, d, e, U, V)
    Q2 = O.apply_rows(Q, np.arange(m), L)
    P2 = O.apply_rows(P, np.arange(n), R)
    assert rel_resid(Aplus, Q2, d2, e2, P2) > 1e-3


def test_pins_detect_a_wrong_rotation_sign():
    m, n = 30, 30
    Q, d, e, P = I.factorization(m, n, config=0, which=22)
    B, C = I.dense_update(m, n, h=10, config=0)
    Aplus = dense_A(Q, d, e, P) + B @ C.T
    U, V = O.project(Q, P, B, C)
    d2, e2, L, R, _ = O.generate(m, n, d, e, U, V)
    R.s = -R.s  # planted: H^T applied to P instead of H
    P2 = O.apply_rows(P, np.arange(n), R)
    Q2 = O.apply_rows(Q, np.arange(m), L)
    assert rel_resid(Aplus, Q2, d2, e2, P2) > 1e-3


# ---------------------------------------------------------------------------
# truncated bidiagonal approximation (Sec. 2, Eqs. trBD, errtrBD)
# ---------------------------------------------------------------------------
def _random_bd(m, n, seed):
    g = np.random.default_rng(seed)
    Q = I.householder_orthogonal(m, g)
    P = I.householder_orthogonal(n, g)
    d = g.uniform(-3, 3, n)
    e = g.standard_normal(max(n - 1, 0))
    return Q, d, e, P


@pytest.mark.parametrize("m,n,r", [(12, 9, 0), (12, 9, 1), (12, 9, 4), (12, 9, 9), (30, 30, 11), (7, 1, 1)])
def test_truncated_bd_error_identity(m, n, r):
    """||A - L R^T||_F^2, formed densely, equals the sum of the dropped
    alpha_i^2 + beta_{i-1}^2 (Eq. errtrBD)."""
    Q, d, e, P = _random_bd(m, n, 100 + m + n + r)
    A = Q @ O.bidiag_dense(d, e, m) @ P.T
    L, R, idx, err2 = O.truncated_bd(Q, d, e, P, r)
    assert L.shape == (m, r) and R.shape == (n, r) and len(idx) == r
    assert np.all(np.diff(idx) > 0) and (r == 0 or (idx[0] >= 1 and idx[-1] <= n))
    direct = np.linalg.norm(A - L @ R.T, "fro") ** 2
    assert abs(direct - err2) <= 1e-12 * max(1.0, np.linalg.norm(A, "fro") ** 2)
    if r == n:
        assert err2 == 0.0 and np.allclose(L @ R.T, A, rtol=0, atol=1e-13 * np.abs(A).max())


def test_truncated_bd_keeps_the_largest_pairs():
    """The kept set maximizes the captured energy: no swap of a kept and a
    dropped index lowers the error (brute force over all r-subsets)."""
    import itertools
    Q, d, e, P = _random_bd(8, 6, 7)
    w = d ** 2 + np.concatenate([[0.0], e ** 2])
    _, _, idx, err2 = O.truncated_bd(Q, d, e, P, 3)
    best = min(sum(w) - sum(w[list(c)]) for c in itertools.combinations(range(6), 3))
    assert abs(err2 - best) <= 1e-14 * sum(w)


def test_truncated_bd_of_a_diagonal_is_the_truncated_svd():
    """beta = 0: the bidiagonal decomposition is an SVD (up to signs), so the
    truncation keeps the r largest |alpha| and its error is the sum of the
    other sigma^2 (the Eckart-Young error of the truncated SVD)."""
    g = np.random.default_rng(3)
    m, n, r = 10, 7, 3
    Q = I.householder_orthogonal(m, g)
    P = I.householder_orthogonal(n, g)
    d = g.uniform(-5, 5, n)
    e = np.zeros(n - 1)
    A = Q @ O.bidiag_dense(d, e, m) @ P.T
    L, R, idx, err2 = O.truncated_bd(Q, d, e, P, r)
    sv = np.linalg.svd(A, compute_uv=False)
    assert abs(err2 - np.sum(sv[r:] ** 2)) <= 1e-12 * np.sum(sv ** 2)
    U, S, Vt = np.linalg.svd(A)
    Ar = (U[:, :r] * S[:r]) @ Vt[:r]
    assert np.linalg.norm(L @ R.T - Ar) <= 1e-12 * np.linalg.norm(A)
    assert set(idx - 1) == set(np.argsort(-np.abs(d))[:r])


# ---------------------------------------------------------------------------
# singular values of the bidiagonal
# ---------------------------------------------------------------------------
def test_bidiagonal_singular_values_2x2_closed_form():
    """[[a, b], [0, c]]: sigma_1 sigma_2 = |a c| and
    sigma_1^2 + sigma_2^2 = a^2 + b^2 + c^2."""
    for a, b, c in ((3.0, 4.0, 5.0), (-1.0, 0.5, 2.0), (1e-3, 7.0, -2.0), (2.0, 0.0, 3.0)):
        s1, s2 = O.singular_values([a, c], [b])
        assert abs(s1 * s2 - abs(a * c)) <= 1e-14 * s1 * s1
        assert abs(s1 * s1 + s2 * s2 - (a * a + b * b + c * c)) <= 1e-14 * (a * a + b * b + c * c)


def test_bidiagonal_singular_values_match_jacobi_and_the_full_matrix():
    """Against the oracle's own one-sided Jacobi (independent code) on small
    random bidiagonals, and against the singular values of A = Q Bd P^T."""
    g = np.random.default_rng(11)
    for n in (1, 3, 8, 15):
        d = g.standard_normal(n) * 3
        e = g.standard_normal(n - 1)
        sv = O.singular_values(d, e)
        assert np.allclose(sv, O.jacobi_sv(O.bidiag_dense(d, e)), rtol=0, atol=1e-13 * sv[0])
        Q = I.householder_orthogonal(n + 4, g)
        P = I.householder_orthogonal(n, g)
        A = Q @ O.bidiag_dense(d, e, n + 4) @ P.T
        assert np.allclose(sv, np.linalg.svd(A, compute_uv=False), rtol=0, atol=1e-12 * sv[0])
