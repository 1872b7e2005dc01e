"""Pins of the BHU oracle (Sec. 3.3, Algorithm 1, Theorem 1) against facts that do
not come from it: a hand-derived example, the Givens oracle (a different method
that also keeps the first right vector, so the bidiagonal agrees up to signs),
LAPACK singular values, exact reconstruction and orthogonality, Theorem 1's
factored form, a rank-1 closed form and the no-update case."""
import json
import os

import numpy as np
import pytest

import oracle as O
from oracle import bhu as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SHAPES = [(1, 1), (3, 1), (2, 2), (3, 2), (3, 3), (4, 3), (6, 6), (9, 4), (20, 20), (33, 17), (40, 40)]


def _case(m, n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n), rng.standard_normal(max(n - 1, 0)), rng.standard_normal(m),
            rng.standard_normal(n))


def test_golden_2x2():
    g = json.load(open(os.path.join(GOLDEN, "bhu_2x2_worked_example.json")))
    r = H.bhu(g["d"], g["e"], g["u"], g["v"], g["m"])
    assert np.allclose(r["alpha"], g["alpha"], rtol=0, atol=1e-15)
    assert np.allclose(r["beta"], g["beta"], rtol=0, atol=1e-15)
    assert np.allclose(r["Y"][:, 0], g["y1"], rtol=0, atol=1e-15)
    assert r["W"].shape[1] == 0


@pytest.mark.parametrize("m,n", SHAPES)
def test_reconstruction_and_orthogonality(m, n):
    d, e, u, v = _case(m, n, 100 * m + n)
    r = H.bhu(d, e, u, v, m)
    Qk, Pk = H.factors(r["Y"], r["W"], m, n)
    A0 = H.bidiag_dense(d, e, m) + np.outer(u, v)
    Bp = H.bidiag_dense(r["alpha"], r["beta"], m)
    scale = np.linalg.norm(A0)
    assert np.abs(Qk @ Bp @ Pk.T - A0).max() <= 1e-14 * scale * max(m, 4)
    assert np.abs(Qk.T @ Qk - np.eye(m)).max() <= 1e-14 * max(m, 4)
    assert np.abs(Pk.T @ Pk - np.eye(n)).max() <= 1e-14 * max(n, 4)
    # no right reflector touches column 1 (exactly: every w has a zero first entry)
    assert np.array_equal(Pk[:, 0], np.eye(n)[:, 0])
    # everything off the two diagonals has been eliminated
    assert np.abs(r["A"] - Bp).max() <= 1e-14 * scale * max(m, 4)
    # reflector vectors: unit norm, zeros above their first row (Eq. YW)
    for j in range(r["Y"].shape[1]):
        assert abs(np.linalg.norm(r["Y"][:, j]) - 1.0) < 1e-14 and not np.any(r["Y"][:j, j])
    for j in range(r["W"].shape[1]):
        assert abs(np.linalg.norm(r["W"][:, j]) - 1.0) < 1e-14 and not np.any(r["W"][:j + 1, j])


@pytest.mark.parametrize("m,n", [s for s in SHAPES if s[1] >= 2])
def test_matches_givens_oracle_up_to_signs(m, n):
    """Both keep P(:,1) fixed, so by the implicit-Q theorem the new bidiagonal is
    unique up to signs when unreduced (the Givens oracle is pinned on its own)."""
    d, e, u, v = _case(m, n, 7 * m + n)
    r = H.bhu(d, e, u, v, m)
    dg, eg = O.generate(m, n, d, e, u.reshape(m, 1), v.reshape(n, 1))[:2]
    scale = np.linalg.norm(H.bidiag_dense(d, e, m) + np.outer(u, v))
    assert np.abs(np.abs(r["alpha"]) - np.abs(dg)).max() <= 1e-12 * scale
    assert np.abs(np.abs(r["beta"]) - np.abs(eg)).max() <= 1e-12 * scale


@pytest.mark.parametrize("m,n", SHAPES)
def test_singular_values_lapack(m, n):
    d, e, u, v = _case(m, n, 3 * m + n)
    r = H.bhu(d, e, u, v, m)
    s0 = np.linalg.svd(H.bidiag_dense(d, e, m) + np.outer(u, v), compute_uv=False)
    s1 = np.linalg.svd(H.bidiag_dense(r["alpha"], r["beta"], m), compute_uv=False)
    assert np.abs(s0 - s1).max() <= 1e-13 * s0[0]


@pytest.mark.parametrize("m,n,k", [(6, 6, 1), (6, 6, 3), (9, 5, 2), (12, 8, 5), (20, 20, 10)])
def test_theorem1_factored_form(m, n, k):
    """A_kk after k left and k right reflectors equals B - U M^{-1} V^T (Eq. comp)."""
    d, e, u, v = _case(m, n, 11 * m + k)
    r = H.bhu(d, e, u, v, m, steps=k)
    assert r["Y"].shape[1] == k and r["W"].shape[1] == k
    F = H.theorem1(d, e, u, v, m, r["Y"], r["W"])
    assert np.abs(F - r["A"]).max() <= 1e-13 * np.linalg.norm(r["A"])


def test_partial_factorization_is_the_leading_part():
    m, n = 15, 12
    d, e, u, v = _case(m, n, 5)
    full = H.bhu(d, e, u, v, m)
    for t in (1, 4, 9):
        p = H.bhu(d, e, u, v, m, steps=t)
        assert np.array_equal(p["alpha"], full["alpha"][:t])
        assert np.array_equal(p["beta"], full["beta"][:t])
        # rows and columns 1..t of A_tt are already bidiagonal
        A = p["A"]
        assert np.abs(A[t:, :t]).max() <= 1e-13 and np.abs(A[:t, :]).max() > 0
        assert np.abs(np.triu(A[:t, :], 2)).max() <= 1e-13


@pytest.mark.parametrize("m,n", [(5, 5), (8, 5), (30, 30)])
def test_rank1_closed_form(m, n):
    """B = 0: A = u v^T has one nonzero singular value ||u|| ||v||, which the
    first column and row carry: alpha_1^2 + beta_1^2 = ||u||^2 ||v||^2."""
    rng = np.random.default_rng(m + n)
    u = rng.standard_normal(m); v = rng.standard_normal(n)
    r = H.bhu(np.zeros(n), np.zeros(n - 1), u, v, m)
    nu = np.linalg.norm(u) * np.linalg.norm(v)
    assert abs(np.hypot(r["alpha"][0], r["beta"][0]) - nu) <= 1e-14 * nu
    assert abs(abs(r["alpha"][0]) - np.linalg.norm(u) * abs(v[0])) <= 1e-14 * nu
    assert np.abs(r["alpha"][1:]).max() <= 1e-14 * nu and np.abs(r["beta"][1:]).max() <= 1e-14 * nu


@pytest.mark.parametrize("m,n", [(5, 5), (7, 4)])
def test_no_update_keeps_magnitudes(m, n):
    """u = 0: every reflector acts on a multiple of e_1 and only flips signs."""
    d, e, _, v = _case(m, n, 9)
    r = H.bhu(d, e, np.zeros(m), v, m)
    assert np.array_equal(np.abs(r["alpha"]), np.abs(d))
    assert np.array_equal(np.abs(r["beta"]), np.abs(e))


def test_full_update_matches_givens_update():
    rng = np.random.default_rng(21)
    m, n, rk = 14, 10, 2
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    P, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d = rng.standard_normal(n); e = rng.standard_normal(n - 1)
    Bm = rng.standard_normal((m, rk)); Cm = rng.standard_normal((n, rk))
    Qh, dh, eh, Ph = H.update(Q, d, e, P, Bm, Cm)
    Qg, dg, eg, Pg, _ = O.update(Q, d, e, P, Bm, Cm)
    A1 = Q @ H.bidiag_dense(d, e, m) @ P.T + Bm @ Cm.T
    assert np.abs(Qh @ H.bidiag_dense(dh, eh, m) @ Ph.T - A1).max() <= 1e-13 * np.linalg.norm(A1)
    assert np.abs(np.abs(dh) - np.abs(dg)).max() <= 1e-12 * np.linalg.norm(A1)
    assert np.abs(np.abs(eh) - np.abs(eg)).max() <= 1e-12 * np.linalg.norm(A1)
    assert np.array_equal(Ph[:, 0], P[:, 0]) or np.abs(Ph[:, 0] - P[:, 0]).max() <= 1e-15


@pytest.mark.parametrize("m,n,rk", [(14, 10, 2), (20, 20, 3), (33, 17, 5), (12, 12, 12)])
def test_direct_rank_r_matches_givens_update(m, n, rk):
    """One BHU sweep on B + U V^T against the Givens oracle's r rank-1 steps:
    both keep P's first column, so the bidiagonals agree up to signs; the
    factorization reconstructs A + B C^T."""
    rng = np.random.default_rng(m * 31 + rk)
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    P, _ = np.linalg.qr(rng.standard_normal((n, n)))
    d = rng.standard_normal(n); e = rng.standard_normal(n - 1)
    Bm = rng.standard_normal((m, rk)); Cm = rng.standard_normal((n, rk))
    Qh, dh, eh, Ph = H.update_direct(Q, d, e, P, Bm, Cm)
    Qg, dg, eg, Pg, _ = O.update(Q, d, e, P, Bm, Cm)
    A1 = Q @ H.bidiag_dense(d, e, m) @ P.T + Bm @ Cm.T
    scale = np.linalg.norm(A1)
    assert np.abs(Qh @ H.bidiag_dense(dh, eh, m) @ Ph.T - A1).max() <= 1e-13 * scale
    assert np.abs(np.abs(dh) - np.abs(dg)).max() <= 1e-12 * scale
    assert np.abs(np.abs(eh) - np.abs(eg)).max() <= 1e-12 * scale
    assert np.array_equal(Ph[:, 0], P[:, 0]) or np.abs(Ph[:, 0] - P[:, 0]).max() <= 1e-15
    s0 = np.linalg.svd(A1, compute_uv=False)
    assert np.abs(s0 - np.linalg.svd(H.bidiag_dense(dh, eh, m), compute_uv=False)).max() <= 1e-13 * s0[0]


@pytest.mark.parametrize("m,n,rk", [(30, 30, 1), (30, 30, 3), (40, 25, 4)])
def test_rank_r_terminates(m, n, rk):
    """B = 0: A = U V^T has rank r, and the Householder bidiagonalization with
    P's first column kept ends after r + 1 columns (its Krylov space from
    p_1 = e_1 has dimension <= r + 1): every later alpha, beta vanishes, and
    alpha, beta carry all of ||U V^T||_F^2."""
    rng = np.random.default_rng(m + 10 * rk)
    U = rng.standard_normal((m, rk)); V = rng.standard_normal((n, rk))
    r = H.bhu(np.zeros(n), np.zeros(n - 1), U, V, m)
    nf = np.linalg.norm(U @ V.T)
    assert np.abs(r["alpha"][rk + 1:]).max() <= 1e-13 * nf
    assert np.abs(r["beta"][rk + 1:]).max() <= 1e-13 * nf
    assert abs(np.sum(r["alpha"] ** 2) + np.sum(r["beta"] ** 2) - nf ** 2) <= 1e-12 * nf ** 2


# ---- the symmetric (tridiagonal) variant

def _tri_case(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n), rng.standard_normal(max(n - 1, 0)), rng.standard_normal(n), float(rng.choice([-1.5, 0.7, 2.0]))


def test_tri_golden_3x3():
    g = json.load(open(os.path.join(GOLDEN, "tri_3x3_worked_example.json")))
    r = H.tri(g["a"], g["b"], g["u"], g["rho"])
    assert np.allclose(r["alpha"], g["alpha"], rtol=0, atol=1e-14)
    assert np.allclose(r["beta"], g["beta"], rtol=0, atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 9, 30, 64])
def test_tri_reconstruction_eigenvalues_first_column(n):
    a, b, u, rho = _tri_case(n, 40 + n)
    r = H.tri(a, b, u, rho)
    M = H.tridiag_dense(a, b) + rho * np.outer(u, u)
    Qk, _ = H.factors(r["Y"], np.zeros((1, 0)), n, 1)
    Tp = H.tridiag_dense(r["alpha"], r["beta"])
    scale = np.linalg.norm(M)
    assert np.abs(Qk @ Tp @ Qk.T - M).max() <= 1e-14 * scale * max(n, 4)
    assert np.array_equal(Qk[:, 0], np.eye(n)[:, 0])
    assert np.abs(r["A"] - Tp).max() <= 1e-14 * scale * max(n, 4)
    assert np.abs(np.linalg.eigvalsh(M) - np.linalg.eigvalsh(Tp)).max() <= 1e-13 * scale


@pytest.mark.parametrize("n", [4, 9, 30, 64])
def test_tri_matches_lapack_hessenberg_up_to_signs(n):
    """LAPACK's Householder reduction to Hessenberg form also keeps e_1, so for a
    symmetric matrix its tridiagonal equals this one up to signs."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    a, b, u, rho = _tri_case(n, 70 + n)
    M = H.tridiag_dense(a, b) + rho * np.outer(u, u)
    Hs = scipy_linalg.hessenberg(M)
    r = H.tri(a, b, u, rho)
    scale = np.linalg.norm(M)
    assert np.abs(np.abs(np.diag(Hs)) - np.abs(r["alpha"])).max() <= 1e-12 * scale
    assert np.abs(np.abs(np.diag(Hs, -1)) - np.abs(r["beta"])).max() <= 1e-12 * scale


def test_tri_no_update_and_rank1_closed_forms():
    a, b, u, _ = _tri_case(12, 3)
    r = H.tri(a, b, u, 0.0)
    assert np.array_equal(r["alpha"], a) and np.array_equal(np.abs(r["beta"]), np.abs(b))
    # T = 0: rho u u^T has the one nonzero eigenvalue rho ||u||^2, carried by the
    # leading 2 x 2 block
    r = H.tri(np.zeros(12), np.zeros(11), u, 1.5)
    nu = 1.5 * np.dot(u, u)
    assert abs(r["alpha"][0] + r["alpha"][1] - nu) <= 1e-14 * nu
    assert abs(r["alpha"][0] * r["alpha"][1] - r["beta"][0] ** 2) <= 1e-13 * nu ** 2
    assert np.abs(r["alpha"][2:]).max() <= 1e-14 * nu and np.abs(r["beta"][1:]).max() <= 1e-14 * nu


def test_tri_update_reconstructs():
    rng = np.random.default_rng(8)
    n = 20
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    a, b, c, rho = _tri_case(n, 9)
    Qn, al, be = H.tri_update(Q, a, b, rho, c)
    A1 = Q @ H.tridiag_dense(a, b) @ Q.T + rho * np.outer(c, c)
    assert np.abs(Qn @ H.tridiag_dense(al, be) @ Qn.T - A1).max() <= 1e-13 * np.linalg.norm(A1)
    assert np.array_equal(Qn[:, 0], Q[:, 0]) or np.abs(Qn[:, 0] - Q[:, 0]).max() <= 1e-15


# ---- the pins catch plausible mistakes planted in copies of the oracle

def _mutant(src_old, src_new):
    """A copy of oracle.bhu with one line changed (compiled from its source)."""
    import inspect
    import types
    src = inspect.getsource(H)
    assert src.count(src_old) == 1, src_old
    mod = types.ModuleType("bhu_mutant")
    exec(compile(src.replace(src_old, src_new), "bhu_mutant", "exec"), mod.__dict__)
    return mod


def _passes_pins(M):
    """The golden examples, reconstruction with the factors, agreement with the
    Givens oracle up to signs and with LAPACK's Hessenberg reduction."""
    try:
        g = json.load(open(os.path.join(GOLDEN, "bhu_2x2_worked_example.json")))
        r = M.bhu(g["d"], g["e"], g["u"], g["v"], g["m"])
        if not (np.allclose(r["alpha"], g["alpha"], atol=1e-14) and np.allclose(r["beta"], g["beta"], atol=1e-14)):
            return False
        g = json.load(open(os.path.join(GOLDEN, "tri_3x3_worked_example.json")))
        r = M.tri(g["a"], g["b"], g["u"], g["rho"])
        if not (np.allclose(r["alpha"], g["alpha"], atol=1e-14) and np.allclose(r["beta"], g["beta"], atol=1e-14)):
            return False
        for (m, n) in ((9, 6), (7, 7)):
            d, e, u, v = _case(m, n, m + n)
            r = M.bhu(d, e, u, v, m)
            Qk, Pk = M.factors(r["Y"], r["W"], m, n)
            A0 = M.bidiag_dense(d, e, m) + np.outer(u, v)
            if np.abs(Qk @ M.bidiag_dense(r["alpha"], r["beta"], m) @ Pk.T - A0).max() > 1e-12:
                return False
            dg, eg = O.generate(m, n, d, e, u.reshape(m, 1), v.reshape(n, 1))[:2]
            if np.abs(np.abs(r["alpha"]) - np.abs(dg)).max() > 1e-10 or np.abs(np.abs(r["beta"]) - np.abs(eg)).max() > 1e-10:
                return False
        a, b, u, rho = _tri_case(8, 2)
        r = M.tri(a, b, u, rho)
        Qk, _ = M.factors(r["Y"], np.zeros((1, 0)), 8, 1)
        Mx = M.tridiag_dense(a, b) + rho * np.outer(u, u)
        return np.abs(Qk @ M.tridiag_dense(r["alpha"], r["beta"]) @ Qk.T - Mx).max() <= 1e-12
    except (AssertionError, ValueError, IndexError, np.linalg.LinAlgError):
        return False


def test_pins_pass_on_the_oracle_itself():
    assert _passes_pins(H)


@pytest.mark.parametrize("old,new", [
    ("    y[0] += s * sigma\n", "    y[0] -= s * sigma\n"),                                   # the other reflector sign
    ("            beta[k], w = house(A[k, k + 1:])\n", "            beta[k], w = house(A[min(k + 1, m - 1), k + 1:])\n"),  # row k+1
    ("            A[k:, :] -= 2.0 * np.outer(y, y @ A[k:, :])\n", "            A[k:, :] -= 1.0 * np.outer(y, y @ A[k:, :])\n"),  # a dropped 2
    ("            A[:, k + 1:] -= 2.0 * np.outer(A[:, k + 1:] @ w, w)\n", "            A[:, k + 1:] -= 2.0 * np.outer(A[:, k + 1:] @ w, w.T)[:, ::-1]\n"),  # a reversed vector
    ("            A[:, k + 1:] -= 2.0 * np.outer(A[:, k + 1:] @ y, y)\n", "            pass\n"),   # one-sided symmetric step
    ("    A = tridiag_dense(a, b) + rho * np.outer(u, u)\n", "    A = tridiag_dense(a, b) - rho * np.outer(u, u)\n"),  # wrong sign of rho
])
def test_pins_catch_a_planted_mistake(old, new):
    assert not _passes_pins(_mutant(old, new))
