"""BHU on the GPU (Sec. 3.3, Algorithm 1, Theorem 1) against the BHU oracle,
through the C ABI (bdu_bhu_factor, bdu_update_bhu).

Tolerances.  Both sides are FP64 Householder processes that differ only in the
order of their sums (the GPU forms each column and row from the factored form
of Theorem 1, the oracle transforms the dense matrix).  A Householder
bidiagonalization is backward stable with an error of O(n u ||A||_F), u the
unit roundoff (Higham, Accuracy and Stability of Numerical Algorithms, Ch. 19),
and on these random inputs the entries of the two results move apart by about
that much: TOL(n) = 1e-14 n ||A||_F (~90 n u) for the bidiagonal, measured
2-7x below it from n = 256 to 4096.  A reflector vector is its source column
(or row) scaled to unit norm, so its error is that column's over the column's
norm |alpha_j| (|beta_j| for w_{j+1}): late columns are small and their vectors
correspondingly less accurate (conditioning, not a defect).  The factors Q, P
inherit that; they are compared within 1e-12 n.  Quantities that are well
conditioned whatever the input are held to the plain FP64 level: singular
values within 1e-12 sigma_1 of LAPACK's on the dense A (Weyl), reconstruction
within 1e-12 ||A||_F."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import bhu as H  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (3, 1), (2, 2), (3, 3), (5, 3), (64, 64), (257, 256), (300, 200), (530, 529), (1030, 700)]


def _bdu():
    from paper_2509_02840_gb300 import bdu
    bdu.load()
    return bdu


def tol(n, scale):
    return 1e-14 * max(n, 1) * scale


def _vec_close(G, O, norms, scale):
    """Column j of G within TOL(n) / |norms[j]| of the oracle's."""
    for j in range(O.shape[1]):
        tol_j = tol(O.shape[0], scale) / max(abs(norms[j]), 1e-300)
        assert np.abs(G[:, j] - O[:, j]).max() <= tol_j, (j, np.abs(G[:, j] - O[:, j]).max(), tol_j)


def _case(m, n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n), rng.standard_normal(max(n - 1, 0)), rng.standard_normal(m),
            rng.standard_normal(n))


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.float64))).cuda()


def _ptr(t):
    return t.data_ptr() if t is not None and t.numel() else 0


def run_factor(m, n, d, e, u, v, steps=None):
    bdu = _bdu()
    steps = n if steps is None else steps
    U = np.asarray(u, dtype=np.float64).reshape(m, -1)
    V = np.asarray(v, dtype=np.float64).reshape(n, -1)
    rk = U.shape[1]
    kl, kr, wb = bdu.bhu_sizes(m, n, steps)
    dd, ee = _dev(d), _dev(e if n > 1 else [0.0])
    uu, vv = _dev(U.T.reshape(-1)), _dev(V.T.reshape(-1))  # column-major
    alpha = torch.zeros(max(steps, 1), dtype=torch.float64, device="cuda")
    beta = torch.zeros(max(min(steps, n - 1), 1), dtype=torch.float64, device="cuda")
    Y = torch.zeros(max(m * kl, 1), dtype=torch.float64, device="cuda")
    W = torch.zeros(max(n * kr, 1), dtype=torch.float64, device="cuda")
    SL = torch.zeros(max(kl * kl, 1), dtype=torch.float64, device="cuda")
    SR = torch.zeros(max(kr * kr, 1), dtype=torch.float64, device="cuda")
    ws = torch.zeros((wb + 7) // 8, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    bdu.bhu_factor(m, n, steps, _ptr(dd), _ptr(ee) if n > 1 else 0, _ptr(uu), _ptr(vv), _ptr(alpha),
                   _ptr(beta) if n > 1 else 0, _ptr(Y) if kl else 0, _ptr(W) if kr else 0, _ptr(SL) if kl else 0,
                   _ptr(SR) if kr else 0, _ptr(ws), s, r=rk)
    torch.cuda.synchronize()
    return {"alpha": alpha.cpu().numpy()[:steps], "beta": beta.cpu().numpy()[:min(steps, n - 1)],
            "Y": Y.cpu().numpy()[:m * kl].reshape(kl, m).T, "W": W.cpu().numpy()[:n * kr].reshape(kr, n).T,
            "SL": SL.cpu().numpy()[:kl * kl].reshape(kl, kl).T, "SR": SR.cpu().numpy()[:kr * kr].reshape(kr, kr).T}


@pytest.mark.parametrize("m,n", SHAPES)
def test_factor_matches_oracle(m, n):
    d, e, u, v = _case(m, n, 31 * m + n)
    g = run_factor(m, n, d, e, u, v)
    o = H.bhu(d, e, u, v, m)
    scale = np.linalg.norm(H.bidiag_dense(d, e, m) + np.outer(u, v))
    assert np.abs(g["alpha"] - o["alpha"]).max() <= tol(n, scale)
    if n > 1:
        assert np.abs(g["beta"] - o["beta"]).max() <= tol(n, scale)
    assert g["Y"].shape == o["Y"].shape and g["W"].shape == o["W"].shape
    if o["Y"].size:
        _vec_close(g["Y"], o["Y"], o["alpha"], scale)
        # the structural zeros are exact
        for j in range(g["Y"].shape[1]):
            assert not np.any(g["Y"][:j, j])
    if o["W"].size:
        _vec_close(g["W"], o["W"], o["beta"], scale)
        for j in range(g["W"].shape[1]):
            assert not np.any(g["W"][:j + 1, j])


@pytest.mark.parametrize("m,n,rk", [(64, 64, 2), (300, 200, 3), (530, 529, 8), (1030, 700, 5)])
def test_factor_rank_r_matches_oracle(m, n, rk):
    """Direct rank-r absorption: one sweep of Algorithm 1 on B + U V^T."""
    rng = np.random.default_rng(m + 7 * rk)
    d, e = rng.standard_normal(n), rng.standard_normal(n - 1)
    U, V = rng.standard_normal((m, rk)), rng.standard_normal((n, rk))
    g = run_factor(m, n, d, e, U, V)
    o = H.bhu(d, e, U, V, m)
    scale = np.linalg.norm(H.bidiag_dense(d, e, m) + U @ V.T)
    assert np.abs(g["alpha"] - o["alpha"]).max() <= tol(n, scale)
    assert np.abs(g["beta"] - o["beta"]).max() <= tol(n, scale)
    _vec_close(g["Y"], o["Y"], o["alpha"], scale)
    _vec_close(g["W"], o["W"], o["beta"], scale)


@pytest.mark.parametrize("m,n", [(5, 3), (64, 64), (300, 200), (530, 529)])
def test_compact_form_is_the_reflector_product(m, n):
    """Q_k = I - Y SL Y^T, P_k = I - W SR W^T with SL = 2 T^{-1}, SR = 2 R^{-1}
    (Eqs. QP, TR): against the oracle's plain products of the reflectors."""
    d, e, u, v = _case(m, n, 17 * m + n)
    g = run_factor(m, n, d, e, u, v)
    Qo, Po = H.factors(g["Y"], g["W"], m, n)
    Qg = np.eye(m) - g["Y"] @ g["SL"] @ g["Y"].T
    Pg = np.eye(n) - g["W"] @ g["SR"] @ g["W"].T
    assert np.abs(Qg - Qo).max() <= 1e-12 * max(m, 8)
    assert np.abs(Pg - Po).max() <= 1e-12 * max(n, 8)
    k = g["Y"].shape[1]
    T = np.eye(k) + np.triu(2.0 * (g["Y"].T @ g["Y"]), 1)
    assert np.abs(g["SL"] - 2.0 * np.linalg.inv(T)).max() <= 1e-10
    assert not np.any(np.tril(g["SL"], -1)) and not np.any(np.tril(g["SR"], -1))
    # the bidiagonal it defines reproduces A
    A0 = H.bidiag_dense(d, e, m) + np.outer(u, v)
    Bp = H.bidiag_dense(g["alpha"], g["beta"], m)
    assert np.abs(Qg @ Bp @ Pg.T - A0).max() <= 1e-12 * np.linalg.norm(A0)


@pytest.mark.parametrize("m,n,t", [(12, 9, 1), (12, 9, 4), (300, 200, 57), (530, 529, 300), (257, 256, 256)])
def test_partial_factorization(m, n, t):
    d, e, u, v = _case(m, n, m + 3 * t)
    g = run_factor(m, n, d, e, u, v, steps=t)
    o = H.bhu(d, e, u, v, m, steps=t)
    scale = np.linalg.norm(H.bidiag_dense(d, e, m) + np.outer(u, v))
    assert np.abs(g["alpha"] - o["alpha"]).max() <= tol(n, scale)
    assert np.abs(g["beta"] - o["beta"]).max() <= tol(n, scale)
    _vec_close(g["Y"], o["Y"], o["alpha"], scale)
    _vec_close(g["W"], o["W"], o["beta"], scale)


@pytest.mark.parametrize("m,n", [(1030, 700), (1024, 1024)])
def test_singular_values_lapack(m, n):
    d, e, u, v = _case(m, n, 5 * m + n)
    g = run_factor(m, n, d, e, u, v)
    s0 = np.linalg.svd(H.bidiag_dense(d, e, m) + np.outer(u, v), compute_uv=False)
    s1 = np.linalg.svd(H.bidiag_dense(g["alpha"], g["beta"], m), compute_uv=False)
    assert np.abs(s0 - s1).max() <= 1e-12 * s0[0]


def test_deterministic():
    m, n = 530, 529
    d, e, u, v = _case(m, n, 2)
    a = run_factor(m, n, d, e, u, v)
    b = run_factor(m, n, d, e, u, v)
    for k in a:
        assert np.array_equal(a[k], b[k])


def _factorization(m, n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    P, _ = np.linalg.qr(rng.standard_normal((n, n)))
    k = min(m, n)
    return Q, rng.standard_normal(k), rng.standard_normal(max(k - 1, 1))[: max(k - 1, 0)], P


@pytest.mark.parametrize("m,n,r", [(40, 30, 1), (64, 64, 2), (300, 200, 2), (257, 257, 1)])
def test_update_bhu_matches_oracle(m, n, r):
    bdu = _bdu()
    Q, d, e, P = _factorization(m, n, m + n)
    rng = np.random.default_rng(m * n)
    A = Q @ H.bidiag_dense(d, e, m) @ P.T
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        for h in range(2):
            Bm = rng.standard_normal((m, r)); Cm = rng.standard_normal((n, r))
            F.update_bhu(Bm, Cm)
            Q, d, e, P = H.update_direct(Q, d, e, P, Bm, Cm)  # one sweep for the r columns
            A = A + Bm @ Cm.T
        Qg, dg, eg, Pg = F.read()
    scale = np.linalg.norm(A)
    assert np.abs(dg - d).max() <= tol(n, scale) and np.abs(eg[: n - 1] - e).max() <= tol(n, scale)
    assert np.abs(Qg - Q).max() <= 1e-12 * m and np.abs(Pg - P).max() <= 1e-12 * n
    assert np.abs(Qg @ H.bidiag_dense(dg, eg[: n - 1], m) @ Pg.T - A).max() <= 1e-12 * scale


def test_update_bhu_lower_and_mixed_methods():
    """m < n (the transposed form) and BHU and Givens updates on one handle: the
    factorization stays exact (reconstruction, orthogonality) and its bidiagonal
    agrees in magnitude with the Givens oracle's (both keep P's first column)."""
    import oracle as O
    bdu = _bdu()
    for (m, n) in ((30, 40), (50, 50)):
        Q, d, e, P = _factorization(m, n, 3 * m + n)
        rng = np.random.default_rng(m + 7 * n)
        A = Q @ (O.lower_bidiag_dense(d, e, m, n) if m < n else H.bidiag_dense(d, e, m)) @ P.T
        with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
            for h in range(3):
                b = rng.standard_normal(m); c = rng.standard_normal(n)
                (F.update_bhu if h != 1 else F.update)(b, c)
                A = A + np.outer(b, c)
            Qg, dg, eg, Pg = F.read()
        k = min(m, n)
        Bg = O.lower_bidiag_dense(dg, eg[: k - 1], m, n) if m < n else H.bidiag_dense(dg, eg[: k - 1], m)
        scale = np.linalg.norm(A)
        assert np.abs(Qg @ Bg @ Pg.T - A).max() <= 1e-12 * scale
        assert np.abs(Qg.T @ Qg - np.eye(m)).max() <= 1e-12 and np.abs(Pg.T @ Pg - np.eye(n)).max() <= 1e-12
        s0 = np.linalg.svd(A, compute_uv=False)
        s1 = np.linalg.svd(Bg, compute_uv=False)
        assert np.abs(s0 - s1).max() <= 1e-12 * s0[0]


def test_update_bhu_needs_fp64():
    bdu = _bdu()
    Q, d, e, P = _factorization(20, 20, 1)
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED) as F:
        with pytest.raises(bdu.BduError):
            F.update_bhu(np.ones(20), np.ones(20))


def test_full_size_against_the_givens_handle():
    """m = n = 4096 recommender update: BHU's bidiagonal equals the FP64 Givens
    update's (bit-identical to its oracle at this size) up to signs."""
    from paper_2509_02840_gb300 import inputs as I
    bdu = _bdu()
    m = n = 4096
    Q, d, e, P = I.factorization(m, n, config=1)
    B, C = I.recommender_update(m, n, 0, config=1)
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        F.update_bhu(B, C)
        _, dh, eh, _ = F.read()
        sh = F.singular_values(64)
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        F.update(B, C)
        _, dg, eg, _ = F.read()
        sg = F.singular_values(64)
    assert np.abs(sh - sg).max() <= 1e-12 * sg[0]
    # ||A+||_F <= ||Bd||_F + ||b|| ||c||
    scale = np.sqrt(np.sum(d ** 2) + np.sum(e ** 2)) + np.linalg.norm(B) * np.linalg.norm(C)
    assert np.abs(np.abs(dh) - np.abs(dg)).max() <= tol(n, scale)
    assert np.abs(np.abs(eh) - np.abs(eg)).max() <= tol(n, scale)


@pytest.mark.parametrize("m,n,rk", [(300, 200, 10), (257, 257, 3)])
def test_update_bhu_rank_r_against_the_givens_handle(m, n, rk):
    """A rank-r update by BHU (sweeps of up to 8 columns) and by the Givens
    update (r rank-1 steps, bit-identical to its oracle) on two handles: the
    bidiagonals agree up to signs, both factorizations reconstruct A + B C^T."""
    bdu = _bdu()
    Q, d, e, P = _factorization(m, n, 9 * m + rk)
    rng = np.random.default_rng(rk)
    Bm = rng.standard_normal((m, rk)); Cm = rng.standard_normal((n, rk))
    A = Q @ H.bidiag_dense(d, e, m) @ P.T + Bm @ Cm.T
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        F.update_bhu(Bm, Cm)
        Qh, dh, eh, Ph = F.read()
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        F.update(Bm, Cm)
        _, dg, eg, _ = F.read()
    scale = np.linalg.norm(A)
    assert np.abs(Qh @ H.bidiag_dense(dh, eh[: n - 1], m) @ Ph.T - A).max() <= 1e-12 * scale
    assert np.abs(np.abs(dh) - np.abs(dg)).max() <= tol(n, scale)
    assert np.abs(np.abs(eh) - np.abs(eg)).max() <= tol(n, scale)
