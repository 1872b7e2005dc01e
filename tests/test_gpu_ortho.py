"""Orthogonality control of the mixed form: the probe's estimate of
||X^T X - I||_2 and the re-orthogonalization that keeps a long FP32 stream
within the stated tolerances (singular values within 1e-5 relative of the
exact ones, ||Q^T Q - I||_2 <= 1e-5)."""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu


def test_probe_estimates_the_spectral_norm():
    m = n = 300
    Q, d, e, P = I.factorization(m, n, config=0, which=2)
    g = np.random.default_rng(0)
    u = g.standard_normal(m); v = g.standard_normal(m)
    Qp = Q + 3e-6 * np.outer(u / np.linalg.norm(u), v / np.linalg.norm(v))
    exact = np.linalg.norm(Qp.T @ Qp - np.eye(m), 2)
    with bdu.Factorization(Qp, d, e, P, precision=bdu.FP64) as F:
        q_est, p_est = F.check_orthogonality()
        st = F.stats()
    assert 0.9 * exact <= q_est <= 1.0001 * exact
    assert p_est < 1e-12
    assert st["ortho_q"] == q_est


def test_block_stream_with_reorthogonalization():
    """Rank-8 block updates (the mixed-form configuration, scaled to m=2048,
    n=512): re-orthogonalization fires and the tolerances hold."""
    m, n, r = 2048, 512, 8
    Q, d, e, P = I.factorization(m, n, config=2)
    A = Q @ O.bidiag_dense(d, e, m) @ P.T
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, reorth_tol=1e-6, check_every=8, reorth_every=0) as F:
        for h in range(6):
            B, C = I.block_update(m, n, h, config=2, r=r)
            A += B @ C.T
            F.update(B, C)
        Qg, dg, eg, Pg = F.read()
        st = F.stats()
    assert st["reorth_q"] + st["reorth_p"] >= 1
    sv_g = np.linalg.svd(O.bidiag_dense(dg, eg), compute_uv=False)
    sv_A = np.linalg.svd(A, compute_uv=False)[:n]
    assert np.max(np.abs(sv_g - sv_A)) / sv_A[0] <= 1e-5
    assert np.linalg.norm(Qg.T @ Qg - np.eye(m), 2) <= 1e-5
    assert np.linalg.norm(Pg.T @ Pg - np.eye(n), 2) <= 1e-5
    R = Qg @ O.bidiag_dense(dg, eg, m) @ Pg.T
    assert np.linalg.norm(A - R) / np.linalg.norm(A) <= 1e-4


def test_reorthogonalization_reduces_the_error():
    m = n = 256
    Q, d, e, P = I.factorization(m, n, config=0, which=9)
    g = np.random.default_rng(1)
    Qp = Q + 2e-5 * g.standard_normal((m, m)) / np.sqrt(m)
    before = np.linalg.norm(Qp.T @ Qp - np.eye(m), 2)
    with bdu.Factorization(Qp, d, e, P, precision=bdu.MIXED, reorth_tol=1e-7, check_every=1, reorth_every=0) as F:
        B, C = I.dense_update(m, n, 0, config=0)
        F.update(B, C)
        Qg, _, _, _ = F.read()
        st = F.stats()
    assert st["reorth_q"] == 1
    after = np.linalg.norm(Qg.T @ Qg - np.eye(m), 2)
    assert after < 0.2 * before and after < 5e-6


def test_block_stream_full_size_invariants():
    """The rank-8 configuration at its full size (m = 8192, n = 2048, mixed
    form, re-orthogonalization above 1e-6): after two updates the factors are
    orthogonal to 1e-5 and a randomized residual ||A+ x - Q Bd P^T x|| / ||A+ x||
    (probe vectors x, FP64 on the host) is at the level of FP32 rounding."""
    m, n, r = 8192, 2048, 8
    Q, d, e, P = I.factorization(m, n, config=2)
    ups = [I.block_update(m, n, h, config=2, r=r) for h in range(2)]
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, reorth_tol=1e-6, check_every=1) as F:
        for B, C in ups:
            F.update(B, C)
        q_est, p_est = F.check_orthogonality()
        Qg, dg, eg, Pg = F.read()
    assert q_est <= 1e-5 and p_est <= 1e-5
    g = np.random.default_rng(7)
    X = g.standard_normal((n, 3))
    # A+ X = Q (Bd (P^T X)) + sum_h B_h (C_h^T X), all in FP64
    want = Q @ (O.bidiag_dense(d, e, m) @ (P.T @ X))
    for B, C in ups:
        want += B @ (C.T @ X)
    got = Qg @ (O.bidiag_dense(dg, eg, m) @ (Pg.T @ X))
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-5



@pytest.mark.parametrize("overlap", [False, True])
def test_default_policy_keeps_the_tolerance_after_every_update(overlap):
    """With the default policy (one Newton-Schulz step after every column) the
    mixed form keeps ||Q^T Q - I||_2 and ||P^T P - I||_2 under 1e-5 after every
    update of the rank-1 recommender stream at m = n = 4096, where FP32
    rounding alone exceeds it after the first update."""
    m = n = 4096
    Q, d, e, P = I.factorization(m, n, config=1)
    worst = 0.0
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, overlap=overlap) as F:
        for h in range(4):
            F.update(*I.recommender_update(m, n, h, config=1))
            q_est, p_est = F.check_orthogonality()
            worst = max(worst, q_est, p_est)
        st = F.stats()
    assert worst <= 1e-5
    assert st["reorth_q"] >= 3 and st["reorth_p"] >= 3


@pytest.mark.parametrize("m,n", [(300, 200), (1024, 1024)])
def test_newton_schulz_step_matches_fp64(m, n):
    """One re-orthogonalization step on the GPU (X^T X in 3xTF32 with the
    diagonal in FP64, X E in TF32, both on the tensor cores) against the same
    step in FP64 on the host, X - X (X^T X - I) / 2 (Sec. 4.2), from the same
    FP32 factor: two handles take the same update, one re-orthogonalizes Q
    after it, the other does not."""
    Q, d, e, P = I.factorization(m, n, config=0, which=11)
    g = np.random.default_rng(3)
    Qp = Q + 3e-5 * g.standard_normal((m, m)) / np.sqrt(m)
    B, C = I.dense_update(m, n, 1, config=0)
    with bdu.Factorization(Qp, d, e, P, precision=bdu.MIXED, reorth_every=0, check_every=0) as F:
        F.update(B, C)
        X, _, _, _ = F.read()
    with bdu.Factorization(Qp, d, e, P, precision=bdu.MIXED, reorth_tol=1e-9, check_every=1, reorth_every=0) as F:
        F.update(B, C)
        Qg, _, _, _ = F.read()
        st = F.stats()
    assert st["reorth_q"] == 1
    E = X.T @ X - np.eye(m)
    want = X - 0.5 * (X @ E)
    # the result is rounded to FP32 (entries up to ~1: half an ulp is 6e-8)
    # and E carries FP32-level error in absolute terms
    assert np.max(np.abs(Qg - want)) <= 2e-7
    assert np.linalg.norm(Qg.T @ Qg - np.eye(m), 2) <= 2e-6
