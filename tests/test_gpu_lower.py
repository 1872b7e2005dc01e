"""m < n: A = Q L P^T with L lower bidiagonal, held on the device as the
transposed problem and updated with A^T + C B^T.  The FP64 form is compared
bit for bit with the oracle's m < n update (itself pinned to the definition
in test_oracle_lower.py), the mixed form within its tolerances; the entry
points that name a side (rotations, statistics, truncation, batches) are
checked to speak of the caller's Q and P."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu

SHAPES = [(1, 4), (2, 3), (30, 64), (150, 301), (255, 256)]


def _dense(Q, d, e, P):
    return Q @ O.lower_bidiag_dense(d, e, Q.shape[0], P.shape[0]) @ P.T


@pytest.mark.parametrize("m,n", SHAPES)
def test_fp64_lower_is_bitwise(m, n):
    Q, d, e, P = I.factorization(m, n, config=0, which=71)
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        left = right = 0
        for h, r in enumerate([1, 2, 1, 3]):
            B, C = I.dense_update(m, n, h, config=0, r=r)
            F.update(B, C)
            Q, d, e, P, cnt = O.update_lower(Q, d, e, P, B, C)
            left += sum(cnt["left"].values())
            right += sum(cnt["right"].values())
        Qg, dg, eg, Pg = F.read()
        st = F.stats()
    assert Qg.shape == (m, m) and Pg.shape == (n, n) and len(dg) == m and len(eg) == m - 1
    for a, b in zip((Qg, dg, eg, Pg), (Q, d, e, P)):
        assert np.array_equal(a, b)
    # statistics: left = rotations on the caller's Q
    assert sum(st["rot_left"]) == left and sum(st["rot_right"]) == right


@pytest.mark.parametrize("overlap", [False, True])
def test_mixed_lower_within_tolerance(overlap):
    m, n = 180, 420
    Q, d, e, P = I.factorization(m, n, config=0, which=72)
    A = _dense(Q, d, e, P)
    Qo, do, eo, Po = Q, d, e, P
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, overlap=overlap) as F:
        for h in range(6):
            B, C = I.dense_update(m, n, h, config=0, r=1 if h % 3 else 2)
            F.update(B, C)
            A = A + B @ C.T
            Qo, do, eo, Po, _ = O.update_lower(Qo, do, eo, Po, B, C)
        Qg, dg, eg, Pg = F.read()
    sv_o = O.singular_values(do, eo)
    assert np.max(np.abs(O.singular_values(dg, eg) - sv_o)) <= 1e-5 * sv_o[0]
    assert np.linalg.norm(Qg.T @ Qg - np.eye(m), 2) <= 1e-5
    assert np.linalg.norm(Pg.T @ Pg - np.eye(n), 2) <= 1e-5
    assert np.linalg.norm(_dense(Qg, dg, eg, Pg) - A) <= 1e-5 * np.linalg.norm(A)


def test_orthogonality_estimates_name_the_callers_factors():
    """A Q that is off orthogonality by ~2e-4 and an exact P: the estimate
    for Q must be the large one."""
    m, n = 60, 130
    Q, d, e, P = I.factorization(m, n, config=0, which=75)
    Q = Q * (1.0 + 1e-4)
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        q_est, p_est = F.check_orthogonality()
        st = F.stats()
    assert 1e-4 < q_est < 4e-4 and p_est < 1e-12
    assert st["ortho_q"] == q_est and st["ortho_p"] == p_est


def test_rotations_name_the_callers_sides():
    """The side-0 rotations of the last column, applied in order to the columns
    of the old Q with the pair update, give the new Q bit for bit (FP64)."""
    m, n = 40, 90
    Q, d, e, P = I.factorization(m, n, config=0, which=73)
    B, C = I.dense_update(m, n, 0, config=0, r=1)
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        F.update(B, C)
        Qg, _, _, Pg = F.read()
        for side, X0, X1 in ((0, Q, Qg), (1, P, Pg)):
            c, s, a = F.read_rotations(side)
            X = X0.copy()
            for ck, sk, ak in zip(c, s, a):
                xa, xb = X[:, ak - 1].copy(), X[:, ak].copy()
                X[:, ak - 1] = ck * xa + sk * xb
                X[:, ak] = -sk * xa + ck * xb
            assert np.array_equal(X, X1)


def test_truncation_and_singular_values_lower():
    m, n = 70, 160
    Q, d, e, P = I.factorization(m, n, config=0, which=74)
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        for h in range(2):
            B, C = I.dense_update(m, n, h, config=0)
            F.update(B, C)
            Q, d, e, P, _ = O.update_lower(Q, d, e, P, B, C)
        A = _dense(Q, d, e, P)
        for r in (0, 1, 9, m):
            L, R, idx, err2 = F.read_truncated(r)
            assert L.shape == (m, r) and R.shape == (n, r)
            # the transposed problem's truncation, sides exchanged
            Lt, Rt, it, et = O.truncated_bd(P, d, e, Q, r)
            assert np.array_equal(idx, it) and err2 == et
            assert np.array_equal(L, Rt) and np.array_equal(R, Lt)
            res = np.linalg.norm(A - L @ R.T) ** 2
            assert abs(res - err2) <= 1e-11 * np.linalg.norm(A) ** 2
        sv = F.singular_values()
        assert len(sv) == m
        np.testing.assert_allclose(sv, np.linalg.svd(A, compute_uv=False), rtol=0, atol=1e-12 * sv[0])
        with pytest.raises(bdu.BduError):
            F.read_truncated(m + 1)


@pytest.mark.parametrize("precision", [bdu.FP64, bdu.MIXED])
def test_batch_with_both_orientations(precision):
    """A batch that holds m < n and m > n factorizations gives each the result
    of its own updates."""
    shapes = [(50, 120), (120, 50), (64, 64), (33, 200)]
    facts = [I.factorization(m, n, config=0, which=80 + i) for i, (m, n) in enumerate(shapes)]
    ups = [[I.dense_update(m, n, h, config=0, r=1 + (h + i) % 2) for h in range(3)]
           for i, (m, n) in enumerate(shapes)]
    alone = []
    for f, u in zip(facts, ups):
        with bdu.Factorization(*f, precision=precision) as F:
            for B, C in u:
                F.update(B, C)
            alone.append(F.read())
    Fs = [bdu.Factorization(*f, precision=precision) for f in facts]
    try:
        for h in range(3):
            keep = [(torch.from_numpy(u[h][0].reshape(-1, order="F").copy()).cuda(),
                     torch.from_numpy(u[h][1].reshape(-1, order="F").copy()).cuda()) for u in ups]
            torch.cuda.synchronize()
            bdu.update_batch(Fs, [b.data_ptr() for b, _ in keep], [c.data_ptr() for _, c in keep],
                             [u[h][0].shape[1] for u in ups])
            for F in Fs:
                F.sync()
        for F, ref in zip(Fs, alone):
            for a, b in zip(F.read(), ref):
                assert np.array_equal(a, b)
    finally:
        for F in Fs:
            F.close()
