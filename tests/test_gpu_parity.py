"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 form: the library and the oracle implement the same schedule with the
same separately rounded IEEE operations, so d, e, Q, P and the rotation
streams must be bit-identical (compared with ==).  Mixed form (FP32 Q/P):
singular values within 1e-5 relative and ||Q^T Q - I||_2 <= 1e-5.
"""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu


def _gpu_update(Q, d, e, P, B, C, precision=bdu.FP64):
    with bdu.Factorization(Q, d, e, P, precision=precision) as F:
        F.update(B, C)
        out = F.read()
        rots = (F.read_rotations(0), F.read_rotations(1)) if B.shape[1] == 1 else None
        st = F.stats()
    return out, rots, st


SHAPES = [(1, 1), (2, 1), (5, 1), (2, 2), (3, 2), (3, 3), (4, 3), (5, 4), (8, 8), (9, 8),
          (17, 5), (33, 33), (40, 39), (64, 16), (100, 100), (130, 97), (256, 128), (300, 300)]


@pytest.mark.parametrize("m,n", SHAPES)
@pytest.mark.parametrize("r", [1, 3])
def test_fp64_bitwise(m, n, r):
    Q, d, e, P = I.factorization(m, n, config=0, which=m * 1000 + n)
    B, C = I.dense_update(m, n, h=r, config=0, r=r)
    (Qg, dg, eg, Pg), rots, st = _gpu_update(Q, d, e, P, B, C)
    Qo, do, eo, Po, cnt = O.update(Q, d, e, P, B, C)
    assert np.array_equal(dg, do) and np.array_equal(eg, eo)
    assert np.array_equal(Qg, Qo) and np.array_equal(Pg, Po)
    assert st["rot_left"] == [cnt["left"][p] for p in O.PHASES]
    assert st["rot_right"] == [cnt["right"][p] for p in O.PHASES]
    if rots is not None:
        U, V = O.project(Q, P, B, C)
        _, _, L, R, _ = O.generate(m, n, d, e, U, V)
        for (c, s, a), ref in ((rots[0], L), (rots[1], R)):
            assert len(c) == len(ref)
            assert np.array_equal(c, ref.c) and np.array_equal(s, ref.s) and np.array_equal(a, ref.a)



@pytest.mark.parametrize("m,n", [(64, 48), (130, 97), (256, 128)])
def test_mixed_rotations_are_the_fp32_coefficients(m, n):
    """The mixed form keeps only the FP32 coefficients its factors are rotated
    with: read_rotations returns FP32 values, as many rotations on the same
    pairs as the oracle generates, each close to the oracle's (its inputs
    differ from the oracle's by the FP32 rounding of Q and P)."""
    Q, d, e, P = I.factorization(m, n, config=0, which=m + n)
    B, C = I.dense_update(m, n, h=1, config=0, r=1)
    _, rots, _ = _gpu_update(Q, d, e, P, B, C, precision=bdu.MIXED)
    U, V = O.project(Q, P, B, C)
    _, _, L, R, _ = O.generate(m, n, d, e, U, V)
    for (c, s, a), ref in ((rots[0], L), (rots[1], R)):
        assert len(c) == len(ref) and np.array_equal(a, ref.a)
        assert np.array_equal(c, c.astype(np.float32).astype(np.float64))
        assert np.array_equal(s, s.astype(np.float32).astype(np.float64))
        assert np.max(np.abs(c * c + s * s - 1.0)) <= 1e-6
        assert np.median(np.abs(c - ref.c)) <= 1e-5 and np.median(np.abs(s - ref.s)) <= 1e-5

def test_fp64_stream_config0():
    """20 sequential rank-1 updates at m=256, n=128, compared after every update."""
    m, n = 256, 128
    Q, d, e, P = I.factorization(m, n, config=0)
    A = Q @ O.bidiag_dense(d, e, m) @ P.T
    Qo, do, eo, Po = Q, d, e, P
    with bdu.Factorization(Q, d, e, P) as F:
        for h in range(20):
            B, C = I.dense_update(m, n, h, config=0)
            A = A + B @ C.T
            F.update(B, C)
            Qo, do, eo, Po, _ = O.update(Qo, do, eo, Po, B, C)
            dg, eg = F.read_bidiagonal()
            assert np.array_equal(dg, do) and np.array_equal(eg, eo), h
        Qg, dg, eg, Pg = F.read()
    assert np.array_equal(Qg, Qo) and np.array_equal(Pg, Po)
    R = Qg @ O.bidiag_dense(dg, eg, m) @ Pg.T
    assert np.linalg.norm(A - R) / np.linalg.norm(A) <= 1e-12


def test_edge_cases_fp64():
    m, n = 20, 12
    Q, d, e, P = I.factorization(m, n, config=0, which=5)
    with bdu.Factorization(Q, d, e, P) as F:
        F.update(np.zeros((m, 0)), np.zeros((n, 0)))    # rank 0: no-op
        F.update(np.zeros(m), np.ones(n))                # b = 0: no rotation
        Qg, dg, eg, Pg = F.read()
        assert F.stats()["rot_left"] == [0, 0, 0, 0]
    assert np.array_equal(dg, d) and np.array_equal(eg, e) and np.array_equal(Qg, Q)
    # Bd = 0, rank-1 start of a stream (closed form sigma_1 = ||b|| ||c||)
    z = np.zeros(n)
    b = np.random.default_rng(0).standard_normal(m); c = np.random.default_rng(1).standard_normal(n)
    (Qg, dg, eg, Pg), _, _ = _gpu_update(Q, z, z[:-1], P, b.reshape(m, 1), c.reshape(n, 1))
    Qo, do, eo, Po, _ = O.update(Q, z, z[:-1], P, b, c)
    assert np.array_equal(dg, do) and np.array_equal(eg, eo)
    assert abs(np.hypot(dg[0], eg[0]) - np.linalg.norm(b) * np.linalg.norm(c)) < 1e-12 * np.linalg.norm(b) * np.linalg.norm(c)


@pytest.mark.parametrize("m,n", [(256, 128), (300, 300)])
def test_mixed_form_tolerances(m, n):
    """FP32 Q/P: singular values within 1e-5 of the oracle's, ||Q^T Q - I||_2 <= 1e-5."""
    Q, d, e, P = I.factorization(m, n, config=0)
    Qo, do, eo, Po = Q, d, e, P
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED) as F:
        for h in range(5):
            B, C = I.dense_update(m, n, h, config=0)
            F.update(B, C)
            Qo, do, eo, Po, _ = O.update(Qo, do, eo, Po, B, C)
        Qg, dg, eg, Pg = F.read()
    sv_g = np.linalg.svd(O.bidiag_dense(dg, eg), compute_uv=False)
    sv_o = np.linalg.svd(O.bidiag_dense(do, eo), compute_uv=False)
    assert np.max(np.abs(sv_g - sv_o) / sv_o[0]) <= 1e-5
    assert np.linalg.norm(Qg.T @ Qg - np.eye(m), 2) <= 1e-5
    assert np.linalg.norm(Pg.T @ Pg - np.eye(n), 2) <= 1e-5


def test_full_size_recommender_sampled_rows():
    """m = n = 4096 recommender update: d, e and sampled rows of Q, P bit-identical."""
    m = n = 4096
    Q, d, e, P = I.factorization(m, n, config=1)
    B, C = I.recommender_update(m, n, h=0, config=1)
    with bdu.Factorization(Q, d, e, P) as F:
        F.update(B, C)
        Qg, dg, eg, Pg = F.read()
    U, V = O.project(Q, P, B, C)
    do, eo, L, R, _ = O.generate(m, n, d, e, U, V)
    assert np.array_equal(dg, do) and np.array_equal(eg, eo)
    rows = np.array([0, 1, 777, 2048, 4094, 4095])
    assert np.array_equal(O.apply_rows(Q, rows, L)[rows], Qg[rows])
    assert np.array_equal(O.apply_rows(P, rows, R)[rows], Pg[rows])
