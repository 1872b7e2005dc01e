"""Both bulge-chase engines (one thread block; a 16-block cluster with the
band in distributed shared memory) give results bit-identical to the oracle
in the FP64 form, and the mixed form's fast rotation arithmetic stays within
the stated tolerances."""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("m,n,r", [(3, 3, 1), (20, 17, 2), (64, 64, 1), (130, 97, 3), (520, 513, 1),
                                   (700, 600, 2)])
def test_engines_fp64_bitwise(engine, m, n, r):
    Q, d, e, P = I.factorization(m, n, config=0, which=7 * m + n)
    B, C = I.dense_update(m, n, h=2, config=0, r=r)
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64, engine=engine) as F:
        F.update(B, C)
        Qg, dg, eg, Pg = F.read()
        st = F.stats()
    Qo, do, eo, Po, cnt = O.update(Q, d, e, P, B, C)
    assert np.array_equal(dg, do) and np.array_equal(eg, eo)
    assert np.array_equal(Qg, Qo) and np.array_equal(Pg, Po)
    assert st["rot_left"] == [cnt["left"][p] for p in O.PHASES]
    assert st["rot_right"] == [cnt["right"][p] for p in O.PHASES]


@pytest.mark.parametrize("engine", [1, 2])
def test_engines_mixed_tolerance(engine):
    m, n = 600, 600
    Q, d, e, P = I.factorization(m, n, config=0, which=3)
    Qo, do, eo, Po = Q, d, e, P
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, engine=engine) as F:
        for h in range(3):
            B, C = I.dense_update(m, n, h, config=0)
            F.update(B, C)
            Qo, do, eo, Po, _ = O.update(Qo, do, eo, Po, B, C)
        Qg, dg, eg, Pg = F.read()
    sv_g = np.linalg.svd(O.bidiag_dense(dg, eg), compute_uv=False)
    sv_o = np.linalg.svd(O.bidiag_dense(do, eo), compute_uv=False)
    assert np.max(np.abs(sv_g - sv_o)) / sv_o[0] <= 1e-5
    assert np.linalg.norm(Qg.T @ Qg - np.eye(m), 2) <= 1e-5
    assert np.linalg.norm(Pg.T @ Pg - np.eye(n), 2) <= 1e-5
