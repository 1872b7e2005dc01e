"""Read-side truncation (bdu_read_truncated; Sec. 2, Eqs. trBD, errtrBD)
against the oracle's definition.  FP64 form: the kept indices, the error and
the columns of L and R are bit-identical to the oracle's.  Mixed form: the same
indices and error (d, e are FP64 in both forms), L and R within FP32 rounding
of the factors."""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n", [(40, 30), (300, 200), (257, 257)])
def test_fp64_truncation_is_bitwise(m, n):
    Q, d, e, P = I.factorization(m, n, config=0, which=61)
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        for h in range(2):
            B, C = I.dense_update(m, n, h, config=0)
            F.update(B, C)
            Q, d, e, P, _ = O.update(Q, d, e, P, B, C)
        for r in (0, 1, 7, n // 2, n):
            L, R, idx, err2 = F.read_truncated(r)
            Lo, Ro, io, eo = O.truncated_bd(Q, d, e, P, r)
            assert np.array_equal(idx, io) and err2 == eo
            assert np.array_equal(L, Lo) and np.array_equal(R, Ro)


@pytest.mark.parametrize("overlap", [False, True])
def test_mixed_truncation(overlap):
    m, n = 320, 288
    Q, d, e, P = I.factorization(m, n, config=0, which=62)
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, overlap=overlap) as F:
        # before any update d, e are the inputs: indices and error exactly the oracle's
        for r in (5, 100):
            L, R, idx, err2 = F.read_truncated(r)
            Lo, Ro, io, eo = O.truncated_bd(Q, d, e, P, r)
            assert np.array_equal(idx, io) and err2 == eo
            assert np.max(np.abs(L - Lo)) <= 1e-6 * np.max(np.abs(Lo))
            assert np.max(np.abs(R - Ro)) <= 1e-6
        # after an update (deferred in the overlapped form) the read sees it
        B, C = I.dense_update(m, n, 0, config=0)
        F.update(B, C)
        Qg, dg, eg, Pg = F.read()
        L, R, idx, err2 = F.read_truncated(50)
        Lo, Ro, io, eo = O.truncated_bd(Qg, dg, eg, Pg, 50)
        assert np.array_equal(idx, io) and err2 == eo
        assert np.max(np.abs(L - Lo)) <= 1e-12 * np.max(np.abs(Lo))


def test_rank_out_of_range_is_rejected():
    Q, d, e, P = I.factorization(20, 10, config=0, which=1)
    with bdu.Factorization(Q, d, e, P) as F:
        for r in (-1, 11):
            with pytest.raises(bdu.BduError):
                F.read_truncated(r)
