"""Batched updates of many resident factorizations of uneven sizes and
ranks (bdu_update_batch): each factorization's result is the same alone and
in the mix -- bit for bit, in both forms -- and equals the oracle in FP64."""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu

SPECS = [(64, 64, 1), (90, 40, 2), (128, 128, 4), (200, 77, 3), (33, 33, 1), (256, 200, 2),
         (300, 300, 1), (17, 5, 4), (520, 300, 2), (700, 650, 3), (1024, 1024, 1), (96, 96, 0)]


def _upload(torch, X):
    return torch.from_numpy(np.asfortranarray(X).reshape(-1, order="F").copy()).cuda()


@pytest.mark.parametrize("precision", [bdu.FP64, bdu.MIXED])
def test_batch_equals_alone(precision):
    import torch
    facs, alone, keep, ptrB, ptrC, ranks = [], [], [], [], [], []
    for idx, (m, n, r) in enumerate(SPECS):
        Q, d, e, P = I.factorization(m, n, config=4, which=idx)
        B, C = I.dense_update(m, n, h=idx, config=4, r=max(r, 1))
        B, C = B[:, :r], C[:, :r]
        facs.append(bdu.Factorization(Q, d, e, P, precision=precision))
        alone.append(bdu.Factorization(Q, d, e, P, precision=precision))
        tb, tc = _upload(torch, B), _upload(torch, C)
        keep += [tb, tc]
        ptrB.append(tb.data_ptr()); ptrC.append(tc.data_ptr()); ranks.append(r)
    torch.cuda.synchronize()
    for rnd in range(2):
        bdu.update_batch(facs, ptrB, ptrC, ranks)
        for f, b, c, r in zip(alone, ptrB, ptrC, ranks):
            f.update_dev(b, c, r)
    for f, g, (m, n, r) in zip(facs, alone, SPECS):
        Qa, da, ea, Pa = f.read()
        Qb, db, eb, Pb = g.read()
        assert np.array_equal(da, db) and np.array_equal(ea, eb), (m, n, r)
        assert np.array_equal(Qa, Qb) and np.array_equal(Pa, Pb), (m, n, r)
    for f in facs + alone:
        f.close()


def test_batch_matches_oracle_fp64():
    import torch
    specs = [(50, 50, 2), (80, 31, 3), (120, 120, 1)]
    facs, keep, ptrB, ptrC, ranks, ref = [], [], [], [], [], []
    for idx, (m, n, r) in enumerate(specs):
        Q, d, e, P = I.factorization(m, n, config=4, which=100 + idx)
        B, C = I.dense_update(m, n, h=idx, config=4, r=r)
        facs.append(bdu.Factorization(Q, d, e, P))
        tb, tc = _upload(torch, B), _upload(torch, C)
        keep += [tb, tc]
        ptrB.append(tb.data_ptr()); ptrC.append(tc.data_ptr()); ranks.append(r)
        ref.append(O.update(Q, d, e, P, B, C))
    torch.cuda.synchronize()
    bdu.update_batch(facs, ptrB, ptrC, ranks)
    for f, (Qo, do, eo, Po, _) in zip(facs, ref):
        Qg, dg, eg, Pg = f.read()
        assert np.array_equal(dg, do) and np.array_equal(eg, eo)
        assert np.array_equal(Qg, Qo) and np.array_equal(Pg, Po)
        f.close()


def test_batch_rejects_repeats_and_mixed_forms():
    import torch
    Q, d, e, P = I.factorization(20, 20, config=4, which=1)
    f = bdu.Factorization(Q, d, e, P)
    g = bdu.Factorization(Q, d, e, P, precision=bdu.MIXED)
    tb = _upload(torch, np.ones((20, 1)))
    with pytest.raises(bdu.BduError):
        bdu.update_batch([f, f], [tb.data_ptr()] * 2, [tb.data_ptr()] * 2, [1, 1])
    with pytest.raises(bdu.BduError):
        bdu.update_batch([f, g], [tb.data_ptr()] * 2, [tb.data_ptr()] * 2, [1, 1])
    f.close(); g.close()
