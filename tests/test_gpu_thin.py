"""Rank-k tracking on the GPU (bdu_thin_*; Sec. 4, Eqs. lrup - bdlrup) against
the oracle's thin_update.  The projections and products are library BLAS
calls whose summation order differs from numpy's, so the FP64 comparison is
within FP64 rounding: the same removed index at every step, d, e and the
factors to 1e-10 relative, the reported truncation error equal to the true
Frobenius error, orthonormal factors, and exact tracking of a stream that
stays within rank k.  The mixed form (FP32 thin factors) is held to the
properties that do not depend on which of two nearly equal column norms is
removed (they can differ by 1e-8 relative): the reported error of every step
equal to its true error, orthogonality within 1e-5, exact tracking within
rank k."""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu


def _start(m, n, k, which, zero=False):
    g = np.random.default_rng(2000 + which)
    Q1 = I.householder_orthogonal(m, g)[:, :k].copy(order="F")
    P1 = I.householder_orthogonal(n, g)[:, :k].copy(order="F")
    d = np.zeros(k) if zero else g.uniform(1.0, 10.0, k)
    e = np.zeros(k - 1) if zero else g.standard_normal(k - 1)
    return Q1, d, e, P1, g


def _dense(Q1, d, e, P1):
    return Q1 @ O.bidiag_dense(d, e) @ P1.T


@pytest.mark.parametrize("m,n,k,steps", [(120, 90, 8, 12), (64, 300, 10, 8), (700, 650, 40, 6), (30, 31, 1, 5)])
def test_thin_matches_oracle(m, n, k, steps):
    Q1, d, e, P1, g = _start(m, n, k, 1)
    Qo, do, eo, Po = Q1, d, e, P1
    with bdu.ThinTracker(Q1, d, e, P1) as T:
        for h in range(steps):
            b = g.standard_normal(m) * (1 + h % 3); c = g.standard_normal(n)
            A = _dense(Qo, do, eo, Po) + np.outer(b, c)
            i, err2 = T.update(b, c)
            Qo, do, eo, Po, io, eo2 = O.thin_update(Qo, do, eo, Po, b, c)
            assert i == io
            assert abs(err2 - eo2) <= 1e-10 * np.linalg.norm(A) ** 2
            Qg, dg, eg, Pg = T.read()
            scale = np.max(np.abs(do))
            assert np.max(np.abs(dg - do)) <= 1e-10 * scale
            assert np.max(np.abs(eg - eo), initial=0.0) <= 1e-10 * scale
            assert np.max(np.abs(Qg - Qo)) <= 1e-9 and np.max(np.abs(Pg - Po)) <= 1e-9
            res = np.linalg.norm(A - _dense(Qg, dg, eg, Pg)) ** 2
            assert abs(res - err2) <= 1e-10 * np.linalg.norm(A) ** 2
        assert np.linalg.norm(Qg.T @ Qg - np.eye(k)) <= 1e-12 * k
        assert np.linalg.norm(Pg.T @ Pg - np.eye(k)) <= 1e-12 * k
        assert T.stats()["updates"] == steps


def test_stream_within_rank_k_is_exact():
    m, n, k = 400, 300, 12
    Q1, d, e, P1, g = _start(m, n, k, 2, zero=True)
    S = np.zeros((m, n))
    with bdu.ThinTracker(Q1, d, e, P1) as T:
        for h in range(9):
            b = g.standard_normal(m); c = g.standard_normal(n)
            S += np.outer(b, c)
            i, err2 = T.update(b, c)
            assert err2 == 0.0 and i == k
        Qg, dg, eg, Pg = T.read()
    assert np.linalg.norm(_dense(Qg, dg, eg, Pg) - S) <= 1e-12 * np.linalg.norm(S)
    sv = np.linalg.svd(S, compute_uv=False)[:k]
    np.testing.assert_allclose(O.singular_values(dg, eg), sv, rtol=0, atol=1e-12 * sv[0])


def test_update_inside_the_subspace_and_device_vectors():
    import torch
    m, n, k = 200, 160, 9
    Q1, d, e, P1, g = _start(m, n, k, 3)
    with bdu.ThinTracker(Q1, d, e, P1) as T:
        b = Q1 @ g.standard_normal(k); c = P1 @ g.standard_normal(k)
        tb = torch.from_numpy(b).cuda(); tc = torch.from_numpy(c).cuda()
        torch.cuda.synchronize()
        i, err2 = T.update_dev(tb.data_ptr(), tc.data_ptr())
        Qg, dg, eg, Pg = T.read()
        st = T.stats()
    _, _, _, _, io, eo2 = O.thin_update(Q1, d, e, P1, b, c)
    assert st["in_span_b"] == 1 and st["in_span_c"] == 1
    assert i == io == k
    A = _dense(Q1, d, e, P1) + np.outer(b, c)
    assert np.linalg.norm(A - _dense(Qg, dg, eg, Pg)) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(Qg.T @ Qg - np.eye(k)) <= 1e-12 * k
    assert np.linalg.norm(Pg.T @ Pg - np.eye(k)) <= 1e-12 * k


def test_bad_arguments():
    Q1, d, e, P1, _ = _start(20, 10, 4, 4)
    for k in (0, 10, 11):
        with pytest.raises(bdu.BduError):
            bdu.ThinTracker(np.zeros((20, k)), np.ones(k), np.ones(max(k - 1, 0)), np.zeros((10, k)))
    L = bdu.load()
    o = bdu.Options()
    L.bdu_default_options(o)
    o.precision = 7
    import ctypes
    h = ctypes.c_void_p()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.bdu_thin_create(ctypes.byref(h), 20, 10, 4, dp(Q1), dp(d), dp(e), dp(P1), ctypes.byref(o)) == 1
    with bdu.ThinTracker(Q1, d, e, P1) as T:
        with pytest.raises(ValueError):
            T.update(np.ones(19), np.ones(10))
        with pytest.raises(bdu.BduError):
            T.update(np.full(20, np.nan), np.ones(10))


def test_mixed_thin_properties():
    m, n, k = 700, 650, 40
    Q1, d, e, P1, g = _start(m, n, k, 5)
    with bdu.ThinTracker(Q1, d, e, P1, precision=bdu.MIXED) as T:
        Qg, dg, eg, Pg = T.read()
        assert np.max(np.abs(Qg - Q1)) <= 1e-7 and np.array_equal(dg, d)
        for h in range(8):
            b = g.standard_normal(m) * (1 + h % 3); c = g.standard_normal(n)
            A = _dense(Qg, dg, eg, Pg) + np.outer(b, c)
            i, err2 = T.update(b, c)
            Qg, dg, eg, Pg = T.read()
            assert 0 <= i <= k
            res = np.linalg.norm(A - _dense(Qg, dg, eg, Pg)) ** 2
            assert abs(res - err2) <= 1e-5 * np.linalg.norm(A) ** 2
            assert np.linalg.norm(Qg.T @ Qg - np.eye(k), 2) <= 1e-5
            assert np.linalg.norm(Pg.T @ Pg - np.eye(k), 2) <= 1e-5


def test_mixed_stream_within_rank_k():
    m, n, k = 400, 300, 12
    Q1, d, e, P1, g = _start(m, n, k, 2, zero=True)
    S = np.zeros((m, n))
    with bdu.ThinTracker(Q1, d, e, P1, precision=bdu.MIXED) as T:
        for h in range(9):
            b = g.standard_normal(m); c = g.standard_normal(n)
            S += np.outer(b, c)
            i, err2 = T.update(b, c)
            assert err2 == 0.0 and i == k
        Qg, dg, eg, Pg = T.read()
    assert np.linalg.norm(_dense(Qg, dg, eg, Pg) - S) <= 1e-5 * np.linalg.norm(S)
    sv = np.linalg.svd(S, compute_uv=False)[:k]
    np.testing.assert_allclose(O.singular_values(dg, eg), sv, rtol=0, atol=1e-5 * sv[0])
