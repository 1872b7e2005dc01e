"""Inputs at the edges of the FP64 range.  Rotation generation scales by exact
powers of two (Eqs. giv, giv1, with the safe scaling the oracle states), so
the FP64 form must stay bit-identical to the oracle when squares of the
entries would overflow or underflow, when entries are subnormal, and when the
two entries of a rotation differ by more than 2^1021; the mixed form (whose
fast generator routes such pairs to the exactly scaled one) must stay within
its tolerances and produce finite, orthogonal factors."""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu


def _spread_column(m, seed):
    """A column whose entries span the FP64 range: huge, tiny, subnormal, zero."""
    g = np.random.default_rng(seed)
    mags = [1e300, 1e-300, 5e-310, 1.0, 0.0, 1e-200, 1e200, 3e-320, 1e150, 1e-150]
    b = np.array([mags[i % len(mags)] for i in range(m)]) * g.choice([-1.0, 1.0], m)
    g.shuffle(b)
    return b.reshape(m, 1)


def _run(Q, d, e, P, ups, precision):
    with bdu.Factorization(Q, d, e, P, precision=precision) as F:
        for B, C in ups:
            F.update(B, C)
        return F.read()


def _oracle(Q, d, e, P, ups):
    for B, C in ups:
        Q, d, e, P, _ = O.update(Q, d, e, P, B, C)
    return Q, d, e, P


@pytest.mark.parametrize("scale", [2.0 ** 700, 2.0 ** -700])
@pytest.mark.parametrize("m,n", [(96, 64), (600, 520)])
def test_fp64_scaled_problem_is_bitwise(scale, m, n):
    Q, d, e, P = I.factorization(m, n, config=0, which=17)
    ups = [(B * scale, C) for B, C in (I.dense_update(m, n, h, config=0) for h in range(2))]
    got = _run(Q, d * scale, e * scale, P, ups, bdu.FP64)
    want = _oracle(Q, d * scale, e * scale, P, ups)
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("m,n", [(40, 24), (33, 33)])
def test_fp64_range_spanning_column_is_bitwise(m, n):
    Q, P = np.eye(m), np.eye(n)
    _, d, e, _ = I.factorization(m, n, config=0, which=3)
    ups = [(_spread_column(m, s), I.dense_update(m, n, s, config=0)[1]) for s in range(2)]
    got = _run(Q, d, e, P, ups, bdu.FP64)
    want = _oracle(Q, d, e, P, ups)
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("m,n", [(40, 24), (33, 33), (700, 600)])
def test_mixed_range_spanning_column(m, n):
    Q, P = np.eye(m), np.eye(n)
    _, d, e, _ = I.factorization(m, n, config=0, which=3)
    ups = [(_spread_column(m, s), I.dense_update(m, n, s, config=0)[1]) for s in range(2)]
    Qg, dg, eg, Pg = _run(Q, d, e, P, ups, bdu.MIXED)
    Qo, do, eo, Po = _oracle(Q, d, e, P, ups)
    assert np.all(np.isfinite(dg)) and np.all(np.isfinite(eg))
    sv_g = np.linalg.svd(O.bidiag_dense(dg, eg), compute_uv=False)
    sv_o = np.linalg.svd(O.bidiag_dense(do, eo), compute_uv=False)
    assert np.max(np.abs(sv_g - sv_o)) / sv_o[0] <= 1e-5
    assert np.linalg.norm(Qg.T @ Qg - np.eye(m), 2) <= 1e-5
    assert np.linalg.norm(Pg.T @ Pg - np.eye(n), 2) <= 1e-5


@pytest.mark.parametrize("scale", [2.0 ** 700, 2.0 ** -700])
def test_mixed_scaled_problem(scale):
    m, n = 600, 520
    Q, d, e, P = I.factorization(m, n, config=0, which=19)
    ups = [(B * scale, C) for B, C in (I.dense_update(m, n, h, config=0) for h in range(2))]
    Qg, dg, eg, Pg = _run(Q, d * scale, e * scale, P, ups, bdu.MIXED)
    Qo, do, eo, Po = _oracle(Q, d * scale, e * scale, P, ups)
    sv_g = np.linalg.svd(O.bidiag_dense(dg / scale, eg / scale), compute_uv=False)
    sv_o = np.linalg.svd(O.bidiag_dense(do / scale, eo / scale), compute_uv=False)
    assert np.max(np.abs(sv_g - sv_o)) / sv_o[0] <= 1e-5
    assert np.linalg.norm(Qg.T @ Qg - np.eye(m), 2) <= 1e-5
