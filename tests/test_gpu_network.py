"""The network stream (symmetric edge insertions B = [w e_i, w e_j],
C = [e_j, e_i] between power-law nodes, rank 2) at the scaled size n = 1024 that
the oracle finishes in seconds: FP64 bit-identical to the oracle; mixed form
within its tolerances."""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu

N = 1024


def _oracle(ups):
    Q, d, e, P = I.factorization(N, N, config=3)
    for B, C in ups:
        Q, d, e, P, _ = O.update(Q, d, e, P, B, C)
    return Q, d, e, P


@pytest.fixture(scope="module")
def stream():
    ups = [I.network_update(N, h, config=3) for h in range(2)]
    return ups, _oracle(ups)


def test_network_stream_fp64_bitwise(stream):
    ups, want = stream
    Q, d, e, P = I.factorization(N, N, config=3)
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        for B, C in ups:
            F.update(B, C)
        got = F.read()
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


def test_network_stream_mixed(stream):
    ups, (Qo, do, eo, Po) = stream
    Q, d, e, P = I.factorization(N, N, config=3)
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED) as F:
        for B, C in ups:
            F.update(B, C)
        Qg, dg, eg, Pg = F.read()
    sv_g = np.linalg.svd(O.bidiag_dense(dg, eg), compute_uv=False)
    sv_o = np.linalg.svd(O.bidiag_dense(do, eo), compute_uv=False)
    assert np.max(np.abs(sv_g - sv_o)) / sv_o[0] <= 1e-5
    assert np.linalg.norm(Qg.T @ Qg - np.eye(N), 2) <= 1e-5
    assert np.linalg.norm(Pg.T @ Pg - np.eye(N), 2) <= 1e-5
