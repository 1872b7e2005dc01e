"""The overlapped mixed form: the application of each rank-1 update to Q and P
runs on a second stream while the next update's rotations are generated, and
the next projection is formed from the factors before that application and
rotated by its rotations (u = G^T Q^T b, Sec. 3.2).  Same tolerances as the
plain mixed form against the FP64 oracle; deferred work is completed by every
call that reads the factors; the FP64 form ignores the option."""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu


def _check(Qg, dg, eg, Pg, Qo, do, eo, Po, A=None):
    m, n = Qg.shape[0], Pg.shape[0]
    sv_g = np.linalg.svd(O.bidiag_dense(dg, eg), compute_uv=False)
    sv_o = np.linalg.svd(O.bidiag_dense(do, eo), compute_uv=False)
    assert np.max(np.abs(sv_g - sv_o) / sv_o[0]) <= 1e-5
    assert np.linalg.norm(Qg.T @ Qg - np.eye(m), 2) <= 1e-5
    assert np.linalg.norm(Pg.T @ Pg - np.eye(n), 2) <= 1e-5
    if A is not None:
        R = Qg @ O.bidiag_dense(dg, eg, m) @ Pg.T
        assert np.linalg.norm(A - R) / np.linalg.norm(A) <= 1e-5


@pytest.mark.parametrize("m,n", [(96, 64), (300, 300), (420, 200), (640, 576)])
def test_overlapped_matches_oracle(m, n):
    Q, d, e, P = I.factorization(m, n, config=0, which=3)
    Qo, do, eo, Po = Q, d, e, P
    A = Q @ O.bidiag_dense(d, e, m) @ P.T
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, overlap=True) as F:
        for h in range(6):
            B, C = I.dense_update(m, n, h, config=0)
            F.update(B, C)
            A += B @ C.T
            Qo, do, eo, Po, _ = O.update(Qo, do, eo, Po, B, C)
        Qg, dg, eg, Pg = F.read()
    _check(Qg, dg, eg, Pg, Qo, do, eo, Po, A)


def test_overlapped_close_to_plain_mixed():
    """Overlapped and plain mixed forms differ only in rounding."""
    m, n = 512, 512
    Q, d, e, P = I.factorization(m, n, config=1)
    outs = []
    for ov in (False, True):
        with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, overlap=ov) as F:
            for h in range(5):
                F.update(*I.recommender_update(m, n, h, config=1))
            outs.append(F.read())
    (Qa, da, ea, Pa), (Qb, db, eb, Pb) = outs
    sa = np.linalg.svd(O.bidiag_dense(da, ea), compute_uv=False)
    sb = np.linalg.svd(O.bidiag_dense(db, eb), compute_uv=False)
    assert np.max(np.abs(sa - sb)) / sa[0] <= 1e-5
    Ra = Qa @ O.bidiag_dense(da, ea, m) @ Pa.T
    Rb = Qb @ O.bidiag_dense(db, eb, m) @ Pb.T
    assert np.linalg.norm(Ra - Rb) / np.linalg.norm(Ra) <= 1e-5


def test_deferred_work_is_completed_by_reads_and_mixed_calls():
    """A read between updates, a rank-2 update (which completes the deferred
    application first), d/e-only reads (which need none) and the orthogonality
    check all see a consistent factorization."""
    m, n = 200, 150
    Q, d, e, P = I.factorization(m, n, config=0, which=5)
    Qo, do, eo, Po = Q, d, e, P
    A = Q @ O.bidiag_dense(d, e, m) @ P.T
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, overlap=True, check_every=2) as F:
        for h in range(7):
            r = 2 if h == 3 else 1
            B, C = I.dense_update(m, n, h, config=0, r=r)
            F.update(B, C)
            A += B @ C.T
            Qo, do, eo, Po, _ = O.update(Qo, do, eo, Po, B, C)
            if h == 1:
                Qm, dm, em, Pm = F.read()
                _check(Qm, dm, em, Pm, Qo, do, eo, Po, A)
            if h == 4:
                dd, ee = F.read_bidiagonal()
                so = np.linalg.svd(O.bidiag_dense(do, eo), compute_uv=False)
                sg = np.linalg.svd(O.bidiag_dense(dd, ee), compute_uv=False)
                assert np.max(np.abs(sg - so)) / so[0] <= 1e-5
            if h == 5:
                q_est, p_est = F.check_orthogonality()
                assert q_est <= 1e-5 and p_est <= 1e-5
        F.sync()
        Qg, dg, eg, Pg = F.read()
    _check(Qg, dg, eg, Pg, Qo, do, eo, Po, A)


def test_flush_then_read_on_a_caller_stream():
    """With the caller's stream, bdu_flush enqueues the deferred application
    there; the factorization read afterwards reconstructs the same matrix as
    the plain mixed form (signs of Q's and P's columns may differ where an
    eliminated entry is at rounding level, so reconstructions are compared)."""
    import torch
    m, n = 256, 256
    Q, d, e, P = I.factorization(m, n, config=0, which=7)
    s = torch.cuda.Stream()
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, overlap=True, stream=s.cuda_stream) as F:
        for h in range(3):
            F.update(*I.dense_update(m, n, h, config=0))
        F.flush()
        s.synchronize()
        Qr, dr, er, Pr = F.read()
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED) as G:
        G.flush()  # a no-op without overlap
        for h in range(3):
            G.update(*I.dense_update(m, n, h, config=0))
        Qs, ds, es, Ps = G.read()
    Rr = Qr @ O.bidiag_dense(dr, er, m) @ Pr.T
    Rs = Qs @ O.bidiag_dense(ds, es, m) @ Ps.T
    assert np.linalg.norm(Rr - Rs) / np.linalg.norm(Rs) <= 1e-5


def test_fp64_form_ignores_overlap():
    m, n = 128, 96
    Q, d, e, P = I.factorization(m, n, config=0, which=11)
    outs = []
    for ov in (False, True):
        with bdu.Factorization(Q, d, e, P, precision=bdu.FP64, overlap=ov) as F:
            for h in range(3):
                F.update(*I.dense_update(m, n, h, config=0))
            outs.append(F.read())
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
