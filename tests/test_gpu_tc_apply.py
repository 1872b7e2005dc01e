"""The blocked tensor-core apply (mixed form, nb = 64, 96, 128): the rotations
of nb/2 consecutive chases over a window of nb/2 columns are accumulated into
an nb x nb orthogonal block and applied as a 3xTF32 product on the tensor
cores (Sec. 3.2, Eq. bidiagplus).

It rounds differently from the rotation-by-rotation FP32 apply.  After one
update both start from the same factors and run the same FP64 chase, so the
bidiagonal is identical and the factors agree to FP32 rounding, element by
element.  From the second update on, the projections differ by that rounding,
and the trailing entries of the bidiagonal of these synthetic factorizations
are ill-conditioned functions of the data (every mixed-form variant then
differs from the FP64 oracle element by element, by O(1)), so longer streams
are checked through what the paper fixes: the residual against A+ accumulated
in FP64, the singular values (Sec. 2: sigma(Bd) = sigma(A)) and orthogonality.
"""
import numpy as np
import pytest

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu


def _run(Q, d, e, P, ups, nb, overlap=False):
    with bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, nb=nb, overlap=overlap) as F:
        out = []
        for B, C in ups:
            F.update(B, C)
            out.append(F.read())
        st = F.stats()
    return out, st


@pytest.mark.parametrize("nb", [64, 96, 128])
@pytest.mark.parametrize("m,n", [(256, 256), (300, 200), (777, 500), (130, 129), (65, 3)])
def test_one_update_matches_the_oracle(m, n, nb):
    Q, d, e, P = I.factorization(m, n, config=0, which=7)
    B, C = I.dense_update(m, n, 3, config=0)
    (got,), st = _run(Q, d, e, P, [(B, C)], nb)
    assert st["apply_variant"] == [nb, nb]
    Qo, do, eo, Po, _ = O.update(Q, d, e, P, B, C)
    Qg, dg, eg, Pg = got
    # the same FP64 chase on the same (FP32-rounded) projections as nb = 1
    (ref,), _ = _run(Q, d, e, P, [(B, C)], 1)
    assert np.array_equal(dg, ref[1]) and np.array_equal(eg, ref[2])
    # factors: within FP32 rounding of the FP64 oracle and of the register apply
    assert np.max(np.abs(Qg - Qo)) <= 2e-5 and np.max(np.abs(Pg - Po)) <= 2e-5
    assert np.max(np.abs(Qg - ref[0])) <= 2e-5 and np.max(np.abs(Pg - ref[3])) <= 2e-5
    for X in (Qg, Pg):
        assert np.linalg.norm(X.T @ X - np.eye(X.shape[0]), 2) <= 1e-5


def _check_invariants(Q, d, e, P, ups, got, res_tol):
    """Residual against A+ accumulated in FP64, every singular value against
    LAPACK's, and orthogonality of both factors."""
    m, n = Q.shape[0], P.shape[0]
    Qg, dg, eg, Pg = got
    A = Q @ O.bidiag_dense(d, e, m) @ P.T
    for B, C in ups:
        A += B @ C.T
    R = Qg @ O.bidiag_dense(dg, eg, m) @ Pg.T
    assert np.linalg.norm(A - R) / np.linalg.norm(A) <= res_tol
    s_ref = np.linalg.svd(A, compute_uv=False)
    s_got = np.linalg.svd(O.bidiag_dense(dg, eg, m), compute_uv=False)
    assert np.max(np.abs(s_ref - s_got)) <= 1e-5 * s_ref[0]
    for X in (Qg, Pg):
        assert np.linalg.norm(X.T @ X - np.eye(X.shape[0]), 2) <= 1e-5


@pytest.mark.parametrize("nb", [64, 128])
def test_stream_keeps_the_mixed_tolerances(nb):
    """Twelve rank-1 updates and one rank-3 update (the rank-r pipeline) with
    the default re-orthogonalization cadence: residual against A+ accumulated
    in FP64, singular values against LAPACK's, orthogonality."""
    m, n = 600, 450
    Q, d, e, P = I.factorization(m, n, config=0, which=8)
    ups = [I.dense_update(m, n, h, config=0) for h in range(12)] + [I.dense_update(m, n, 99, config=0, r=3)]
    outs, st = _run(Q, d, e, P, ups, nb)
    # FP32 rounding budget of 15 rank-1 columns at this size (the register
    # apply leaves about 6e-6 here)
    _check_invariants(Q, d, e, P, ups, outs[-1], 3e-5)


@pytest.mark.parametrize("nb", [64, 128])
def test_overlapped_form_with_the_blocked_apply(nb):
    m = n = 512
    Q, d, e, P = I.factorization(m, n, config=1, which=2)
    ups = [I.recommender_update(m, n, h, config=1) for h in range(8)]
    a, st = _run(Q, d, e, P, ups, nb, overlap=True)
    assert st["apply_variant"] == [nb, nb]
    _check_invariants(Q, d, e, P, ups, a[-1], 3e-5)


def test_library_choice_of_the_apply():
    """With nb = 0 the mixed form takes the blocked apply (order 128) for
    factors of order >= 1024, by rule rather than by timing, so that every
    path of a shape rounds alike; below that the autotuner picks among the
    FP32 variants, which all round alike: the tuned result equals the one of
    the chosen variant asked for explicitly, bit for bit."""
    m = n = 1056  # (orders no other test uses: the tuner's choices are cached per order)
    Q, d, e, P = I.factorization(m, n, config=1, which=3)
    ups = [I.recommender_update(m, n, h, config=1) for h in range(3)]
    outs, st = _run(Q, d, e, P, ups, 0)
    assert st["apply_variant"] == [128, 128] and st["tunings"] == 0
    Qg, dg, eg, Pg = outs[-1]
    for X in (Qg, Pg):
        assert np.linalg.norm(X.T @ X - np.eye(X.shape[0]), 2) <= 1e-5
    m = n = 656
    Q, d, e, P = I.factorization(m, n, config=1, which=4)
    ups = [I.recommender_update(m, n, h, config=1) for h in range(3)]
    outs, st = _run(Q, d, e, P, ups, 0)
    assert st["tunings"] >= 1
    v = st["apply_variant"]
    assert all(1 <= x <= 5 for x in v), v
    if v[0] == v[1]:
        ref, _ = _run(Q, d, e, P, ups, v[0])
        for a, b in zip(outs[-1], ref[-1]):
            assert np.array_equal(a, b)
