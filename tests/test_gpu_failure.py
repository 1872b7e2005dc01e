"""Failure detection without a GPU fault: the chase's watchdog (a bound on its
synchronous steps per column, bdu_options.step_budget) runs out, the kernel
stops and records the fact in the handle's device status word, and the next
synchronizing call reports BDU_ETIMEOUT.  The handle is then poisoned (later
updates answer BDU_EPOISONED, reads and destroy still work), and the CUDA
context stays usable: a fresh handle on the same device updates correctly."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2509_02840_gb300 import bdu, inputs as I

pytestmark = pytest.mark.gpu

ETIMEOUT, EPOISONED = 4, 7


def _healthy_update_still_works(m, n):
    Q, d, e, P = I.factorization(m, n, config=0, which=3)
    B, C = I.dense_update(m, n, 0, config=0)
    with bdu.Factorization(Q, d, e, P) as F:
        F.update(B, C)
        got = F.read()
    want = O.update(Q, d, e, P, B, C)[:4]
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("m,n,precision,overlap", [(64, 48, bdu.FP64, False), (600, 560, bdu.FP64, False),
                                                   (600, 560, bdu.MIXED, True)])
def test_step_budget_expiry_is_reported_and_poisons(m, n, precision, overlap):
    Q, d, e, P = I.factorization(m, n, config=0, which=1)
    F = bdu.Factorization(Q, d, e, P, precision=precision, overlap=overlap, step_budget=10)
    try:
        with pytest.raises(bdu.BduError) as info:
            F.update(*I.dense_update(m, n, 0, config=0))
            F.sync()
        assert info.value.code == ETIMEOUT and "step budget" in str(info.value)
        with pytest.raises(bdu.BduError) as again:
            F.update(*I.dense_update(m, n, 1, config=0))
        assert again.value.code == EPOISONED
        Qr, dr, er, Pr = F.read()  # still answered (the state is not trustworthy)
        assert Qr.shape == (m, m) and dr.shape == (n,)
    finally:
        F.close()
    _healthy_update_still_works(m, n)


def test_step_budget_expiry_in_a_batch():
    m, n = 200, 150
    Q, d, e, P = I.factorization(m, n, config=0, which=2)
    good = bdu.Factorization(Q, d, e, P)
    bad = bdu.Factorization(Q, d, e, P, step_budget=5)
    try:
        B, C = I.dense_update(m, n, 0, config=0)
        tb = torch.from_numpy(B.reshape(-1, order="F").copy()).cuda()
        tc = torch.from_numpy(C.reshape(-1, order="F").copy()).cuda()
        torch.cuda.synchronize()
        bdu.update_batch([good, bad], [tb.data_ptr()] * 2, [tc.data_ptr()] * 2, [1, 1])
        with pytest.raises(bdu.BduError) as info:
            bad.sync()
        assert info.value.code == ETIMEOUT
        # the other item of the batch is unaffected
        got = good.read()
        want = O.update(Q, d, e, P, B, C)[:4]
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
    finally:
        good.close()
        bad.close()
    _healthy_update_still_works(m, n)


def test_negative_budget_is_rejected():
    Q, d, e, P = I.factorization(20, 10, config=0, which=1)
    with pytest.raises(bdu.BduError):
        bdu.Factorization(Q, d, e, P, step_budget=-1)


@pytest.mark.parametrize("site,rank,what", [(bdu.INJECT_APPLY_STALL, 1, "rotation apply"),
                                            (bdu.INJECT_ROTVEC_STALL, 2, "vector rotation")])
def test_bounded_waits_expire_and_poison(site, rank, what):
    """The FP32 register-resident apply's and the vector rotation's waits on
    their record rings: failure injection keeps the producer warp from
    starting any copy and shortens the bound, so the compute threads' waits run
    out with nothing in flight; the kernel records the expiry in the status
    word and returns.  (nb=1 fixes the register layout, so no autotuning run
    meets the injection; rank 2 sends the later column's projections through
    the vector rotation.)"""
    m, n = 600, 560
    Q, d, e, P = I.factorization(m, n, config=0, which=4)
    B, C = I.dense_update(m, n, 0, config=0, r=rank)
    F = bdu.Factorization(Q, d, e, P, precision=bdu.MIXED, nb=1, graphs=False)
    try:
        bdu.set_fault_injection(site, 2000)
        try:
            with pytest.raises(bdu.BduError) as info:
                F.update(B, C)
                F.sync()
        finally:
            bdu.set_fault_injection(bdu.INJECT_NONE)
        assert info.value.code == ETIMEOUT and what in str(info.value)
        with pytest.raises(bdu.BduError) as again:
            F.update(B, C)
        assert again.value.code == EPOISONED
    finally:
        F.close()
    _healthy_update_still_works(m, n)


def test_bhu_grid_barrier_expires_and_poisons():
    """BHU's grid barriers are bounded waits: failure injection makes the first
    block leave before it arrives, so every other block's first wait runs out
    (after 2000 polls); the kernel records the expiry and all blocks return."""
    m, n = 96, 80
    Q, d, e, P = I.factorization(m, n, config=0, which=5)
    B, C = I.dense_update(m, n, 0, config=0, r=1)
    F = bdu.Factorization(Q, d, e, P, precision=bdu.FP64)
    try:
        bdu.set_fault_injection(bdu.INJECT_BHU_STALL, 2000)
        try:
            with pytest.raises(bdu.BduError) as info:
                F.update_bhu(B, C)
                F.sync()
        finally:
            bdu.set_fault_injection(bdu.INJECT_NONE)
        assert info.value.code == ETIMEOUT and "grid barrier" in str(info.value)
        with pytest.raises(bdu.BduError) as again:
            F.update_bhu(B, C)
        assert again.value.code == EPOISONED
    finally:
        F.close()
    # a fresh handle runs BHU normally afterwards
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as G:
        G.update_bhu(B, C)
        G.sync()
    _healthy_update_still_works(m, n)
