"""The allocation-free entry point (bdu_update_rank1_noalloc).

It serves callers that cannot allocate device memory: the caller owns every
input and output buffer on the device and the library keeps its
intermediates in one fixed device array.  This file is collected last so
that a run that stops at the first failure has run every other test first.

The entry point's results are compared with the regular handle path
(bdu_create / bdu_update) on the same data, for two calls in a row, with the
tolerance the FP64 parity tests use: exact equality.
"""
import ctypes

import numpy as np
import pytest

from paper_2509_02840_gb300 import bdu, inputs as I


def _fn():
    L = bdu.load()
    f = L.bdu_update_rank1_noalloc
    f.argtypes = [ctypes.c_int64, ctypes.c_int64] + [ctypes.c_void_p] * 7
    f.restype = ctypes.c_int
    return f


def test_noalloc_rejects_sizes_beyond_its_maximum():
    f = _fn()
    # argument checks happen before any device work
    assert f(2000, 100, 1, 1, 1, 1, 1, 1, None) == 1   # m > 1024
    assert f(300, 257, 1, 1, 1, 1, 1, 1, None) == 1    # n > 256
    assert f(10, 20, 1, 1, 1, 1, 1, 1, None) == 1      # m < n
    assert f(10, 5, None, 1, 1, 1, 1, 1, None) == 1    # NULL pointer


@pytest.mark.gpu
@pytest.mark.parametrize("m,n", [(200, 150), (256, 256), (1024, 256), (1024, 100), (300, 1)])
def test_noalloc_matches_handle_path_twice(m, n):
    import torch
    f = _fn()
    Q, d, e, P = I.factorization(m, n, config=0, which=31)
    ups = [I.dense_update(m, n, h, config=0) for h in (41, 42)]
    dev = torch.device("cuda", 0)
    tQ = torch.from_numpy(Q.reshape(-1, order="F").copy()).to(dev)
    tP = torch.from_numpy(P.reshape(-1, order="F").copy()).to(dev)
    td = torch.from_numpy(d.copy()).to(dev)
    te = torch.from_numpy(e.copy()).to(dev) if n > 1 else None  # e may be NULL when n == 1
    stream = torch.cuda.current_stream(dev)
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        for B, C in ups:
            tb = torch.from_numpy(B[:, 0].copy()).to(dev)
            tc = torch.from_numpy(C[:, 0].copy()).to(dev)
            torch.cuda.synchronize()
            code = f(m, n, tQ.data_ptr(), td.data_ptr(), te.data_ptr() if te is not None else None,
                     tP.data_ptr(), tb.data_ptr(), tc.data_ptr(), stream.cuda_stream)
            assert code == 0
            F.update(B, C)
            Qh, dh, eh, Ph = F.read()
            assert np.array_equal(td.cpu().numpy(), dh)
            if te is not None:
                assert np.array_equal(te.cpu().numpy(), eh)
            assert np.array_equal(tQ.cpu().numpy().reshape(m, m, order="F"), Qh)
            assert np.array_equal(tP.cpu().numpy().reshape(n, n, order="F"), Ph)


@pytest.mark.gpu
def test_noalloc_failure_leaves_the_callers_buffers_unchanged():
    """When the chase's watchdog runs out (forced here by failure injection,
    no GPU fault), the call reports BDU_ETIMEOUT and the kernels that would
    write Q, P, d and e skip their work; the next call, without injection,
    gives the handle path's result again."""
    import torch
    f = _fn()
    m, n = 300, 200
    Q, d, e, P = I.factorization(m, n, config=0, which=32)
    B, C = I.dense_update(m, n, 43, config=0)
    dev = torch.device("cuda", 0)
    tQ = torch.from_numpy(Q.reshape(-1, order="F").copy()).to(dev)
    tP = torch.from_numpy(P.reshape(-1, order="F").copy()).to(dev)
    td = torch.from_numpy(d.copy()).to(dev)
    te = torch.from_numpy(e.copy()).to(dev)
    tb = torch.from_numpy(B[:, 0].copy()).to(dev)
    tc = torch.from_numpy(C[:, 0].copy()).to(dev)
    stream = torch.cuda.current_stream(dev)
    torch.cuda.synchronize()
    args = (m, n, tQ.data_ptr(), td.data_ptr(), te.data_ptr(), tP.data_ptr(), tb.data_ptr(), tc.data_ptr(),
            stream.cuda_stream)
    bdu.set_fault_injection(bdu.INJECT_STEP_BUDGET, 5)
    try:
        assert f(*args) == 4  # BDU_ETIMEOUT
    finally:
        bdu.set_fault_injection(bdu.INJECT_NONE)
    assert np.array_equal(tQ.cpu().numpy().reshape(m, m, order="F"), Q)
    assert np.array_equal(tP.cpu().numpy().reshape(n, n, order="F"), P)
    assert np.array_equal(td.cpu().numpy(), d)
    assert np.array_equal(te.cpu().numpy(), e)
    assert f(*args) == 0
    with bdu.Factorization(Q, d, e, P, precision=bdu.FP64) as F:
        F.update(B, C)
        Qh, dh, eh, Ph = F.read()
    assert np.array_equal(td.cpu().numpy(), dh)
    assert np.array_equal(tQ.cpu().numpy().reshape(m, m, order="F"), Qh)
