"""The C-ABI library builds, loads and exports what include/bdu.h declares,
and rejects invalid arguments before touching a GPU (no GPU needed)."""
import ctypes

import numpy as np
import pytest

from paper_2509_02840_gb300 import bdu


@pytest.fixture(scope="module")
def lib():
    return bdu.load()


def test_exports_every_declared_function(lib):
    names = bdu.declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def test_version_and_defaults(lib):
    assert lib.bdu_version() >= 100
    o = bdu.Options()
    lib.bdu_default_options(ctypes.byref(o))
    assert o.precision == bdu.FP64 and o.nb == 0 and o.device == 0
    assert o.reorth_tol == pytest.approx(5e-6) and o.check_every == 10 and o.reorth_every == -1
    assert o.graphs == 1 and o.step_budget == 0 and o.overlap == 0


def _create(lib, m, n, Q, d, e, P):
    h = ctypes.c_void_p()
    dp = lambda a: None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    code = lib.bdu_create(ctypes.byref(h), m, n, dp(Q), dp(d), dp(e), dp(P), None)
    return code, h


def test_create_rejects_bad_arguments_without_a_gpu(lib):
    I4 = np.eye(4); I3 = np.eye(3); d = np.ones(4); e = np.ones(3)
    code, h = _create(lib, 0, 4, I3, d, e, I4)          # m < 1
    assert code == 1 and not h.value
    assert b"m, n >= 1" in lib.bdu_last_error(None)
    code, _ = _create(lib, 4, 0, I4, d, e, I4)          # n < 1
    assert code == 1
    # m < n is held as the transposed problem: its arguments are checked the same way
    code, _ = _create(lib, 3, 4, None, d, e, I4)        # NULL Q
    assert code == 1
    code, _ = _create(lib, 3, 4, I3, d, None, I4)       # NULL e with min(m, n) > 1
    assert code == 1
    bad3 = I3.copy(); bad3[0, 1] = np.nan
    code, _ = _create(lib, 3, 4, bad3, d, e, I4)        # non-finite Q
    assert code == 1 and b"non-finite" in lib.bdu_last_error(None)
    code, _ = _create(lib, 4, 4, None, d, e, I4)        # NULL Q
    assert code == 1
    code, _ = _create(lib, 4, 4, I4, d, None, I4)       # NULL e with n > 1
    assert code == 1
    bad = I4.copy(); bad[1, 2] = np.nan
    code, _ = _create(lib, 4, 4, bad, d, e, I4)         # non-finite
    assert code == 1 and b"non-finite" in lib.bdu_last_error(None)
    dinf = d.copy(); dinf[0] = np.inf
    code, _ = _create(lib, 4, 4, I4, dinf, e, I4)
    assert code == 1


def test_null_handle_calls_are_rejected(lib):
    assert lib.bdu_update(None, None, None, 1) == 1
    assert lib.bdu_sync(None) == 1
    assert lib.bdu_read(None, None, None, None, None) == 1
    lib.bdu_destroy(None)  # accepted
    assert lib.bdu_last_error(None) is not None


def test_thin_create_rejects_bad_arguments_without_a_gpu(lib):
    dp = lambda a: None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    m, n = 12, 9
    Q1 = np.zeros((m, 3), order="F"); P1 = np.zeros((n, 3), order="F")
    d = np.ones(3); e = np.ones(2)

    def create(m_, n_, k_, q, dd, ee, p, precision=None):
        h = ctypes.c_void_p()
        o = None
        if precision is not None:
            o = bdu.Options()
            lib.bdu_default_options(ctypes.byref(o))
            o.precision = precision
        code = lib.bdu_thin_create(ctypes.byref(h), m_, n_, k_, dp(q), dp(dd), dp(ee), dp(p),
                                   None if o is None else ctypes.byref(o))
        return code, h

    for k in (0, 9, 12):  # k must satisfy 1 <= k < min(m, n)
        code, h = create(m, n, k, Q1, d, e, P1)
        assert code == 1 and not h.value
    assert b"min(m, n)" in lib.bdu_thin_last_error(None)
    assert create(m, n, 3, None, d, e, P1)[0] == 1          # NULL Q1
    assert create(m, n, 3, Q1, d, None, P1)[0] == 1         # NULL e with k > 1
    assert create(m, n, 3, Q1, d, e, P1, precision=5)[0] == 1
    bad = Q1.copy(); bad[0, 0] = np.inf
    assert create(m, n, 3, bad, d, e, P1)[0] == 1
    assert b"non-finite" in lib.bdu_thin_last_error(None)


def test_thin_null_handle_calls_are_rejected(lib):
    assert lib.bdu_thin_update(None, None, None, None, None) == 1
    assert lib.bdu_thin_read(None, None, None, None, None) == 1
    assert lib.bdu_thin_stats(None, None, None, None) == 1
    lib.bdu_thin_destroy(None)  # accepted


def test_fault_injection_arguments_without_a_gpu(lib):
    """bdu_set_fault_injection validates its site and value; the setting is
    process-wide and switched off again at the end."""
    assert lib.bdu_set_fault_injection(9, 1) == 1       # unknown site
    assert lib.bdu_set_fault_injection(-1, 1) == 1
    assert lib.bdu_set_fault_injection(bdu.INJECT_APPLY_STALL, 0) == 1  # value < 1
    assert lib.bdu_set_fault_injection(bdu.INJECT_STEP_BUDGET, 7) == 0
    assert lib.bdu_set_fault_injection(bdu.INJECT_NONE, 0) == 0
    with pytest.raises(bdu.BduError):
        bdu.set_fault_injection(bdu.INJECT_ROTVEC_STALL, 0)


def test_bhu_sizes_and_argument_checks_without_a_gpu(lib):
    """bdu_bhu_sizes gives Algorithm 1's reflector counts (Sec. 3.3: n-1 left
    and n-2 right for m = n, one more left for m > n; fewer for a partial run)
    and validates its sizes; the BHU entry points reject bad arguments before
    touching the device."""
    import ctypes
    kl, kr, wb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    for (m, n, t, el, er) in ((6, 6, 6, 5, 4), (9, 6, 6, 6, 4), (9, 6, 2, 2, 2), (5, 1, 1, 1, 0), (2, 2, 2, 1, 0)):
        assert lib.bdu_bhu_sizes(m, n, t, ctypes.byref(kl), ctypes.byref(kr), ctypes.byref(wb)) == 0
        assert (kl.value, kr.value) == (el, er) and wb.value > 0
    assert lib.bdu_bhu_sizes(5, 6, 5, None, None, None) == 1      # m < n
    assert lib.bdu_bhu_sizes(6, 6, 7, None, None, None) == 1      # steps > n
    assert lib.bdu_bhu_sizes(6, 0, 0, None, None, None) == 1      # n < 1
    assert lib.bdu_bhu_factor(5, 6, 1, 5, *([None] * 12)) == 1
    assert lib.bdu_bhu_factor(6, 6, 1, 6, *([None] * 12)) == 1    # NULL pointers
    assert lib.bdu_bhu_factor(6, 6, 9, 6, *([None] * 12)) == 1    # r > BDU_BHU_MAX_RANK
    assert lib.bdu_bhu_factor(6, 6, 0, 6, *([None] * 12)) == 1
    assert lib.bdu_update_bhu(None, None, None, 1) == 1
    assert lib.bdu_update_bhu_dev(None, None, None, 1) == 1
    assert lib.bdu_set_fault_injection(bdu.INJECT_BHU_STALL, 0) == 1
    assert lib.bdu_set_fault_injection(bdu.INJECT_BHU_STALL, 5) == 0
    assert lib.bdu_set_fault_injection(bdu.INJECT_NONE, 0) == 0


def test_tri_sizes_and_argument_checks_without_a_gpu(lib):
    """bdu_tri_sizes gives the symmetric variant's reflector count (n-2 for a
    complete run) and validates its sizes; the entry points reject bad
    arguments before touching the device."""
    import ctypes
    k, wb, ub = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    for (n, t, ek) in ((6, 6, 4), (6, 2, 2), (2, 2, 0), (1, 1, 0)):
        assert lib.bdu_tri_sizes(n, t, ctypes.byref(k), ctypes.byref(wb), ctypes.byref(ub)) == 0
        assert k.value == ek and wb.value > 0 and ub.value > wb.value
    assert lib.bdu_tri_sizes(0, 0, None, None, None) == 1
    assert lib.bdu_tri_sizes(5, 6, None, None, None) == 1
    assert lib.bdu_tri_factor(6, 6, None, None, 1.0, None, None, None, None, None, None, None) == 1
    assert lib.bdu_tri_factor(6, 7, None, None, 1.0, None, None, None, None, None, None, None) == 1
    assert lib.bdu_tri_update_dev(6, None, None, None, 1.0, None, None, None) == 1
