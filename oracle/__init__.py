"""Plain FP64 CPU oracle for the Givens bidiagonal update (BGU).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library.  The arithmetic lives in
``bgu_oracle.c`` (Sec. 3.4, Algorithm 2, in the schedule documented at the top
of that file); this module only marshals numpy arrays through ctypes.

Functions
---------
rot(f, g)                       rotation generator (Eqs. giv, giv1)
update(Q, d, e, P, B, C)        full update, Eqs. rk1 / bidiagsubproblem / bidiagplus
update_lower(Q, d, e, P, B, C)  the same for m < n (lower bidiagonal, by transposition)
generate(m, n, d, e, U, V)      the reduction only: rotation lists + new (d, e)
apply_rows(X, rows, rotlist)    X(rows, :) <- X(rows, :) * prod(rotations)
jacobi_sv(X)                    one-sided Jacobi singular values (tiny inputs)
truncated_bd(Q, d, e, P, r)     truncated bidiagonal approximation, Eqs. trBD / errtrBD
singular_values(d, e)           singular values of the bidiagonal (library SVD)
thin_update(Q1, d, e, P1, b, c) rank-k subspace tracking step, Eqs. lrup - bdlrup
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

PHASES = ("spike", "phase1", "phase2", "phase3")


class _RotList(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int64),
        ("cap", ctypes.c_int64),
        ("c", ctypes.POINTER(ctypes.c_double)),
        ("s", ctypes.POINTER(ctypes.c_double)),
        ("a", ctypes.POINTER(ctypes.c_int32)),
        ("phase", ctypes.POINTER(ctypes.c_int8)),
    ]


class _Counts(ctypes.Structure):
    _fields_ = [
        ("left", ctypes.c_int64 * 4),
        ("right", ctypes.c_int64 * 4),
        ("band_violations", ctypes.c_int64),
        ("zero_violations", ctypes.c_int64),
    ]


class OracleError(RuntimeError):
    pass


_ERR = {1: "invalid argument", 2: "out of memory", 3: "band invariant violated",
        4: "an entry the schedule must zero is not exactly zero"}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        i32p = ctypes.POINTER(ctypes.c_int32)
        L.orc_rot.argtypes = [ctypes.c_double, ctypes.c_double, dp, dp, dp]
        L.orc_rot.restype = ctypes.c_int
        L.orc_update.argtypes = [ctypes.c_int] * 3 + [dp, ctypes.c_int, dp, dp, dp, ctypes.c_int,
                                                      dp, ctypes.c_int, dp, ctypes.c_int,
                                                      ctypes.POINTER(_Counts)]
        L.orc_update.restype = ctypes.c_int
        L.orc_generate.argtypes = [ctypes.c_int] * 3 + [dp, dp, dp, dp, ctypes.POINTER(_RotList),
                                                        ctypes.POINTER(_RotList), ctypes.POINTER(_Counts)]
        L.orc_generate.restype = ctypes.c_int
        L.orc_project.argtypes = [ctypes.c_int] * 3 + [dp, ctypes.c_int, dp, ctypes.c_int, dp,
                                                       ctypes.c_int, dp, ctypes.c_int, dp, dp]
        L.orc_project.restype = None
        L.orc_apply_rows.argtypes = [dp, ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int,
                                     ctypes.POINTER(_RotList)]
        L.orc_apply_rows.restype = None
        L.orc_free_list.argtypes = [ctypes.POINTER(_RotList)]
        L.orc_free_list.restype = None
        L.orc_num_threads.argtypes = []
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_jacobi_sv.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int]
        L.orc_jacobi_sv.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.array(a, dtype=np.float64, order="F", copy=True)


def num_threads() -> int:
    return lib().orc_num_threads()


def rot(f: float, g: float):
    """Returns (applied, c, s, r) for [c s; -s c][f; g] = [r; 0]."""
    c, s, r = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    ok = lib().orc_rot(float(f), float(g), ctypes.byref(c), ctypes.byref(s), ctypes.byref(r))
    return bool(ok), c.value, s.value, r.value


def _counts_dict(cnt):
    return {
        "left": {PHASES[i]: int(cnt.left[i]) for i in range(4)},
        "right": {PHASES[i]: int(cnt.right[i]) for i in range(4)},
        "total": int(sum(cnt.left) + sum(cnt.right)),
        "band_violations": int(cnt.band_violations),
        "zero_violations": int(cnt.zero_violations),
    }


def update(Q, d, e, P, B, C, check=True):
    """Returns (Q+, d+, e+, P+, counts) for A + B C^T with A = Q diag-band(d, e) P^T."""
    Q = _f64(Q); P = _f64(P); d = _f64(d); e = _f64(e)
    m, n = Q.shape[0], P.shape[0]
    B = _f64(np.asarray(B, dtype=np.float64).reshape(m, -1))
    C = _f64(np.asarray(C, dtype=np.float64).reshape(n, -1))
    r = B.shape[1]
    if e.size == 0:
        e = np.zeros(1)
    cnt = _Counts()
    rc = lib().orc_update(m, n, r, _dp(Q), m, _dp(d), _dp(e), _dp(P), n, _dp(B), m, _dp(C), n,
                          ctypes.byref(cnt))
    if rc != 0 and check:
        raise OracleError(_ERR.get(rc, str(rc)) + f" ({_counts_dict(cnt)})")
    return Q, d, e[: n - 1], P, _counts_dict(cnt)


def update_lower(Q, d, e, P, B, C, check=True):
    """m < n: A = Q L P^T with L lower bidiagonal (L(i,i) = d_i, L(i+1,i) = e_i,
    m x n, columns m+1..n zero).  Sec. 1 states the factorization with an upper
    bidiagonal and Algorithm 2 for m >= n; the m < n case is read as the
    transposed problem A^T = P L^T Q^T (L^T upper bidiagonal, n x m), updated
    with A^T + C B^T by the m >= n update.  Returns (Q+, d+, e+, P+, counts)
    with counts' "left" the rotations on Q (the transposed problem's right
    rotations) and "right" those on P."""
    Q = _f64(Q); P = _f64(P)
    m, n = Q.shape[0], P.shape[0]
    if m >= n:
        raise ValueError("update_lower is for m < n")
    B = np.asarray(B, dtype=np.float64).reshape(m, -1)
    C = np.asarray(C, dtype=np.float64).reshape(n, -1)
    P2, d2, e2, Q2, cnt = update(P, d, e, Q, C, B, check)
    cnt = dict(cnt)
    cnt["left"], cnt["right"] = cnt["right"], cnt["left"]
    return Q2, d2, e2, P2, cnt


def lower_bidiag_dense(d, e, m, n):
    """The m x n lower bidiagonal with diagonal d and subdiagonal e (m < n)."""
    L = np.zeros((m, n))
    k = len(d)
    L[np.arange(k), np.arange(k)] = d
    if k > 1:
        L[np.arange(1, k), np.arange(k - 1)] = e[: k - 1]
    return L


class RotationList:
    """Rotations in generation order: pair (a, a+1) with 1-based a."""

    def __init__(self, raw: _RotList):
        k = raw.count
        if k:
            self.c = np.ctypeslib.as_array(raw.c, shape=(k,)).copy()
            self.s = np.ctypeslib.as_array(raw.s, shape=(k,)).copy()
            self.a = np.ctypeslib.as_array(raw.a, shape=(k,)).copy()
            self.phase = np.ctypeslib.as_array(raw.phase, shape=(k,)).copy()
        else:
            self.c = np.zeros(0); self.s = np.zeros(0)
            self.a = np.zeros(0, np.int32); self.phase = np.zeros(0, np.int8)

    def __len__(self):
        return len(self.c)

    def _raw(self):
        raw = _RotList()
        raw.count = len(self)
        raw.cap = len(self)
        self._keep = (np.ascontiguousarray(self.c), np.ascontiguousarray(self.s),
                      np.ascontiguousarray(self.a, dtype=np.int32),
                      np.ascontiguousarray(self.phase, dtype=np.int8))
        raw.c = _dp(self._keep[0]); raw.s = _dp(self._keep[1])
        raw.a = self._keep[2].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        raw.phase = self._keep[3].ctypes.data_as(ctypes.POINTER(ctypes.c_int8))
        return raw


def project(Q, P, B, C):
    """U = Q^T B, V = P^T C with the oracle's plain loops."""
    Q = _f64(Q); P = _f64(P)
    m, n = Q.shape[0], P.shape[0]
    B = _f64(np.asarray(B, dtype=np.float64).reshape(m, -1))
    C = _f64(np.asarray(C, dtype=np.float64).reshape(n, -1))
    r = B.shape[1]
    U = np.zeros((m, r), order="F"); V = np.zeros((n, r), order="F")
    lib().orc_project(m, n, r, _dp(Q), m, _dp(P), n, _dp(B), m, _dp(C), n, _dp(U), _dp(V))
    return U, V


def generate(m, n, d, e, U, V, check=True):
    """The reduction alone: returns (d+, e+, left RotationList, right RotationList, counts)."""
    d = _f64(d); e = _f64(e) if n > 1 else np.zeros(1)
    U = _f64(np.asarray(U, dtype=np.float64).reshape(m, -1))
    V = _f64(np.asarray(V, dtype=np.float64).reshape(n, -1))
    r = U.shape[1]
    L, R, cnt = _RotList(), _RotList(), _Counts()
    rc = lib().orc_generate(m, n, r, _dp(d), _dp(e), _dp(U), _dp(V), ctypes.byref(L),
                            ctypes.byref(R), ctypes.byref(cnt))
    try:
        if rc != 0 and check:
            raise OracleError(_ERR.get(rc, str(rc)) + f" ({_counts_dict(cnt)})")
        return d, e[: n - 1], RotationList(L), RotationList(R), _counts_dict(cnt)
    finally:
        lib().orc_free_list(ctypes.byref(L))
        lib().orc_free_list(ctypes.byref(R))


def apply_rows(X, rows, rotlist: RotationList):
    """Returns a copy of X with the rotations applied to the given (0-based) rows."""
    X = _f64(X)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    raw = rotlist._raw()
    lib().orc_apply_rows(_dp(X), X.shape[0], X.shape[1],
                         rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(rows),
                         ctypes.byref(raw))
    return X


def jacobi_sv(X, max_sweeps=60):
    """Singular values of a small matrix by one-sided (Hestenes) Jacobi, sorted descending."""
    X = _f64(X)
    rows, cols = X.shape
    if rows < cols:
        X = _f64(X.T)
        rows, cols = cols, rows
    sv = np.zeros(cols)
    sweeps = lib().orc_jacobi_sv(_dp(X), rows, cols, _dp(sv), max_sweeps)
    if sweeps < 0:
        raise OracleError("Jacobi did not converge")
    return np.sort(sv)[::-1]


def bidiag_dense(d, e, rows=None):
    """The bidiagonal as a dense (rows x n) matrix; rows defaults to n."""
    n = len(d)
    rows = n if rows is None else rows
    M = np.zeros((rows, n))
    M[np.arange(n), np.arange(n)] = d
    if n > 1:
        M[np.arange(n - 1), np.arange(1, n)] = e
    return M


def truncated_bd(Q, d, e, P, r):
    """Truncated bidiagonal approximation (Sec. 2, Eq. trBD) and its error
    (Eq. errtrBD), written out from their definitions.

    With alpha_i = d_i, beta_i = e_i (beta_0 = 0), the rank-r approximation keeps
    the r indices i with the largest alpha_i^2 + beta_{i-1}^2 (ties: the lower i
    first) and is A_r = L R^T with L(:, k) = alpha_i q_i + beta_{i-1} q_{i-1},
    R(:, k) = p_i, the kept indices in increasing order.  The error
    ||A - A_r||_F^2 is the sum of alpha_i^2 + beta_{i-1}^2 over the others,
    added in increasing i.  Weights, products and sums are separately rounded
    FP64 operations.  Returns (L, R, idx (1-based i), err2).
    """
    Q = _f64(Q); P = _f64(P)
    d = np.asarray(d, dtype=np.float64); e = np.asarray(e, dtype=np.float64)
    n = len(d)
    if not 0 <= r <= n:
        raise ValueError("0 <= r <= n required")
    w = np.empty(n)
    for i in range(n):
        a2 = d[i] * d[i]
        w[i] = a2 if i == 0 else a2 + e[i - 1] * e[i - 1]
    order = sorted(range(n), key=lambda i: (-w[i], i))
    keep = sorted(order[:r])
    kept = set(keep)
    err2 = 0.0
    for i in range(n):
        if i not in kept:
            err2 = err2 + w[i]
    m = Q.shape[0]
    L = np.zeros((m, r), order="F")
    R = np.zeros((P.shape[0], r), order="F")
    for k, i in enumerate(keep):
        L[:, k] = d[i] * Q[:, i] if i == 0 else d[i] * Q[:, i] + e[i - 1] * Q[:, i - 1]
        R[:, k] = P[:, i]
    return L, R, np.array([i + 1 for i in keep], dtype=np.int64), err2


def singular_values(d, e):
    """Singular values of the upper bidiagonal (d, e), descending: the plain
    definition, evaluated by a library SVD of the dense n x n matrix."""
    return np.linalg.svd(bidiag_dense(d, e), compute_uv=False)


# ---------------------------------------------------------------------------
# Thin (rank-k) tracking, Sec. 4 (Eqs. lrup, defup, qrlr, equivlrup, bdlrup)
# ---------------------------------------------------------------------------
THIN_TAU = 2.0 ** -40          # b is taken to lie in span(Q1) when ||b_perp|| <= THIN_TAU ||b||
GOLDEN = 0.6180339887498949    # the FP64 value nearest (sqrt(5) - 1) / 2


def fill_vector(m):
    """The fixed direction used when b lies in span(Q1): z_i = frac(i * GOLDEN) - 0.5,
    i = 0..m-1, each step one IEEE operation."""
    t = np.arange(m, dtype=np.float64) * GOLDEN
    return t - np.floor(t) - 0.5


def _cgs2(X, b):
    """Classical Gram-Schmidt against the columns of X, run twice: returns
    (X^T b accumulated over both passes, the remainder)."""
    h1 = X.T @ b
    r = b - X @ h1
    h2 = X.T @ r
    r = r - X @ h2
    return h1 + h2, r


def _augment(X, b):
    """Eq. defup and Eq. qrlr: (projection, delta, new unit column)."""
    bh, r = _cgs2(X, b)
    delta = float(np.linalg.norm(r))
    if delta > THIN_TAU * float(np.linalg.norm(b)):
        return bh, delta, r / delta
    _, rz = _cgs2(X, fill_vector(X.shape[0]))
    return bh, 0.0, rz / np.linalg.norm(rz)


def thin_update(Q1, d, e, P1, b, c, full=False):
    """One step of rank-k tracking (Sec. 4): A+ = Q1 B P1^T + b c^T with Q1 (m x k),
    P1 (n x k) orthonormal and B = diag-band(d, e) k x k upper bidiagonal.

    b+ = Q1^T b, b_perp = b - Q1 b+, delta = ||b_perp|| (Eq. defup; the
    projection is taken twice, classical Gram-Schmidt with one reorthogonalization);
    Q1bar = [Q1, b_perp / delta] (Eq. qrlr), likewise for c.  The middle matrix
    [B 0; 0 0] + [b+; delta][c+; gamma]^T (Eq. equivlrup) is reduced by the update
    of this module (Algorithm 2 on the (k+1)-order problem with identity factors),
    giving Q2, Bbar+, P2 and A+ = (Q1bar Q2) Bbar+ (P1bar P2)^T (Eq. bdlrup).  The
    index i with the smallest column norm alpha_i^2 + beta_{i-1}^2 of Bbar+ (ties:
    the last such i) is removed with its row and column; the kept superdiagonal
    entry between the neighbours of i is zero.  When ||b_perp|| <= THIN_TAU ||b||
    (b in span(Q1)), delta = 0 and the new column is the fixed vector
    orthogonalized against Q1 the same way (it then carries a zero row of the
    middle matrix).

    Returns (Q1+, d+, e+, P1+, i (0-based removed index), err2 = ||A+ - Q1+ B+ P1+^T||_F^2
    = alpha_i^2 + beta_{i-1}^2 + beta_i^2); with full=True also the untruncated
    (Q1bar Q2, dbar, ebar, P1bar P2)."""
    Q1 = np.asarray(Q1, dtype=np.float64); P1 = np.asarray(P1, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64).ravel(); e = np.asarray(e, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel(); c = np.asarray(c, dtype=np.float64).ravel()
    k = Q1.shape[1]
    if k < 1 or P1.shape[1] != k or len(d) != k or len(e) != k - 1:
        raise ValueError("Q1 m x k, P1 n x k, d (k), e (k-1) with k >= 1 required")
    bh, delta, qa = _augment(Q1, b)
    ch, gamma, pa = _augment(P1, c)
    Qb = np.column_stack([Q1, qa])
    Pb = np.column_stack([P1, pa])
    I = np.eye(k + 1)
    Q2, d2, e2, P2, _ = update(I, np.append(d, 0.0), np.append(e, 0.0), I,
                               np.append(bh, delta), np.append(ch, gamma))
    w = d2 * d2
    w[1:] = w[1:] + e2 * e2
    i = int(np.flatnonzero(w == w.min())[-1])
    keep = [j for j in range(k + 1) if j != i]
    Q1n = Qb @ Q2[:, keep]
    P1n = Pb @ P2[:, keep]
    dn = d2[keep]
    en = np.array([e2[keep[t]] if keep[t + 1] == keep[t] + 1 else 0.0 for t in range(k - 1)])
    err2 = d2[i] * d2[i]
    if i > 0:
        err2 = err2 + e2[i - 1] * e2[i - 1]
    if i < k:
        err2 = err2 + e2[i] * e2[i]
    out = (Q1n, dn, en, P1n, i, float(err2))
    if full:
        out = out + ((Qb @ Q2, d2, e2, Pb @ P2),)
    return out
