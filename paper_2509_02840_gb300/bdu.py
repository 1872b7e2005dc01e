"""ctypes binding of libbdu (include/bdu.h): argument marshalling only.

Every step of the update runs in the library's CUDA kernels.  Loading fails
loudly when libbdu.so is missing; there is no other implementation to fall
back to.
"""
import ctypes
import os
import re

import numpy as np

from . import build as _build

FP64, MIXED = 0, 1
STATUS = {0: "BDU_OK", 1: "BDU_EINVAL", 2: "BDU_ENOMEM", 3: "BDU_ECUDA", 4: "BDU_ETIMEOUT",
          5: "BDU_ENOTORTH", 6: "BDU_EBUSY", 7: "BDU_EPOISONED", 8: "BDU_EINTERNAL"}
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bdu.h")


class BduError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("nb", ctypes.c_int), ("reorth_tol", ctypes.c_double),
                ("check_every", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("engine", ctypes.c_int), ("overlap", ctypes.c_int), ("graphs", ctypes.c_int),
                ("step_budget", ctypes.c_int64), ("reorth_every", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("updates", ctypes.c_int64), ("rot_left", ctypes.c_int64 * 4),
                ("rot_right", ctypes.c_int64 * 4), ("chase_steps", ctypes.c_int64),
                ("reorth_q", ctypes.c_int64), ("reorth_p", ctypes.c_int64),
                ("ortho_q", ctypes.c_double), ("ortho_p", ctypes.c_double),
                ("launches", ctypes.c_int64), ("timed_updates", ctypes.c_int64),
                ("ms_project", ctypes.c_double), ("ms_chase", ctypes.c_double),
                ("ms_apply_q", ctypes.c_double), ("ms_apply_p", ctypes.c_double),
                ("apply_launches", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("graph_replays", ctypes.c_int64), ("apply_variant", ctypes.c_int64 * 2),
                ("tunings", ctypes.c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p)

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libbdu.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libbdu.so not found at {_build.LIB}; run paper_2509_02840_gb300.build.build()")
    L = ctypes.CDLL(_build.LIB)
    dp = ctypes.POINTER(ctypes.c_double)
    H = ctypes.c_void_p
    L.bdu_default_options.argtypes = [ctypes.POINTER(Options)]
    L.bdu_default_options.restype = None
    L.bdu_create.argtypes = [ctypes.POINTER(H), ctypes.c_int64, ctypes.c_int64, dp, dp, dp, dp,
                             ctypes.POINTER(Options)]
    L.bdu_create.restype = ctypes.c_int
    L.bdu_update.argtypes = [H, dp, dp, ctypes.c_int64]
    L.bdu_update.restype = ctypes.c_int
    L.bdu_update_dev.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
    L.bdu_update_dev.restype = ctypes.c_int
    L.bdu_sync.argtypes = [H]
    L.bdu_sync.restype = ctypes.c_int
    L.bdu_flush.argtypes = [H]
    L.bdu_flush.restype = ctypes.c_int
    L.bdu_read.argtypes = [H, dp, dp, dp, dp]
    L.bdu_read.restype = ctypes.c_int
    L.bdu_read_rotations.argtypes = [H, ctypes.c_int, dp, dp, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    L.bdu_read_rotations.restype = ctypes.c_int
    L.bdu_read_truncated.argtypes = [H, ctypes.c_int64, dp, dp, ctypes.POINTER(ctypes.c_int64), dp]
    L.bdu_read_truncated.restype = ctypes.c_int
    L.bdu_singular_values.argtypes = [H, ctypes.c_int64, dp]
    L.bdu_singular_values.restype = ctypes.c_int
    L.bdu_stats.argtypes = [H, ctypes.POINTER(Stats)]
    L.bdu_stats.restype = ctypes.c_int
    L.bdu_update_batch.argtypes = [ctypes.POINTER(H), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                   ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]
    L.bdu_update_batch.restype = ctypes.c_int
    L.bdu_check_orthogonality.argtypes = [H, dp, dp]
    L.bdu_check_orthogonality.restype = ctypes.c_int
    L.bdu_set_timing.argtypes = [H, ctypes.c_int]
    L.bdu_set_timing.restype = ctypes.c_int
    L.bdu_destroy.argtypes = [H]
    L.bdu_destroy.restype = None
    L.bdu_last_error.argtypes = [H]
    L.bdu_last_error.restype = ctypes.c_char_p
    L.bdu_set_allocator.argtypes = [ALLOC_FN, FREE_FN, ctypes.c_void_p]
    L.bdu_set_allocator.restype = None
    L.bdu_version.argtypes = []
    L.bdu_version.restype = ctypes.c_int
    L.bdu_set_fault_injection.argtypes = [ctypes.c_int, ctypes.c_int64]
    L.bdu_set_fault_injection.restype = ctypes.c_int
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.bdu_thin_create.argtypes = [ctypes.POINTER(H), ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, dp, dp, dp, dp,
                                  ctypes.POINTER(Options)]
    L.bdu_thin_create.restype = ctypes.c_int
    L.bdu_thin_update.argtypes = [H, dp, dp, i64p, dp]
    L.bdu_thin_update.restype = ctypes.c_int
    L.bdu_thin_update_dev.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, i64p, dp]
    L.bdu_thin_update_dev.restype = ctypes.c_int
    L.bdu_thin_read.argtypes = [H, dp, dp, dp, dp]
    L.bdu_thin_read.restype = ctypes.c_int
    L.bdu_thin_stats.argtypes = [H, i64p, i64p, i64p]
    L.bdu_thin_stats.restype = ctypes.c_int
    L.bdu_thin_last_error.argtypes = [H]
    L.bdu_thin_last_error.restype = ctypes.c_char_p
    L.bdu_thin_destroy.argtypes = [H]
    L.bdu_thin_destroy.restype = None
    L.bdu_bhu_sizes.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, i64p, i64p, i64p]
    L.bdu_bhu_sizes.restype = ctypes.c_int
    vp = ctypes.c_void_p
    L.bdu_bhu_factor.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64] + [vp] * 12
    L.bdu_bhu_factor.restype = ctypes.c_int
    L.bdu_tri_sizes.argtypes = [ctypes.c_int64, ctypes.c_int64, i64p, i64p, i64p]
    L.bdu_tri_sizes.restype = ctypes.c_int
    L.bdu_tri_factor.argtypes = [ctypes.c_int64, ctypes.c_int64, vp, vp, ctypes.c_double, vp, vp, vp, vp, vp, vp, vp]
    L.bdu_tri_factor.restype = ctypes.c_int
    L.bdu_tri_update_dev.argtypes = [ctypes.c_int64, vp, vp, vp, ctypes.c_double, vp, vp, vp]
    L.bdu_tri_update_dev.restype = ctypes.c_int
    L.bdu_update_bhu.argtypes = [H, dp, dp, ctypes.c_int64]
    L.bdu_update_bhu.restype = ctypes.c_int
    L.bdu_update_bhu_dev.argtypes = [H, vp, vp, ctypes.c_int64]
    L.bdu_update_bhu_dev.restype = ctypes.c_int
    _lib = L
    return L


INJECT_NONE, INJECT_STEP_BUDGET, INJECT_APPLY_STALL, INJECT_ROTVEC_STALL, INJECT_BHU_STALL = 0, 1, 2, 3, 4


def set_fault_injection(site: int, value: int = 1) -> None:
    """bdu_set_fault_injection: process-wide failure injection for tests of
    the bounded device-side waits (INJECT_NONE switches it off)."""
    code = load().bdu_set_fault_injection(int(site), int(value))
    if code != 0:
        raise BduError(code, "bdu_set_fault_injection: unknown site or value < 1")


def declared_functions(header: str = HEADER):
    """Names of the functions declared in include/bdu.h."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bdu_[a-z_0-9]+)\s*\(", text)) - {"bdu_alloc_fn", "bdu_free_fn"})


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _check(L, h, code):
    if code != 0:
        msg = L.bdu_last_error(h)
        raise BduError(code, msg.decode() if msg else "")


_keep_alloc = []


def set_allocator(alloc=None, free=None):
    """Installs Python callables alloc(bytes, device) -> int and free(ptr, device)
    as the device allocator of handles created afterwards; None restores cudaMalloc."""
    L = load()
    if alloc is None:
        L.bdu_set_allocator(ALLOC_FN(), FREE_FN(), None)
        _keep_alloc.clear()
        return
    fa = ALLOC_FN(lambda nbytes, dev, ctx: alloc(int(nbytes), int(dev)) or None)
    ff = FREE_FN(lambda ptr, dev, ctx: free(int(ptr), int(dev)))
    _keep_alloc[:] = [fa, ff]
    L.bdu_set_allocator(fa, ff, None)


def use_torch_allocator():
    """Routes the library's device memory through PyTorch's caching allocator."""
    import torch

    def alloc(nbytes, dev):
        return int(torch.cuda.caching_allocator_alloc(nbytes, device=dev))

    def free(ptr, dev):
        torch.cuda.caching_allocator_delete(ptr)

    set_allocator(alloc, free)


def bhu_sizes(m: int, n: int, steps: int):
    """bdu_bhu_sizes: (kl, kr, workspace bytes) after `steps` iterations of Algorithm 1."""
    L = load()
    kl, kr, wb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    code = L.bdu_bhu_sizes(int(m), int(n), int(steps), ctypes.byref(kl), ctypes.byref(kr), ctypes.byref(wb))
    if code != 0:
        raise BduError(code, (L.bdu_last_error(None) or b"").decode())
    return kl.value, kr.value, wb.value


BHU_MAX_RANK = 8


def bhu_factor(m: int, n: int, steps: int, d: int, e: int, u: int, v: int, alpha: int, beta: int, Y: int, W: int,
               SL: int, SR: int, workspace: int, stream: int = 0, r: int = 1):
    """bdu_bhu_factor with device pointers (ints; 0 for NULL); u, v hold r
    columns (leading dimensions m and n)."""
    L = load()
    ptrs = [ctypes.c_void_p(p or None) for p in (d, e, u, v, alpha, beta, Y, W, SL, SR, workspace, stream)]
    code = L.bdu_bhu_factor(int(m), int(n), int(r), int(steps), *ptrs)
    if code != 0:
        raise BduError(code, (L.bdu_last_error(None) or b"").decode())


def tri_sizes(n: int, steps: int):
    """bdu_tri_sizes: (k, factor workspace bytes, update workspace bytes)."""
    L = load()
    k, wb, ub = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    code = L.bdu_tri_sizes(int(n), int(steps), ctypes.byref(k), ctypes.byref(wb), ctypes.byref(ub))
    if code != 0:
        raise BduError(code, (L.bdu_last_error(None) or b"").decode())
    return k.value, wb.value, ub.value


def tri_factor(n: int, steps: int, a: int, b: int, rho: float, u: int, alpha: int, beta: int, Y: int, S: int,
               workspace: int, stream: int = 0):
    """bdu_tri_factor with device pointers (ints; 0 for NULL)."""
    L = load()
    v = lambda p: ctypes.c_void_p(p or None)
    code = L.bdu_tri_factor(int(n), int(steps), v(a), v(b), float(rho), v(u), v(alpha), v(beta), v(Y), v(S),
                            v(workspace), v(stream))
    if code != 0:
        raise BduError(code, (L.bdu_last_error(None) or b"").decode())


def tri_update_dev(n: int, Q: int, a: int, b: int, rho: float, c: int, workspace: int, stream: int = 0):
    """bdu_tri_update_dev: A + rho c c^T in place on device buffers."""
    L = load()
    v = lambda p: ctypes.c_void_p(p or None)
    code = L.bdu_tri_update_dev(int(n), v(Q), v(a), v(b), float(rho), v(c), v(workspace), v(stream))
    if code != 0:
        raise BduError(code, (L.bdu_last_error(None) or b"").decode())


def update_batch(factorizations, ptrB, ptrC, ranks, stream=None):
    """Batched update (bdu_update_batch): ptrB[i], ptrC[i] are device pointers
    (FP64, column-major) of factorization i's update of rank ranks[i]."""
    L = load()
    k = len(factorizations)
    hs = (ctypes.c_void_p * k)(*[f._h for f in factorizations])
    bs = (ctypes.c_void_p * k)(*[int(p) for p in ptrB])
    cs = (ctypes.c_void_p * k)(*[int(p) for p in ptrC])
    rs = (ctypes.c_int64 * k)(*[int(r) for r in ranks])
    code = L.bdu_update_batch(hs, k, bs, cs, rs, ctypes.c_void_p(int(stream)) if stream else None)
    if code != 0:
        msg = L.bdu_last_error(hs[0]) if k else L.bdu_last_error(None)
        raise BduError(code, msg.decode() if msg else "")


class Factorization:
    """A = Q diag-band(d, e) P^T resident on the GPU (bdu_create / bdu_update / bdu_read).
    The band is upper bidiagonal for m >= n and lower bidiagonal for m < n;
    d has min(m, n) entries and e one fewer."""

    def __init__(self, Q, d, e, P, precision=FP64, stream=None, device=0, reorth_tol=None,
                 check_every=None, engine=0, overlap=False, graphs=True, nb=0,
                 step_budget=0, reorth_every=None):
        L = load()
        Q = _f64(Q); P = _f64(P); d = _f64(d).ravel(); e = _f64(e).ravel()
        self.m, self.n = Q.shape[0], P.shape[0]
        self.k = min(self.m, self.n)
        if e.size == 0:
            e = np.zeros(1)
        opt = Options()
        L.bdu_default_options(ctypes.byref(opt))
        opt.precision = int(precision)
        opt.device = int(device)
        opt.engine = int(engine)
        opt.overlap = 1 if overlap else 0
        opt.graphs = 1 if graphs else 0
        opt.nb = int(nb)
        opt.step_budget = int(step_budget)
        if reorth_every is not None:
            opt.reorth_every = int(reorth_every)
        if reorth_tol is not None:
            opt.reorth_tol = float(reorth_tol)
        if check_every is not None:
            opt.check_every = int(check_every)
        if stream is not None:
            opt.cuda_stream = ctypes.c_void_p(int(stream))
        h = ctypes.c_void_p()
        code = L.bdu_create(ctypes.byref(h), self.m, self.n, _dp(Q), _dp(d), _dp(e), _dp(P), ctypes.byref(opt))
        if code != 0:
            raise BduError(code, L.bdu_last_error(None).decode())
        self._h = h
        self._L = L
        self.precision = precision

    def close(self):
        if getattr(self, "_h", None):
            self._L.bdu_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def update(self, B, C):
        B = _f64(np.asarray(B, dtype=np.float64).reshape(self.m, -1))
        C = _f64(np.asarray(C, dtype=np.float64).reshape(self.n, -1))
        if B.shape[1] != C.shape[1]:
            raise ValueError("B and C need the same number of columns")
        _check(self._L, self._h, self._L.bdu_update(self._h, _dp(B), _dp(C), B.shape[1]))

    def update_dev(self, ptrB: int, ptrC: int, r: int):
        """B, C as device pointers (FP64, column-major, leading dimensions m and n)."""
        _check(self._L, self._h, self._L.bdu_update_dev(self._h, ctypes.c_void_p(ptrB), ctypes.c_void_p(ptrC), int(r)))

    def update_bhu(self, B, C):
        """The update by BHU (bdu_update_bhu; FP64 handles)."""
        B = _f64(np.asarray(B, dtype=np.float64).reshape(self.m, -1))
        C = _f64(np.asarray(C, dtype=np.float64).reshape(self.n, -1))
        if B.shape[1] != C.shape[1]:
            raise ValueError("B and C need the same number of columns")
        _check(self._L, self._h, self._L.bdu_update_bhu(self._h, _dp(B), _dp(C), B.shape[1]))

    def update_bhu_dev(self, ptrB: int, ptrC: int, r: int):
        """bdu_update_bhu_dev: B, C as device pointers."""
        _check(self._L, self._h, self._L.bdu_update_bhu_dev(self._h, ctypes.c_void_p(ptrB), ctypes.c_void_p(ptrC),
                                                            int(r)))

    def sync(self):
        _check(self._L, self._h, self._L.bdu_sync(self._h))

    def flush(self):
        """Enqueues the deferred application of the overlapped form (bdu_flush)."""
        _check(self._L, self._h, self._L.bdu_flush(self._h))

    def read(self):
        m, n, k = self.m, self.n, self.k
        Q = np.zeros((m, m), order="F"); P = np.zeros((n, n), order="F")
        d = np.zeros(k); e = np.zeros(max(k - 1, 1))
        _check(self._L, self._h, self._L.bdu_read(self._h, _dp(Q), _dp(d), _dp(e), _dp(P)))
        return Q, d, e[: k - 1], P

    def read_bidiagonal(self):
        k = self.k
        d = np.zeros(k); e = np.zeros(max(k - 1, 1))
        _check(self._L, self._h, self._L.bdu_read(self._h, None, _dp(d), _dp(e), None))
        return d, e[: k - 1]

    def read_rotations(self, side):
        cnt = ctypes.c_int64()
        _check(self._L, self._h, self._L.bdu_read_rotations(self._h, side, None, None, None, 0, ctypes.byref(cnt)))
        k = cnt.value
        c = np.zeros(max(k, 1)); s = np.zeros(max(k, 1)); a = np.zeros(max(k, 1), dtype=np.int32)
        _check(self._L, self._h, self._L.bdu_read_rotations(
            self._h, side, _dp(c), _dp(s), a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), k, ctypes.byref(cnt)))
        return c[:k], s[:k], a[:k]

    def read_truncated(self, r):
        """Truncated bidiagonal approximation A_r = L R^T (bdu_read_truncated):
        returns (L m x r, R n x r, idx (1-based kept indices), err2)."""
        r = int(r)
        L = np.zeros((self.m, max(r, 1)), order="F"); R = np.zeros((self.n, max(r, 1)), order="F")
        idx = np.zeros(max(r, 1), dtype=np.int64)
        err2 = ctypes.c_double()
        _check(self._L, self._h, self._L.bdu_read_truncated(
            self._h, r, _dp(L), _dp(R), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(err2)))
        return L[:, :r], R[:, :r], idx[:r], err2.value

    def singular_values(self, k=None):
        """The k largest singular values of Bd, descending (bdu_singular_values)."""
        k = self.k if k is None else int(k)
        sv = np.zeros(max(k, 1))
        _check(self._L, self._h, self._L.bdu_singular_values(self._h, k, _dp(sv)))
        return sv[:k]

    def stats(self):
        st = Stats()
        _check(self._L, self._h, self._L.bdu_stats(self._h, ctypes.byref(st)))
        return {"updates": st.updates, "rot_left": list(st.rot_left), "rot_right": list(st.rot_right),
                "chase_steps": st.chase_steps, "reorth_q": st.reorth_q, "reorth_p": st.reorth_p,
                "ortho_q": st.ortho_q, "ortho_p": st.ortho_p, "launches": st.launches,
                "timed_updates": st.timed_updates, "ms_project": st.ms_project,
                "ms_chase": st.ms_chase, "ms_apply_q": st.ms_apply_q,
                "ms_apply_p": st.ms_apply_p, "apply_launches": st.apply_launches,
                "device_bytes": st.device_bytes, "graph_replays": st.graph_replays,
                "apply_variant": list(st.apply_variant), "tunings": st.tunings}

    def check_orthogonality(self):
        q = ctypes.c_double(); p = ctypes.c_double()
        _check(self._L, self._h, self._L.bdu_check_orthogonality(self._h, ctypes.byref(q), ctypes.byref(p)))
        return q.value, p.value

    def set_timing(self, on=True):
        _check(self._L, self._h, self._L.bdu_set_timing(self._h, 1 if on else 0))


class ThinTracker:
    """Rank-k subspace tracking A ~ Q1 B P1^T under rank-1 updates, truncated
    back to rank k after each (bdu_thin_create / bdu_thin_update / bdu_thin_read;
    Sec. 4).  precision FP64, or MIXED (FP32 thin factors, FP64 middle band)."""

    def __init__(self, Q1, d, e, P1, precision=FP64, stream=None, device=0, engine=0, graphs=True):
        L = load()
        Q1 = _f64(Q1); P1 = _f64(P1); d = _f64(d).ravel(); e = _f64(e).ravel()
        self.m, self.k = Q1.shape
        self.n = P1.shape[0]
        if e.size == 0:
            e = np.zeros(1)
        opt = Options()
        L.bdu_default_options(ctypes.byref(opt))
        opt.precision = int(precision)
        opt.device = int(device)
        opt.engine = int(engine)
        opt.graphs = 1 if graphs else 0
        if stream is not None:
            opt.cuda_stream = ctypes.c_void_p(int(stream))
        h = ctypes.c_void_p()
        code = L.bdu_thin_create(ctypes.byref(h), self.m, self.n, self.k, _dp(Q1), _dp(d), _dp(e), _dp(P1),
                                 ctypes.byref(opt))
        if code != 0:
            raise BduError(code, L.bdu_thin_last_error(None).decode())
        self._h = h
        self._L = L

    def _check(self, code):
        if code != 0:
            msg = self._L.bdu_thin_last_error(self._h)
            raise BduError(code, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            self._L.bdu_thin_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def update(self, b, c):
        """One step; returns (removed index (0-based, 0..k), truncation error ||.||_F^2)."""
        b = np.ascontiguousarray(np.asarray(b, dtype=np.float64).ravel())
        c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).ravel())
        if b.size != self.m or c.size != self.n:
            raise ValueError("b needs m entries and c n entries")
        i = ctypes.c_int64(); err2 = ctypes.c_double()
        self._check(self._L.bdu_thin_update(self._h, _dp(b), _dp(c), ctypes.byref(i), ctypes.byref(err2)))
        return i.value, err2.value

    def update_dev(self, ptr_b: int, ptr_c: int):
        i = ctypes.c_int64(); err2 = ctypes.c_double()
        self._check(self._L.bdu_thin_update_dev(self._h, ctypes.c_void_p(ptr_b), ctypes.c_void_p(ptr_c),
                                                ctypes.byref(i), ctypes.byref(err2)))
        return i.value, err2.value

    def read(self):
        m, n, k = self.m, self.n, self.k
        Q1 = np.zeros((m, k), order="F"); P1 = np.zeros((n, k), order="F")
        d = np.zeros(k); e = np.zeros(max(k - 1, 1))
        self._check(self._L.bdu_thin_read(self._h, _dp(Q1), _dp(d), _dp(e), _dp(P1)))
        return Q1, d, e[: k - 1], P1

    def stats(self):
        u, sb, sc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self._L.bdu_thin_stats(self._h, ctypes.byref(u), ctypes.byref(sb), ctypes.byref(sc)))
        return {"updates": u.value, "in_span_b": sb.value, "in_span_c": sc.value}
