"""The symmetric variant (Sec. 6) on the GPU: the tridiagonalization of
T + rho u u^T (bdu_tri_factor) and the in-place update A + rho c c^T of
A = Q T Q^T (bdu_tri_update_dev), against the oracle (oracle/bhu.py: tri,
tri_update) and LAPACK.  Tolerances as in test_gpu_bhu.py: the two sides are
Householder processes that differ in the order of their sums, TOL(n) =
1e-14 n ||M||_F for the tridiagonal entries, a reflector vector's column over
its source column's norm |beta_j|, eigenvalues within 1e-12 of the largest."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import bhu as H  # noqa: E402

pytestmark = pytest.mark.gpu


def _bdu():
    from paper_2509_02840_gb300 import bdu
    bdu.load()
    return bdu


def tol(n, scale):
    return 1e-14 * max(n, 1) * scale


def _case(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n), rng.standard_normal(max(n - 1, 0)), rng.standard_normal(n), float(
        rng.choice([-1.5, 0.7, 2.0]))


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.float64))).cuda()


def run_tri(n, a, b, u, rho, steps=None):
    bdu = _bdu()
    steps = n if steps is None else steps
    k, wb, _ = bdu.tri_sizes(n, steps)
    aa, bb, uu = _dev(a), _dev(b if n > 1 else [0.0]), _dev(u)
    z = lambda c: torch.zeros(max(c, 1), dtype=torch.float64, device="cuda")
    al, be, Y, S, ws = z(steps), z(min(steps, n - 1)), z(n * k), z(k * k), z((wb + 7) // 8)
    bdu.tri_factor(n, steps, aa.data_ptr(), bb.data_ptr() if n > 1 else 0, rho, uu.data_ptr(), al.data_ptr(),
                   be.data_ptr() if n > 1 else 0, Y.data_ptr() if k else 0, S.data_ptr() if k else 0, ws.data_ptr(),
                   torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return {"alpha": al.cpu().numpy()[:steps], "beta": be.cpu().numpy()[:min(steps, n - 1)],
            "Y": Y.cpu().numpy()[:n * k].reshape(k, n).T, "S": S.cpu().numpy()[:k * k].reshape(k, k).T}


@pytest.mark.parametrize("n", [1, 2, 3, 5, 64, 257, 530, 1030])
def test_tri_factor_matches_oracle(n):
    a, b, u, rho = _case(n, 13 * n)
    g = run_tri(n, a, b, u, rho)
    o = H.tri(a, b, u, rho)
    scale = np.linalg.norm(H.tridiag_dense(a, b) + rho * np.outer(u, u))
    assert np.abs(g["alpha"] - o["alpha"]).max() <= tol(n, scale)
    if n > 1:
        assert np.abs(g["beta"] - o["beta"]).max() <= tol(n, scale)
    assert g["Y"].shape == o["Y"].shape
    for j in range(o["Y"].shape[1]):
        tj = tol(n, scale) / max(abs(o["beta"][j]), 1e-300)
        assert np.abs(g["Y"][:, j] - o["Y"][:, j]).max() <= tj
        assert not np.any(g["Y"][:j + 1, j])
    if o["Y"].size:
        # the compact form (S = 2 T^{-1}) against the plain product of the same reflectors
        Qg = np.eye(n) - g["Y"] @ g["S"] @ g["Y"].T
        Qp, _ = H.factors(g["Y"], np.zeros((1, 0)), n, 1)
        assert np.abs(Qg - Qp).max() <= 1e-12 * n
        Tg = H.tridiag_dense(g["alpha"], g["beta"])
        M = H.tridiag_dense(a, b) + rho * np.outer(u, u)
        assert np.abs(Qg @ Tg @ Qg.T - M).max() <= 1e-12 * scale


@pytest.mark.parametrize("n,t", [(12, 4), (300, 57), (530, 300)])
def test_tri_partial(n, t):
    a, b, u, rho = _case(n, n + t)
    g = run_tri(n, a, b, u, rho, steps=t)
    o = H.tri(a, b, u, rho, steps=t)
    scale = np.linalg.norm(H.tridiag_dense(a, b) + rho * np.outer(u, u))
    assert np.abs(g["alpha"] - o["alpha"]).max() <= tol(n, scale)
    assert np.abs(g["beta"] - o["beta"]).max() <= tol(n, scale)


@pytest.mark.parametrize("n", [1024, 2048])
def test_tri_eigenvalues_lapack(n):
    a, b, u, rho = _case(n, 5 * n)
    g = run_tri(n, a, b, u, rho)
    e0 = np.linalg.eigvalsh(H.tridiag_dense(a, b) + rho * np.outer(u, u))
    e1 = np.linalg.eigvalsh(H.tridiag_dense(g["alpha"], g["beta"]))
    assert np.abs(e0 - e1).max() <= 1e-12 * np.abs(e0).max()


@pytest.mark.parametrize("n", [3, 64, 300])
def test_tri_update_in_place(n):
    bdu = _bdu()
    rng = np.random.default_rng(n)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    a, b, c, rho = _case(n, 2 * n)
    _, _, ub = bdu.tri_sizes(n, n)
    Qd = torch.from_numpy(np.asfortranarray(Q).reshape(-1, order="F").copy()).cuda()
    ad, bd, cd = _dev(a), _dev(b), _dev(c)
    ws = torch.zeros((ub + 7) // 8, dtype=torch.float64, device="cuda")
    bdu.tri_update_dev(n, Qd.data_ptr(), ad.data_ptr(), bd.data_ptr(), rho, cd.data_ptr(), ws.data_ptr(),
                       torch.cuda.current_stream().cuda_stream)
    Qg = Qd.cpu().numpy().reshape(n, n, order="F")
    ag, bg = ad.cpu().numpy(), bd.cpu().numpy()
    Qo, ao, bo = H.tri_update(Q, a, b, rho, c)
    A1 = Q @ H.tridiag_dense(a, b) @ Q.T + rho * np.outer(c, c)
    scale = np.linalg.norm(A1)
    assert np.abs(ag - ao).max() <= tol(n, scale) and np.abs(bg - bo).max() <= tol(n, scale)
    assert np.abs(Qg - Qo).max() <= 1e-12 * n
    assert np.abs(Qg @ H.tridiag_dense(ag, bg) @ Qg.T - A1).max() <= 1e-12 * scale
    assert np.abs(Qg[:, 0] - Q[:, 0]).max() <= 1e-15


def test_tri_grid_barrier_expires():
    """The symmetric kernel's grid barriers are the bounded waits of BHU's: with
    the first block held back by failure injection the others give up after
    2000 polls and the call reports BDU_ETIMEOUT; a later call is unaffected."""
    bdu = _bdu()
    n = 64
    a, b, u, rho = _case(n, 1)
    bdu.set_fault_injection(bdu.INJECT_BHU_STALL, 2000)
    try:
        with pytest.raises(bdu.BduError) as info:
            run_tri(n, a, b, u, rho)
    finally:
        bdu.set_fault_injection(bdu.INJECT_NONE)
    assert info.value.code == 4 and "grid barrier" in str(info.value)
    g = run_tri(n, a, b, u, rho)
    o = H.tri(a, b, u, rho)
    assert np.abs(g["alpha"] - o["alpha"]).max() <= tol(n, np.linalg.norm(H.tridiag_dense(a, b) + rho * np.outer(u, u)))
