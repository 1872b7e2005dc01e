"""Seeded synthetic workloads (no arithmetic of the update method itself).

These generators stand in for the paper's datasets (MovieLens ratings,
Flickr/Slashdot adjacency streams, SuiteSparse matrices), which are not
available: they reproduce the shapes, value distributions and structure of
those workloads.  Both the oracle tests and the CUDA path draw from here.

Factorization (all configurations): Q and P are products of 8 Householder
reflectors I - 2 v v^T / (v^T v) with v ~ N(0, 1); the bidiagonal has
d_i ~ U(1, 10) and e_i ~ N(0, 1).

Streams:
  * dense      -- b ~ N(0,1)^m, c ~ N(0,1)^n                          (20 rank-1)
  * recommender-- b: round(0.02 m) distinct rows chosen uniformly, values
                  uniform in {1,...,5}; c = e_j with j = h mod n ("set item
                  column", Sec. 4.2, Eq. streamsys shape)                (rank-1)
  * block      -- B ~ N(0,1)^{m x r}, C ~ N(0,1)^{n x r} / sqrt(n)      (rank-8)
  * network    -- B = [w e_i, w e_j], C = [e_j, e_i]; (i, j) drawn with
                  Chung-Lu weights of a power law with exponent 2.1, no self
                  loops, w ~ U(0.5, 1.5) (Sec. 4.1 edge insertions)      (rank-2)
"""
import numpy as np

SEED_BASE = 0x250902840


def rng(config: int, stream: int = 0) -> np.random.Generator:
    return np.random.default_rng([SEED_BASE + int(config), int(stream)])


def householder_orthogonal(n: int, g: np.random.Generator, reflectors: int = 8) -> np.ndarray:
    """Random orthogonal n x n matrix as a product of Householder reflectors."""
    X = np.eye(n)
    for _ in range(reflectors):
        v = g.standard_normal(n)
        X -= np.outer(X @ v, v) * (2.0 / np.dot(v, v))
    return np.asfortranarray(X)


def factorization(m: int, n: int, config: int = 0, which: int = 0):
    """Returns (Q, d, e, P) in FP64, column-major; d has min(m, n) entries
    (the band is lower bidiagonal when m < n)."""
    g = rng(config, 1_000_000 + which)
    Q = householder_orthogonal(m, g)
    P = householder_orthogonal(n, g)
    k = min(m, n)
    d = g.uniform(1.0, 10.0, k)
    e = g.standard_normal(max(k - 1, 0))
    return Q, d, e, P


def dense_update(m: int, n: int, h: int, config: int = 0, r: int = 1):
    g = rng(config, h)
    B = g.standard_normal((m, r))
    C = g.standard_normal((n, r))
    return np.asfortranarray(B), np.asfortranarray(C)


def recommender_update(m: int, n: int, h: int, config: int = 1, density: float = 0.02):
    """Sparse ratings column b (values 1..5 on round(density*m) rows), c = e_j, j = h mod n."""
    g = rng(config, h)
    k = int(round(density * m))
    rows = g.choice(m, size=k, replace=False)
    B = np.zeros((m, 1))
    B[rows, 0] = g.integers(1, 6, size=k).astype(np.float64)
    C = np.zeros((n, 1))
    C[h % n, 0] = 1.0
    return np.asfortranarray(B), np.asfortranarray(C)


def block_update(m: int, n: int, h: int, config: int = 2, r: int = 8):
    g = rng(config, h)
    B = g.standard_normal((m, r))
    C = g.standard_normal((n, r)) / np.sqrt(n)
    return np.asfortranarray(B), np.asfortranarray(C)


def chung_lu_weights(n: int, exponent: float = 2.1) -> np.ndarray:
    """Expected-degree weights w_i proportional to i^(-1/(exponent-1))."""
    i = np.arange(1, n + 1, dtype=np.float64)
    w = i ** (-1.0 / (exponent - 1.0))
    return w / w.sum()


def network_update(n: int, h: int, config: int = 3, exponent: float = 2.1):
    """Symmetric edge insertion B = [w e_i, w e_j], C = [e_j, e_i]."""
    g = rng(config, h)
    p = chung_lu_weights(n, exponent)
    i = int(g.choice(n, p=p))
    j = i
    while j == i:
        j = int(g.choice(n, p=p))
    w = g.uniform(0.5, 1.5)
    B = np.zeros((n, 2)); C = np.zeros((n, 2))
    B[i, 0] = w; B[j, 1] = w
    C[j, 0] = 1.0; C[i, 1] = 1.0
    return np.asfortranarray(B), np.asfortranarray(C)


def thin_factors(m: int, n: int, k: int, config: int = 3, which: int = 0):
    """(Q1 m x k, d k, e k-1, P1 n x k): orthonormal columns from the QR
    factorization of Gaussian matrices, d ~ U(1, 10), e ~ N(0, 1)."""
    g = rng(config, 2_000_000 + which)
    Q1 = np.linalg.qr(g.standard_normal((m, k)))[0]
    P1 = np.linalg.qr(g.standard_normal((n, k)))[0]
    d = g.uniform(1.0, 10.0, k)
    e = g.standard_normal(max(k - 1, 0))
    return np.asfortranarray(Q1), d, e, np.asfortranarray(P1)


def serving_mix(count: int = 256, lo: int = 64, hi: int = 2048, config: int = 4):
    """(m, n) pairs, each log-uniform in [lo, hi], swapped so that m >= n."""
    g = rng(config, 0)
    a = np.exp(g.uniform(np.log(lo), np.log(hi), count)).astype(int)
    b = np.exp(g.uniform(np.log(lo), np.log(hi), count)).astype(int)
    return [(int(max(x, y)), int(min(x, y))) for x, y in zip(a, b)]


def serving_update(m: int, n: int, stream: int, h: int, config: int = 4):
    """Rank r ~ U{1..4}, N(0,1) entries."""
    g = rng(config, 1000 * stream + h + 1)
    r = int(g.integers(1, 5))
    return np.asfortranarray(g.standard_normal((m, r))), np.asfortranarray(g.standard_normal((n, r)))
