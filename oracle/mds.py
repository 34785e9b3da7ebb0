"""CPU oracle for classical MDS of the read-distance matrix -- TEST INFRASTRUCTURE ONLY.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may import
this module; the library never does, and this module imports nothing from the library.

Plain numpy in float64, dense n x n matrices, so it is meant for n up to a few thousand.

What it follows (arxiv 1803.02272):
  * section 6.2 (classical MDS, after Torgerson): the scalar products <x_i, x_j> are
    recovered from the distances alone by double centering of the squared distances,
    giving the Gram matrix G; its eigenpairs (lambda_a, u_a), lambda_1 >= lambda_2 >= ...,
    give the coordinates X = U Lambda^(1/2), of which the first r columns are kept;
  * sections 3.2-3.3 (the paper's contribution): the first r eigenpairs come from a
    randomized SVD (Halko, Martinsson and Tropp 2011) instead of a full eigensolver,
    using that for a symmetric matrix the singular values are |lambda|.

Readings where the paper is silent (each one a parameter here):
  * the randomized SVD is the randomized subspace iteration (Halko et al., Algorithm 4.4:
    sketch Y = G Omega, orthonormalise, q rounds of multiplying by G^T and by G with an
    orthonormalisation after every product) followed by the direct eigendecomposition
    for Hermitian matrices (their Algorithm 5.3: B = Q^T G Q, B = V Lambda V^T, U = Q V);
  * the sketch has k = r + oversampling columns (the library's default k = 64 for
    r = 50) and q = 2 rounds; the Gaussian test matrix Omega is an input;
  * eigenpairs are ordered by eigenvalue, largest first, and the coordinates of a
    negative eigenvalue (a non-Euclidean distance) are 0: X[:, a] = u_a sqrt(max(lambda_a, 0)).
"""
from __future__ import annotations

import numpy as np


def tri_to_square(tri, n: int) -> np.ndarray:
    """The symmetric n x n distance matrix (zero diagonal) of a strict upper triangle
    stored row-major: tri[k(i, j)], k(i, j) = i*n - i*(i+1)/2 + (j-i-1), i < j."""
    tri = np.asarray(tri)
    m = n * (n - 1) // 2
    if tri.shape[0] != m:
        raise ValueError(f"triangle of {tri.shape[0]} entries, expected {m}")
    D = np.zeros((n, n), dtype=np.float64)
    iu = np.triu_indices(n, 1)          # row-major order of the strict upper triangle
    D[iu] = tri.astype(np.float64)
    return D + D.T


def gram(D: np.ndarray) -> np.ndarray:
    """G = -1/2 J (D o D) J with J = I - 11^T/n (section 6.2, step 1: double centering of the
    squared distances; entry (i, j) is the scalar product <x_i, x_j>)."""
    D = np.asarray(D, dtype=np.float64)
    n = D.shape[0]
    J = np.eye(n) - np.full((n, n), 1.0 / n)
    return -0.5 * J @ (D * D) @ J


def _top(lam: np.ndarray, U: np.ndarray, r: int):
    order = np.argsort(-lam, kind="stable")[:r]
    lam_r = lam[order]
    U_r = U[:, order]
    X = U_r * np.sqrt(np.maximum(lam_r, 0.0))[None, :]
    return lam_r, U_r, X


def mds_exact(D: np.ndarray, r: int):
    """Classical MDS with a full symmetric eigensolver (section 6.2, steps 1-3).
    Returns (lambda[r], U[n, r], X[n, r])."""
    G = gram(D)
    lam, U = np.linalg.eigh(G)
    return _top(lam, U, r)


def _orth(Y: np.ndarray) -> np.ndarray:
    Q, _ = np.linalg.qr(Y, mode="reduced")
    return Q


def range_finder(G: np.ndarray, omega: np.ndarray, q: int) -> np.ndarray:
    """Randomized subspace iteration (Halko et al. Algorithm 4.4): an orthonormal
    n x k basis Q whose range approximates the dominant range of G."""
    Q = _orth(G @ omega)
    for _ in range(q):
        Qt = _orth(G.T @ Q)
        Q = _orth(G @ Qt)
    return Q


def mds_randomized(D: np.ndarray, r: int, omega: np.ndarray, q: int = 2):
    """Classical MDS through the randomized SVD of section 3.2: range finder on G with
    the n x k Gaussian matrix omega (k >= r), then B = Q^T G Q, B = V Lambda V^T,
    U = Q V (Halko et al. Algorithm 5.3).  Returns (lambda[r], U[n, r], X[n, r])."""
    G = gram(D)
    omega = np.asarray(omega, dtype=np.float64)
    if omega.shape[0] != G.shape[0] or omega.shape[1] < r:
        raise ValueError("omega must be n x k with k >= r")
    Q = range_finder(G, omega, q)
    B = Q.T @ G @ Q
    B = 0.5 * (B + B.T)
    lam, V = np.linalg.eigh(B)
    return _top(lam, Q @ V, r)
