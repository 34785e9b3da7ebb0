"""Pins of the classical-MDS oracle (oracle/mds.py) to facts outside itself.

* Euclidean point clouds: classical MDS recovers the centred Gram matrix exactly, so
  G = Xc Xc^T, the non-zero eigenvalues are those of Xc^T Xc and the rest vanish
  (Torgerson; section 6.2 of the paper).
* Points on a line with integer coordinates give an integer distance triangle whose MDS
  is the centred coordinate itself, up to sign.
* The triangle layout, by hand on n = 4.
* The randomized SVD is exact when rank(G) <= k (Halko et al. section 1.3) and obeys
  Cauchy interlacing for any symmetric G (B = Q^T G Q with orthonormal Q).
"""
import numpy as np
import pytest

from oracle import mds
from paper_1803_02272_gb300 import synth


def _points(n, dim, seed):
    return synth.Stream(seed, 7).uniform((n, dim)) * 10.0 - 5.0


def _euclid(P):
    diff = P[:, None, :] - P[None, :, :]
    return np.sqrt((diff * diff).sum(-1))


def _gaussian(n, k, seed):
    return synth.Stream(seed, 11).normal((n, k))


def test_triangle_layout_by_hand():
    tri = np.array([1, 2, 3, 4, 5, 6], dtype=np.uint16)   # (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
    D = mds.tri_to_square(tri, 4)
    want = np.array([[0, 1, 2, 3], [1, 0, 4, 5], [2, 4, 0, 6], [3, 5, 6, 0]], dtype=float)
    assert np.array_equal(D, want)
    with pytest.raises(ValueError):
        mds.tri_to_square(tri[:5], 4)


def test_gram_of_euclidean_points_is_centred_gram():
    P = _points(60, 3, 1)
    Pc = P - P.mean(0)
    G = mds.gram(_euclid(P))
    assert np.allclose(G, Pc @ Pc.T, rtol=0, atol=1e-9 * np.abs(Pc @ Pc.T).max())


def test_exact_mds_recovers_euclidean_configuration():
    P = _points(80, 3, 2)
    Pc = P - P.mean(0)
    lam, U, X = mds.mds_exact(_euclid(P), 6)
    ev = np.sort(np.linalg.eigvalsh(Pc.T @ Pc))[::-1]
    assert np.allclose(lam[:3], ev, rtol=1e-10)
    assert np.all(np.abs(lam[3:]) < 1e-9 * lam[0])
    assert np.allclose(X[:, :3] @ X[:, :3].T, Pc @ Pc.T, atol=1e-8 * lam[0])
    assert np.allclose(U.T @ U, np.eye(6), atol=1e-10)


def test_points_on_a_line_from_integer_triangle():
    x = np.array([0, 3, 7, 12, 20, 21, 40, 41, 55, 90], dtype=np.int64)
    n = len(x)
    iu = np.triu_indices(n, 1)
    tri = np.abs(x[iu[0]] - x[iu[1]]).astype(np.uint16)
    lam, U, X = mds.mds_exact(mds.tri_to_square(tri, n), 2)
    xc = x - x.mean()
    assert lam[0] == pytest.approx(float((xc * xc).sum()), rel=1e-12)
    assert abs(lam[1]) < 1e-9 * lam[0]
    col = X[:, 0] * np.sign(X[0, 0] * xc[0])
    assert np.allclose(col, xc, atol=1e-9 * np.abs(xc).max())


def test_randomized_is_exact_for_low_rank():
    P = _points(200, 5, 3)
    D = _euclid(P)
    omega = _gaussian(200, 16, 4)
    for q in (0, 1, 2):
        lam_r, _, X_r = mds.mds_randomized(D, 5, omega, q)
        lam_e, _, X_e = mds.mds_exact(D, 5)
        assert np.allclose(lam_r, lam_e, rtol=1e-9)
        assert np.allclose(X_r @ X_r.T, X_e @ X_e.T, atol=1e-8 * lam_e[0])


def test_randomized_interlaces_exact_spectrum():
    # a non-Euclidean integer distance matrix: eigenvalues of both signs
    n, k = 150, 24
    tri = synth.Stream(5, 3).integers(0, 400, (n * (n - 1) // 2,)).astype(np.uint16)
    D = mds.tri_to_square(tri, n)
    ev = np.sort(np.linalg.eigvalsh(mds.gram(D)))[::-1]
    assert ev[-1] < 0 < ev[0]
    omega = _gaussian(n, k, 6)
    lam, U, _ = mds.mds_randomized(D, k, omega, q=2)
    tol = 1e-9 * abs(ev[0])
    assert np.all(lam <= ev[:k] + tol)                 # lambda_i(B) <= lambda_i(G)
    assert np.all(lam >= ev[n - k:] - tol)             # lambda_i(B) >= lambda_{i+n-k}(G)
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-10)


def test_randomized_converges_on_a_dominant_subspace():
    # two well-separated directions (a planar configuration, coordinates ~ 1e3) plus
    # integer noise: subspace iteration with q = 2 pins the two leading eigenpairs
    n, k = 300, 16
    P = _points(n, 2, 9) * 200.0
    noise = synth.Stream(9, 5).integers(0, 20, (n, n)).astype(float)
    D = np.rint(_euclid(P) + np.triu(noise, 1) + np.triu(noise, 1).T)
    ev, V = np.linalg.eigh(mds.gram(D))
    ev, V = ev[::-1], V[:, ::-1]
    assert ev[1] > 50 * abs(ev[2])
    lam, U, _ = mds.mds_randomized(D, 2, _gaussian(n, k, 10), q=2)
    assert np.allclose(lam, ev[:2], rtol=1e-9)
    assert np.allclose(np.abs(np.sum(U * V[:, :2], axis=0)), 1.0, atol=1e-9)


def test_negative_eigenvalues_give_zero_coordinates():
    n = 40
    tri = synth.Stream(8, 1).integers(0, 50, (n * (n - 1) // 2,)).astype(np.uint16)
    lam, U, X = mds.mds_exact(mds.tri_to_square(tri, n), n)
    neg = lam < 0
    assert neg.any()
    assert np.all(X[:, neg] == 0.0)
    assert np.allclose(X[:, ~neg], U[:, ~neg] * np.sqrt(lam[~neg]))
