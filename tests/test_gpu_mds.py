"""Classical MDS on the GPU (gbd_sqdist_square, gbd_gram_apply, gbd_mds) against the
oracle in oracle/mds.py.

Floating point here, so the bars are tolerances derived from the arithmetic:
* the fp16 square W = fp16(d^2 2^-s) is compared bit for bit with numpy's
  round-to-nearest float16 of the same value (exact in float32 for d < 4096);
* G X is exact (up to the final float32 rounding) when every input is exactly
  representable: small integer distances, integer X with zero column means;
* otherwise the tensor-core inputs are rounded to fp16 (unit roundoff u = 2^-11), so
  |Delta (W X)| <= 2u |D o D| |X| elementwise (plus float32 accumulation, n 2^-24), and
  the eigenvalues of the randomized SVD move by at most about ||Delta G||_2 <=
  u ||D o D||_F (Weyl), eigenvectors by ||Delta G|| / gap (Davis-Kahan).
All inputs are synthetic (synth.py) or come from the oracle.
"""
import numpy as np
import pytest

import oracle
from oracle import mds as omds
from paper_1803_02272_gb300 import synth

pytestmark = pytest.mark.gpu
U16 = 2.0 ** -11


@pytest.fixture(scope="module")
def env():
    import torch
    torch.cuda.set_device(0)
    from paper_1803_02272_gb300 import gbd
    ctx = gbd.Context(0)
    return gbd, ctx, torch


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _tri_dev(torch, tri):
    return _dev(torch, np.asarray(tri, dtype=np.uint16).view(np.int16))


def _expected_square(tri, n, ld):
    D = omds.tri_to_square(tri, n) if n >= 2 else np.zeros((n, n))
    dmax = D.max() if n >= 2 else 0.0
    s = 0
    while dmax * dmax * 2.0 ** -s > 65504.0:
        s += 1
    W = np.zeros((ld, ld), dtype=np.float16)
    W[:n, :n] = (D * D * 2.0 ** -s).astype(np.float16)
    return W.view(np.uint16), s


@pytest.mark.parametrize("n,ld,dhi", [(130, 256, 450), (2, 128, 7), (1, 128, 0), (300, 384, 4000),
                                      (700, 768, 65535)])
def test_sqdist_square(env, n, ld, dhi):
    gbd, ctx, torch = env
    m = n * (n - 1) // 2
    tri = synth.Stream(31, n).integers(0, dhi, (m,)).astype(np.uint16)
    if m:
        tri[m // 2] = dhi                              # the maximum is reached
    W = torch.full((ld * ld,), -1, dtype=torch.int16, device="cuda")
    d_tri = _tri_dev(torch, tri) if m else None
    s = gbd.gbd_sqdist_square(ctx.handle, d_tri, n, W, ld)
    torch.cuda.synchronize()
    got = W.cpu().numpy().view(np.uint16).reshape(ld, ld)
    want, s_want = _expected_square(tri, n, ld)
    assert s == s_want
    if dhi < 4096:
        np.testing.assert_array_equal(got, want)
    else:
        # d^2 >= 2^24 is rounded to float32 first: at most one fp16 ulp apart
        diff = np.abs(got.astype(np.int64) - want.astype(np.int64))
        assert diff.max() <= 1
    assert np.array_equal(got, got.T)


def test_sqdist_square_rejects_bad_ld(env):
    gbd, ctx, torch = env
    W = torch.empty(256 * 256, dtype=torch.int16, device="cuda")
    tri = _tri_dev(torch, np.zeros(10, np.uint16))
    for ld in (100, 0):
        with pytest.raises(gbd.GbdError) as e:
            gbd.gbd_sqdist_square(ctx.handle, tri, 5, W, ld)
        assert e.value.code == gbd.GBD_EINVAL
    with pytest.raises(gbd.GbdError):
        gbd.gbd_sqdist_square(ctx.handle, tri, 300, W, 256)       # ld < n


def _exact_inputs(n, k, seed):
    """Distances <= 20 and integer X with zero column means: every tensor-core input is
    exact in fp16 and every partial sum exact in float32."""
    m = n * (n - 1) // 2
    tri = synth.Stream(seed, 1).integers(0, 20, (m,)).astype(np.uint16)
    X = synth.Stream(seed, 2).integers(-1, 1, (n, k)).astype(np.float64)
    X[-1] = -X[:-1].sum(0)
    return tri, X.astype(np.float32)


@pytest.mark.parametrize("n,k", [(300, 64), (2000, 64), (2000, 16), (1000, 112), (640, 256)])
def test_gram_apply_exact_inputs(env, n, k):
    """Y = G X through the tcgen05 product, with inputs it represents exactly: matches
    the float64 oracle to float32 rounding.  Several row blocks, K slices and a ragged
    padding; any layout or descriptor error shows up as O(1) differences."""
    gbd, ctx, torch = env
    tri, X = _exact_inputs(n, k, 7 + n + k)
    ld = (n + 127) // 128 * 128
    W = torch.empty(ld * ld, dtype=torch.int16, device="cuda")
    s = gbd.gbd_sqdist_square(ctx.handle, _tri_dev(torch, tri), n, W, ld)
    assert s == 0
    Y = torch.empty((n, k), dtype=torch.float32, device="cuda")
    gbd.gbd_gram_apply(ctx.handle, W, n, ld, s, _dev(torch, X), k, Y)
    torch.cuda.synchronize()
    want = omds.gram(omds.tri_to_square(tri, n)) @ X.astype(np.float64)
    got = Y.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=2e-7, atol=2e-7 * np.abs(want).max())


def test_gram_apply_rounded_inputs(env):
    """SW distances of 800 synthetic reads and a Gaussian X: within the fp16 bound."""
    gbd, ctx, torch = env
    rs = synth.workload_paper_scale(n=800)
    n, k = rs.n, 64
    tri = oracle.all_pairs(rs)
    X = synth.Stream(77, 0).normal((n, k)).astype(np.float32)
    ld = (n + 127) // 128 * 128
    W = torch.empty(ld * ld, dtype=torch.int16, device="cuda")
    s = gbd.gbd_sqdist_square(ctx.handle, _tri_dev(torch, tri), n, W, ld)
    Y = torch.empty((n, k), dtype=torch.float32, device="cuda")
    gbd.gbd_gram_apply(ctx.handle, W, n, ld, s, _dev(torch, X), k, Y)
    torch.cuda.synchronize()
    D = omds.tri_to_square(tri, n)
    Xd = X.astype(np.float64)
    want = omds.gram(D) @ Xd
    Xc = Xd - Xd.mean(0)
    E = (D * D) @ np.abs(Xc) * (2 * U16 + n * 2.0 ** -24)      # bound on |Delta (D o D) Xc|
    bound = 0.5 * (E + E.mean(0)) * 1.01 + 1e-6 * np.abs(want).max()
    err = np.abs(Y.cpu().numpy().astype(np.float64) - want)
    assert np.all(err <= bound), float((err / bound).max())


def _mds_case(env, rs_or_tri, n, k, r, q, seed):
    gbd, ctx, torch = env
    tri = rs_or_tri
    omega = synth.Stream(seed, 0).normal((n, k)).astype(np.float32)
    lam = torch.empty(r, dtype=torch.float32, device="cuda")
    X = torch.empty((n, r), dtype=torch.float32, device="cuda")
    gbd.gbd_mds(ctx.handle, _tri_dev(torch, tri), n, _dev(torch, omega), k, r, q, lam, X)
    torch.cuda.synchronize()
    return lam.cpu().numpy().astype(np.float64), X.cpu().numpy().astype(np.float64), omega


@pytest.mark.parametrize("n,k,r,q", [(600, 32, 8, 2), (1000, 64, 50, 2), (300, 16, 4, 0)])
def test_mds_matches_oracle(env, n, k, r, q):
    """gbd_mds on SW distances of synthetic reads vs the oracle's randomized MDS with the
    same Gaussian test matrix."""
    rs = synth.workload_paper_scale(n=n)
    tri = oracle.all_pairs(rs)
    lam, X, omega = _mds_case(env, tri, n, k, r, q, 100 + n)
    D = omds.tri_to_square(tri, n)
    lam_o, U_o, X_o = omds.mds_randomized(D, r, omega.astype(np.float64), q)
    G = omds.gram(D)
    tol = 3.0 * (U16 * np.sqrt(np.mean((D * D) ** 2) / 3.0) * np.sqrt(n) + U16 * abs(lam_o[0]))
    assert np.all(np.diff(lam) <= 0)
    assert np.all(np.abs(lam - lam_o) <= tol), (np.abs(lam - lam_o).max(), tol)
    # eigenvectors of well-separated eigenvalues agree up to sign (Davis-Kahan)
    pos = lam_o > 0
    U = np.zeros_like(X)
    U[:, pos] = X[:, pos] / np.sqrt(lam[pos])[None, :]
    checked = 0
    for a in range(r):
        gap = min([abs(lam_o[a] - lam_o[b]) for b in range(r) if b != a] + [np.inf])
        if not pos[a] or gap < 10 * tol:
            continue
        c = abs(float(U[:, a] @ U_o[:, a]))
        assert 1.0 - c <= 8 * (tol / gap) ** 2 + 1e-5, (a, c, tol / gap)
        checked += 1
    assert checked >= 2
    # the coordinates reproduce the leading part of G
    assert np.linalg.norm(X @ X.T - X_o @ X_o.T) <= 0.02 * np.linalg.norm(X_o @ X_o.T) + 1e-3 * np.linalg.norm(G)


def test_mds_properties_on_gpu_distances(env):
    """At a size the dense oracle does not reach (6000 reads, distances from the GPU's own
    all-pairs call): eigenvalues sorted, coordinate columns centred and mutually
    orthogonal with squared norms equal to the eigenvalues."""
    gbd, ctx, torch = env
    rs = synth.workload_paper_scale(n=6000)
    s = ctx.load(rs)
    tri = ctx.all_pairs(s)
    n, k, r = rs.n, 64, 50
    omega = _dev(torch, synth.Stream(5, 0).normal((n, k)).astype(np.float32))
    lam = torch.empty(r, dtype=torch.float32, device="cuda")
    X = torch.empty((n, r), dtype=torch.float32, device="cuda")
    gbd.gbd_mds(ctx.handle, tri, n, omega, k, r, 2, lam, X)
    torch.cuda.synchronize()
    lam = lam.cpu().numpy().astype(np.float64)
    X = X.cpu().numpy().astype(np.float64)
    assert np.all(np.diff(lam) <= 0) and lam[0] > 0
    pos = lam > 1e-6 * lam[0]
    XtX = X.T @ X
    np.testing.assert_allclose(np.diag(XtX)[pos], lam[pos], rtol=2e-3)
    off = XtX - np.diag(np.diag(XtX))
    assert np.abs(off).max() <= 2e-3 * lam[0]
    assert np.abs(X.sum(0)).max() <= 1e-3 * np.sqrt(lam[0] * n)


def test_mds_zero_distances(env):
    n, k, r = 200, 16, 3
    lam, X, _ = _mds_case(env, np.zeros(n * (n - 1) // 2, np.uint16), n, k, r, 1, 3)
    assert np.all(lam == 0.0) and np.all(X == 0.0)


def test_mds_points_on_a_line(env):
    """Integer points on a line: the first coordinate is the centred position (up to
    sign), the rest vanish."""
    n, k, r = 400, 16, 3
    x = synth.Stream(12, 0).integers(0, 300, (n,)).astype(np.int64)
    iu = np.triu_indices(n, 1)
    tri = np.abs(x[iu[0]] - x[iu[1]]).astype(np.uint16)
    lam, X, _ = _mds_case(env, tri, n, k, r, 2, 13)
    xc = x - x.mean()
    assert lam[0] == pytest.approx(float(xc @ xc), rel=4 * U16)
    col = X[:, 0] * np.sign(X[:, 0] @ xc)
    assert np.abs(col - xc).max() <= 8 * U16 * np.abs(xc).max()
    assert np.all(np.abs(lam[1:]) <= 4 * U16 * lam[0])


@pytest.mark.parametrize("n,k,r,q", [(64, 64, 8, 1), (1000, 40, 8, 1), (1000, 128, 8, 1),
                                     (1000, 64, 65, 1), (1000, 64, 0, 1)])
def test_mds_rejects_bad_sizes(env, n, k, r, q):
    gbd, ctx, torch = env
    tri = _tri_dev(torch, np.zeros(n * (n - 1) // 2, np.uint16))
    om = torch.zeros((n, max(k, 1)), dtype=torch.float32, device="cuda")
    lam = torch.empty(max(r, 1), dtype=torch.float32, device="cuda")
    X = torch.empty((n, max(r, 1)), dtype=torch.float32, device="cuda")
    with pytest.raises(gbd.GbdError) as e:
        gbd.gbd_mds(ctx.handle, tri, n, om, k, r, q, lam, X)
    assert e.value.code == gbd.GBD_EINVAL


def test_mds_kept_square_reused_grown_and_trimmed(env):
    """The context keeps the fp16 square between calls: a smaller problem after a larger
    one reuses it, a larger one replaces it, gbd_trim frees it; every call gives the same
    result as the first call of its size (the arithmetic is deterministic)."""
    gbd, ctx, torch = env
    rng = np.random.default_rng(17)
    small = rng.integers(1, 400, size=500 * 499 // 2).astype(np.uint16)
    large = rng.integers(1, 400, size=900 * 899 // 2).astype(np.uint16)
    first_small = _mds_case(env, small, 500, 32, 8, 1, 5)
    first_large = _mds_case(env, large, 900, 32, 8, 1, 6)
    again_small = _mds_case(env, small, 500, 32, 8, 1, 5)
    gbd.gbd_trim(ctx.handle)
    after_trim = _mds_case(env, large, 900, 32, 8, 1, 6)
    for a, b in ((first_small, again_small), (first_large, after_trim)):
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
