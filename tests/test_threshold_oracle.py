"""Pins of the threshold oracle (oracle/threshold.py): hand cases, the triangle layout,
and connected components checked against scipy's graph routine on random graphs."""
import numpy as np
import pytest

from oracle import threshold as th
from paper_1803_02272_gb300 import synth


def test_hit_rule_by_hand():
    # 97 % homology: d <= 3 % of the longer read, exactly at the boundary included
    assert th.is_hit(3, 100, 90, 3, 100)
    assert not th.is_hit(4, 100, 90, 3, 100)
    assert th.is_hit(13, 450, 300, 3, 100)          # 1300 <= 1350
    assert not th.is_hit(14, 450, 300, 3, 100)      # 1400 > 1350
    # absolute threshold alone (num = den = 1 never binds: d <= max(la, lb))
    assert th.is_hit(5, 10, 10, 1, 1, abs_max=5)
    assert not th.is_hit(6, 10, 10, 1, 1, abs_max=5)
    # both
    assert not th.is_hit(3, 100, 100, 3, 100, abs_max=2)


def test_components_by_hand():
    lab = th.components(7, [(0, 1), (1, 2), (4, 5), (6, 6)])
    assert lab.tolist() == [0, 0, 0, 3, 4, 4, 6]
    lab = th.components(5, [(3, 4), (2, 4), (0, 2)])
    assert lab.tolist() == [0, 1, 0, 0, 0]


def test_components_match_scipy():
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    from scipy.sparse import coo_matrix
    for seed in range(5):
        st = synth.Stream(400 + seed, 0)
        n = 300
        m = int(st.integers(50, 400, ()))
        a = st.integers(0, n - 1, (m,))
        b = st.integers(0, n - 1, (m,))
        edges = list(zip(a.tolist(), b.tolist()))
        lab = th.components(n, edges)
        A = coo_matrix((np.ones(m), (a, b)), shape=(n, n))
        k, ref = csgraph.connected_components(A, directed=False)
        # same partition
        assert len(set(lab.tolist())) == k
        pairs = {(int(x), int(y)) for x, y in zip(lab, ref)}
        assert len(pairs) == k
        # canonical label = smallest member
        for c in set(lab.tolist()):
            members = np.nonzero(lab == c)[0]
            assert members.min() == c


def test_threshold_edges_layout_by_hand():
    # n = 4, triangle (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
    tri = np.array([1, 9, 9, 2, 9, 9], dtype=np.uint16)
    lens = np.array([10, 10, 10, 10])
    assert th.threshold_edges(tri, lens, 1, 1, abs_max=2) == [(0, 1), (1, 2)]
    assert th.components(4, th.threshold_edges(tri, lens, 1, 1, abs_max=2)).tolist() == [0, 0, 0, 3]


def test_annotation_by_hand():
    D = np.array([[1, 2, 50, 50],      # two hits, both species 7 -> 7
                  [1, 50, 2, 50],      # species 7 and 9 -> ambiguous
                  [50, 50, 50, 1],     # only an unlabelled reference -> none
                  [50, 50, 50, 50],    # no hit -> none
                  [1, 50, 50, 1]])     # species 7 and an unlabelled reference -> 7
    lq = [100] * 5
    lr = [100] * 4
    labels = [7, 7, 9, -1]
    got = th.annotate(D, lq, lr, labels, 3, 100)
    assert got.tolist() == [7, th.AMBIGUOUS, th.NONE, th.NONE, 7]


def test_hits_rect():
    D = np.array([[0, 5], [3, 4]])
    assert th.hits_rect(D, [100, 100], [100, 100], 3, 100) == {(0, 0, 0), (1, 0, 3)}


def test_rule_equals_per_read_bound_form():
    """The GPU streams test d <= max(T[la], T[lb]) with T[L] = min(abs_max, floor(num*L/den),
    65535), a rewrite that holds because T is non-decreasing in L.  Checked here against
    the oracle's rule on random rules, lengths and distances at the boundary."""
    st = synth.Stream(4242, 0)
    k = 20000
    num = st.integers(0, (1 << 20) - 1, (k,))
    den = st.integers(1, (1 << 20) - 1, (k,))
    am = st.integers(0, 70000, (k,))
    la, lb = st.integers(0, 65535, (k,)), st.integers(0, 65535, (k,))

    def bound(L):
        return np.minimum(np.minimum(am, num * L // den), 65535)

    edge = bound(np.maximum(la, lb))
    d = np.where(st.uniform((k,)) < 0.5, st.integers(0, 65535, (k,)), np.clip(edge + st.integers(-2, 2, (k,)), 0, 65535))
    want = np.array([th.is_hit(int(d[t]), int(la[t]), int(lb[t]), int(num[t]), int(den[t]), int(am[t]))
                     for t in range(k)])
    got = d <= np.maximum(bound(la), bound(lb))
    np.testing.assert_array_equal(got, want)
    assert want.sum() > k // 10
