"""Pins of the CPU oracle against things other than itself (CPU only).

The oracle computes the Smith-Waterman local score from the full DP matrix and the
distance d = max(la, lb) - S (paper section 2.2).  It is checked here against
  * hand-worked cases (tests/golden/hand_cases.txt),
  * a brute force that lists every alignment of every substring pair (C, no DP table),
    itself cross-checked by a second, pure-Python brute force,
  * exhaustive enumeration of all read pairs of length <= 4, random pairs of length 5-6,
  * invariants: d(x,x) = 0, symmetry, |la - lb| <= d <= max(la, lb),
  * closed forms: a read inside another gives S = |x|; S is at least the best
    gap-free diagonal segment (a maximum-subarray problem, solved by Kadane's scan),
  * the strict upper-triangle layout of ~n^2/2 values for n reads (section 2.2),
  * the other score-to-distance readings (min length minus S, the raw score, the
    normalised 1 - S/max): hand-worked values (tests/golden/conversions.txt) and the
    relations between the readings that the definitions fix.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1803_02272_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.txt")


def _hand_cases():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            a, b, S, d = line.split()
            rows.append(("" if a == "-" else a, "" if b == "-" else b, int(S), int(d)))
    return rows


HAND = _hand_cases()


def test_hand_cases_loaded():
    assert len(HAND) >= 12


@pytest.mark.parametrize("a,b,S,d", HAND)
def test_oracle_hand_cases(a, b, S, d):
    assert oracle.sw_score(a, b) == S
    assert oracle.distance(a, b) == d
    assert oracle.distance(b, a) == d


@pytest.mark.parametrize("a,b,S,d", HAND)
def test_brute_hand_cases(a, b, S, d):
    if len(a) + len(b) <= 13:
        assert oracle.brute_score(a, b) == S
    if len(a) + len(b) <= 9:
        assert oracle.brute_score_py(a, b) == S


def test_two_brute_forces_agree():
    st = synth.Stream(77, 0)
    for _ in range(60):
        la, lb = (int(x) for x in st.integers(0, 4, (2,)))
        a = "".join("ACGT"[c] for c in synth.random_codes(st, (la,)))
        b = "".join("ACGT"[c] for c in synth.random_codes(st, (lb,)))
        for m, x, g in [(1, -1, 1), (2, -3, 2)]:
            assert oracle.brute_score(a, b, m, x, g) == oracle.brute_score_py(a, b, m, x, g)


def _strings_readset(strings):
    return synth.from_strings(strings)


@pytest.mark.parametrize("scores", [(1, -1, 1), (2, -3, 2), (1, -2, 3)])
def test_exhaustive_len4(scores):
    """Every pair of reads over ACGT with lengths 0..4 (341^2 = 116,281 pairs)."""
    m, x, g = scores
    strings = oracle.brute_strings(4)
    brute = oracle.brute_exhaustive(4, m, x, g)
    rs = _strings_readset(strings)
    n = len(strings)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    S = oracle.pair_scores(rs, ii.ravel(), jj.ravel(), match=m, mismatch=x, gap=g)
    np.testing.assert_array_equal(S, brute.ravel())
    if scores == (1, -1, 1):
        d = oracle.pairs(rs, ii.ravel(), jj.ravel()).astype(np.int64)
        L = rs.lengths
        np.testing.assert_array_equal(np.maximum(L[ii.ravel()], L[jj.ravel()]) - d, brute.ravel())


def test_random_len5_6():
    st = synth.Stream(2024, 5)
    strs_a, strs_b = [], []
    for _ in range(1500):
        la, lb = (int(v) for v in st.integers(5, 6, (2,)))
        strs_a.append("".join("ACGT"[c] for c in synth.random_codes(st, (la,))))
        strs_b.append("".join("ACGT"[c] for c in synth.random_codes(st, (lb,))))
    # a small alphabet makes long matches likely; add low-entropy reads too
    strs_a += ["AAAAAA", "ACACAC", "AAAAA", "GGGGGG"]
    strs_b += ["AAAAAA", "CACACA", "AATAAA", "GGCGGG"]
    A, B = synth.from_strings(strs_a), synth.from_strings(strs_b)
    k = np.arange(len(strs_a))
    d = oracle.pairs(A, k, k, B).astype(np.int64)
    for p, (a, b) in enumerate(zip(strs_a, strs_b)):
        assert max(len(a), len(b)) - d[p] == oracle.brute_score(a, b), (a, b)


def test_invariants_small_workload():
    rs = synth.workload_plain_small()
    n = 60
    sub = rs.subset(range(n))
    D = oracle.rect(sub, 0, n, sub, 0, n)
    L = sub.lengths
    assert np.all(np.diag(D) == 0)                                   # d(x,x) = 0
    np.testing.assert_array_equal(D, D.T)                            # symmetry
    lo = np.abs(L[:, None] - L[None, :])
    hi = np.maximum(L[:, None], L[None, :])
    assert np.all(D >= lo) and np.all(D <= hi)                       # length bounds
    # reads from a shared ancestor are close, unrelated reads are far
    assert np.median(D[np.triu_indices(n, 1)]) > 20


def test_substring_closed_form():
    st = synth.Stream(31, 1)
    for _ in range(40):
        ly = int(st.integers(20, 200, (1,))[0])
        y = "".join("ACGT"[c] for c in synth.random_codes(st, (ly,)))
        i0 = int(st.integers(0, ly - 1, (1,))[0])
        i1 = int(st.integers(i0, ly, (1,))[0])
        x = y[i0:i1]
        assert oracle.sw_score(x, y) == len(x)
        assert oracle.distance(x, y) == ly - len(x)


def _best_ungapped(a: str, b: str) -> int:
    """Best gap-free local segment: maximum-subarray (Kadane) over every diagonal."""
    best = 0
    for off in range(-len(a) + 1, len(b)):
        run = 0
        for i in range(len(a)):
            j = i + off
            if 0 <= j < len(b):
                run = max(0, run + (1 if a[i] == b[j] else -1))
                best = max(best, run)
    return best


def test_gap_free_lower_bound_and_equal_when_gaps_cannot_help():
    st = synth.Stream(99, 2)
    for _ in range(30):
        L = int(st.integers(30, 80, (1,))[0])
        a = "".join("ACGT"[c] for c in synth.random_codes(st, (L,)))
        flip = st.uniform((L,)) < 0.1                    # substitutions only
        b ="".join("ACGT"["ACGT".index(ch) ^ (1 if f else 0)] for ch, f in zip(a, flip))
        S = oracle.sw_score(a, b)
        assert S >= _best_ungapped(a, b)
    # with gaps made prohibitively expensive the local score is exactly the best
    # gap-free segment
    for _ in range(30):
        la, lb = (int(v) for v in st.integers(5, 40, (2,)))
        a = "".join("ACGT"[c] for c in synth.random_codes(st, (la,)))
        b = "".join("ACGT"[c] for c in synth.random_codes(st, (lb,)))
        assert oracle.sw_score(a, b, 1, -1, 1000) == _best_ungapped(a, b)


def test_triangle_layout():
    rs = synth.workload_plain_small().subset(range(23))
    n = rs.n
    tri = oracle.all_pairs(rs)
    assert tri.shape == (n * (n - 1) // 2,)
    k = 0
    pi, pj = [], []
    for i in range(n):
        for j in range(i + 1, n):
            assert oracle.tri_index(i, j, n) == k
            pi.append(i)
            pj.append(j)
            k += 1
    np.testing.assert_array_equal(tri, oracle.pairs(rs, pi, pj))
    # the paper's count: ~5e9 values for 1e5 reads is n(n-1)/2
    assert 100_000 * 99_999 // 2 == 4_999_950_000


def test_rect_matches_pairs():
    rs = synth.workload_plain_small()
    A = rs.subset(range(0, 17))
    B = rs.subset(range(40, 53))
    R = oracle.rect(A, 2, 15, B, 1, 13)
    ii, jj = np.meshgrid(np.arange(2, 15), np.arange(1, 13), indexing="ij")
    np.testing.assert_array_equal(R.ravel(), oracle.pairs(A, ii.ravel(), jj.ravel(), B))


# ------------------------------------------------------------------ affine gaps (Gotoh)

@pytest.mark.parametrize("scores", [(1, -1, 1, 2), (2, -3, 1, 3), (1, -2, 2, 1)])
def test_affine_exhaustive_len4(scores):
    """Affine mode (a run of L gapped bases costs gap_open + L * gap) against the brute
    force that charges each gap run explicitly, on every pair of reads of length <= 4."""
    m, x, g, go = scores
    strings = oracle.brute_strings(4)
    brute = oracle.brute_exhaustive(4, m, x, g, go)
    rs = _strings_readset(strings)
    n = len(strings)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    S = oracle.pair_scores(rs, ii.ravel(), jj.ravel(), match=m, mismatch=x, gap=g, gap_open=go)
    np.testing.assert_array_equal(S, brute.ravel())


def test_affine_by_hand_and_limits():
    # one gap of length 2: AAAAGGTTTT vs AAAATTTT, 8 matches - (open + 2 * extend)
    assert oracle.sw_score_affine("AAAAGGTTTT", "AAAATTTT", gap_open=1, gap=1) == 8 - 3
    assert oracle.brute_score_affine("AAAAGGTTTT", "AAAATTTT", gap_open=1, gap=1) == 5
    # shorter flanks: the gapped alignment (6 - 3) loses to the gap-free AAAA (4)
    assert oracle.sw_score_affine("AAAAGGTT", "AAAATT", gap_open=1, gap=1) == 4
    # under a large open penalty the best local alignment avoids the gap (AAAA or TTTT)
    assert oracle.sw_score_affine("AAAAGGTTTT", "AAAATTTT", gap_open=5, gap=1) == 4
    # gap_open = 0 is the linear model
    st = synth.Stream(31, 1)
    for _ in range(200):
        la, lb = (int(v) for v in st.integers(0, 12, (2,)))
        a = "".join("ACGT"[c] for c in synth.random_codes(st, (la,)))
        b = "".join("ACGT"[c] for c in synth.random_codes(st, (lb,)))
        assert oracle.sw_score_affine(a, b, gap_open=0, gap=1) == oracle.sw_score(a, b)
        # a positive open penalty never raises the score, and never lowers it below the
        # best gap-free segment
        assert oracle.sw_score_affine(a, b, gap_open=2, gap=1) <= oracle.sw_score(a, b)


def test_affine_random_len5_6_brute():
    st = synth.Stream(2025, 5)
    for _ in range(300):
        la, lb = (int(v) for v in st.integers(5, 6, (2,)))
        a = "".join("ACGT"[c] for c in synth.random_codes(st, (la,)))
        b = "".join("ACGT"[c] for c in synth.random_codes(st, (lb,)))
        assert oracle.sw_score_affine(a, b, gap_open=2, gap=1) == oracle.brute_score_affine(a, b, 2, 1)


def test_distance_clamped_into_uint16_range():
    # match +2 lets S exceed max(la, lb): the stored distance is clamped at 0
    rs = synth.from_strings(["ACGTACGT", "ACGTACGT", "ACG"])
    tri = oracle.all_pairs(rs, match=2, mismatch=-3, gap=1)
    assert tri.tolist() == [0, 2, 2]                  # S = 16, 6, 6 against max = 8, 8, 8
    assert oracle.all_pairs(rs).tolist() == [0, 5, 5]


# ------------------------------------------------------------------ conversions

CONV_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "conversions.txt")


def _conv_cases():
    rows = []
    with open(CONV_GOLDEN) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            a, b, S, dmax, dmin, dnorm = line.split()
            rows.append(("" if a == "-" else a, "" if b == "-" else b, int(S), int(dmax), int(dmin), int(dnorm)))
    return rows


CONV = _conv_cases()


def test_conversion_cases_loaded():
    assert len(CONV) >= 12


@pytest.mark.parametrize("a,b,S,dmax,dmin,dnorm", CONV)
def test_conversion_hand_cases(a, b, S, dmax, dmin, dnorm):
    for x, y in ((a, b), (b, a)):
        assert oracle.sw_score(x, y) == S
        assert oracle.distance_conv(x, y, oracle.CONV_MAX) == dmax
        assert oracle.distance_conv(x, y, oracle.CONV_MIN) == dmin
        assert oracle.distance_conv(x, y, oracle.CONV_SCORE) == S
        assert oracle.distance_conv(x, y, oracle.CONV_NORM) == dnorm


def test_conversion_clamps_hand_cases():
    """With match +3 the score can exceed both lengths: every length-based reading clamps
    at 0 (worked by hand: AC vs AC scores 6; A vs AC scores 3)."""
    for a, b, S in (("AC", "AC", 6), ("A", "AC", 3)):
        for conv, want in ((oracle.CONV_MAX, 0), (oracle.CONV_MIN, 0), (oracle.CONV_NORM, 0),
                           (oracle.CONV_SCORE, S)):
            assert oracle.distance_conv(a, b, conv, match=3, mismatch=-1, gap=1) == want


def test_conversion_relations_exhaustive_len4():
    """Every pair of reads of length <= 4 (default scores; the score S from the brute force,
    which shares nothing with the DP):
      * dmax - dmin = |la - lb| (both subtract the same S);
      * dmin = 0 exactly when the shorter read occurs in the longer one gap-free;
      * dnorm = 0 exactly when dmax = 0, dnorm = 65535 exactly when S = 0 and a read is
        non-empty, and dnorm is non-decreasing in dmax among pairs of one longer length;
      * the raw-score reading equals the brute-force score."""
    strings = oracle.brute_strings(4)
    brute = oracle.brute_exhaustive(4)
    rs = synth.from_strings([s.decode() for s in strings])
    n = len(strings)
    pi, pj = (x.ravel() for x in np.meshgrid(np.arange(n), np.arange(n), indexing="ij"))
    got = {c: oracle.pairs(rs, pi, pj, conversion=c).astype(np.int64)
           for c in (oracle.CONV_MAX, oracle.CONV_MIN, oracle.CONV_SCORE, oracle.CONV_NORM)}
    L = np.array([len(s) for s in strings])
    la, lb = L[pi], L[pj]
    S = brute.ravel()
    np.testing.assert_array_equal(got[oracle.CONV_SCORE], S)
    np.testing.assert_array_equal(got[oracle.CONV_MAX] - got[oracle.CONV_MIN], np.abs(la - lb))
    inside = np.array([(strings[x] in strings[y]) if len(strings[x]) <= len(strings[y]) else (strings[y] in strings[x])
                       for x, y in zip(pi, pj)])
    np.testing.assert_array_equal(got[oracle.CONV_MIN] == 0, inside)
    dn, dm = got[oracle.CONV_NORM], got[oracle.CONV_MAX]
    np.testing.assert_array_equal(dn == 0, dm == 0)
    nonempty = np.maximum(la, lb) > 0
    np.testing.assert_array_equal(dn == 65535, (S == 0) & nonempty)
    m = np.maximum(la, lb)
    for mv in range(1, 5):
        sel = m == mv
        order = np.argsort(dm[sel], kind="stable")
        assert np.all(np.diff(dn[sel][order]) >= 0)


@pytest.mark.parametrize("go", [0, 3])
def test_conversion_drivers_agree(go):
    """The triangle, pair-list and rectangle drivers apply the same rule as the single-pair
    function, for every reading, with linear and affine gaps."""
    rs = synth.workload_plain_small().subset(range(12))
    n = rs.n
    pi, pj = np.triu_indices(n, 1)
    for conv in (oracle.CONV_MAX, oracle.CONV_MIN, oracle.CONV_SCORE, oracle.CONV_NORM):
        one = np.array([oracle.distance_conv(rs.read(i), rs.read(j), conv, gap_open=go) for i, j in zip(pi, pj)])
        np.testing.assert_array_equal(oracle.all_pairs(rs, gap_open=go, conversion=conv), one)
        np.testing.assert_array_equal(oracle.pairs(rs, pi, pj, gap_open=go, conversion=conv), one)
        R = oracle.rect(rs, 0, n, rs, 0, n, gap_open=go, conversion=conv)
        np.testing.assert_array_equal(R[pi, pj], one)
