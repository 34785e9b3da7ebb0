"""Threshold epilogue on the GPU (gbd_tile_hits, gbd_threshold_components) against the
oracle (oracle/threshold.py on distances from the distance oracle).

Integer decisions throughout, so the bar is exact: the same hit set, the same row
annotations, the same component labels (smallest read of each component).
"""
import numpy as np
import pytest

import oracle
from oracle import mds as omds
from oracle import threshold as oth
from paper_1803_02272_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    torch.cuda.set_device(0)
    from paper_1803_02272_gb300 import gbd
    return gbd, torch


@pytest.fixture(scope="module")
def ref_and_queries():
    # 20 sibling ancestors of the paper-scale tree; narrow lengths, so that distances within
    # an ancestor fall under the usual thresholds and the hit lists are rich
    anc = synth.paper_scale_ancestors()[:20]
    ref, ref_lab = synth.reads_from_ancestors(synth.Stream(71, 0), anc, 500, 345, 355, 0.01, 0.003,
                                              return_parents=True)
    qs = synth.reads_from_ancestors(synth.Stream(72, 0), anc, 90, 340, 360, 0.01, 0.003)
    D = oracle.rect(qs, 0, qs.n, ref, 0, ref.n)
    return ref, ref_lab, qs, D


def _ctx(gbd, kernel="auto"):
    k = {"auto": gbd.GBD_KERNEL_AUTO, "general": gbd.GBD_KERNEL_GENERAL}[kernel]
    return gbd.Context(0, kernel=k)


def _hits_of(torch, hits, count, cap):
    n = int(count.cpu().numpy()[0])
    h = hits[: 3 * min(n, cap)].cpu().numpy().view(np.uint32).reshape(-1, 3)
    return n, {(int(a), int(b), int(c)) for a, b, c in h}


@pytest.mark.parametrize("kernel", ["auto", "general"])
@pytest.mark.parametrize("num,den,abs_max", [(3, 100, 65535), (6, 100, 65535), (1, 1, 20), (12, 100, 40)])
def test_tile_hits_and_annotation(env, ref_and_queries, kernel, num, den, abs_max):
    gbd, torch = env
    ref, ref_lab, qs, D = ref_and_queries
    ctx = _ctx(gbd, kernel)
    A, B = ctx.load(qs), ctx.load(ref)
    th = gbd.threshold(num, den, abs_max)
    cap = D.size
    hits = torch.empty(3 * cap, dtype=torch.int32, device="cuda")
    count = torch.empty(1, dtype=torch.int64, device="cuda")
    labs = torch.from_numpy(ref_lab).cuda()
    rows = torch.empty(qs.n, dtype=torch.int32, device="cuda")
    gbd.gbd_tile_hits(ctx.handle, A.handle, 0, qs.n, B.handle, 0, ref.n, th, None, 0, hits, cap, count,
                      labs, rows)
    torch.cuda.synchronize()
    n, got = _hits_of(torch, hits, count, cap)
    want = oth.hits_rect(D, qs.lengths, ref.lengths, num, den, abs_max)
    assert n == len(want)
    assert got == want
    ann = oth.annotate(D, qs.lengths, ref.lengths, ref_lab, num, den, abs_max)
    np.testing.assert_array_equal(rows.cpu().numpy(), ann)


def test_tile_hits_with_dense_output_and_subrange(env, ref_and_queries):
    gbd, torch = env
    ref, ref_lab, qs, D = ref_and_queries
    ctx = _ctx(gbd)
    A, B = ctx.load(qs), ctx.load(ref)
    a0, a1, b0, b1 = 7, 61, 33, 470
    ld = (b1 - b0) + 5
    out = torch.full(((a1 - a0) * ld,), -1, dtype=torch.int16, device="cuda")
    count = torch.empty(1, dtype=torch.int64, device="cuda")
    gbd.gbd_tile_hits(ctx.handle, A.handle, a0, a1, B.handle, b0, b1, gbd.threshold(8, 100), out, ld,
                      None, 0, count)
    torch.cuda.synchronize()
    dense = out.cpu().numpy().view(np.uint16).reshape(a1 - a0, ld)[:, : b1 - b0]
    np.testing.assert_array_equal(dense, D[a0:a1, b0:b1])
    sub = D[a0:a1, b0:b1]
    want = oth.hits_rect(sub, qs.lengths[a0:a1], ref.lengths[b0:b1], 8, 100)
    assert int(count.cpu().numpy()[0]) == len(want)


def test_tile_hits_capacity_overflow(env, ref_and_queries):
    gbd, torch = env
    ref, ref_lab, qs, D = ref_and_queries
    ctx = _ctx(gbd)
    A, B = ctx.load(qs), ctx.load(ref)
    want = oth.hits_rect(D, qs.lengths, ref.lengths, 12, 100)
    cap = len(want) // 3
    assert cap > 0
    hits = torch.empty(3 * cap, dtype=torch.int32, device="cuda")
    count = torch.empty(1, dtype=torch.int64, device="cuda")
    gbd.gbd_tile_hits(ctx.handle, A.handle, 0, qs.n, B.handle, 0, ref.n, gbd.threshold(12, 100), None, 0,
                      hits, cap, count)
    torch.cuda.synchronize()
    n, got = _hits_of(torch, hits, count, cap)
    assert n == len(want) and len(got) == cap and got <= want


def test_tile_hits_rejects(env, ref_and_queries):
    gbd, torch = env
    ref, _, qs, _ = ref_and_queries
    ctx = _ctx(gbd)
    A, B = ctx.load(qs), ctx.load(ref)
    hits = torch.empty(30, dtype=torch.int32, device="cuda")
    for th, kw in [(gbd.threshold(3, 0), {}), (gbd.threshold(), {"d_hits": hits, "hit_capacity": 10})]:
        with pytest.raises(gbd.GbdError) as e:
            gbd.gbd_tile_hits(ctx.handle, A.handle, 0, 5, B.handle, 0, 5, th, **kw)
        assert e.value.code == gbd.GBD_EINVAL


def _components_case(env, rs, num, den, abs_max, kernel="auto", want_tri=False, band_entries=0):
    gbd, torch = env
    k = {"auto": gbd.GBD_KERNEL_AUTO, "general": gbd.GBD_KERNEL_GENERAL}[kernel]
    ctx = gbd.Context(0, kernel=k, band_entries=band_entries)
    s = ctx.load(rs)
    n = rs.n
    labels = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    edges = torch.empty(1, dtype=torch.int64, device="cuda")
    tri = torch.empty(max(n * (n - 1) // 2, 1), dtype=torch.int16, device="cuda") if want_tri else None
    gbd.gbd_threshold_components(ctx.handle, s.handle, gbd.threshold(num, den, abs_max), labels, edges, tri)
    torch.cuda.synchronize()
    return (labels.cpu().numpy()[:n].astype(np.int64), int(edges.cpu().numpy()[0]),
            None if tri is None else tri.cpu().numpy().view(np.uint16)[: n * (n - 1) // 2])


def _clustered_set(n, seed):
    anc = synth.paper_scale_ancestors()[:20]
    return synth.reads_from_ancestors(synth.Stream(seed, 0), anc, n, 340, 360, 0.01, 0.003)


@pytest.mark.parametrize("num,den,abs_max", [(3, 100, 65535), (6, 100, 65535), (1, 1, 12), (100, 100, 0)])
def test_components_match_oracle(env, num, den, abs_max):
    rs = _clustered_set(700, 73)
    tri = oracle.all_pairs(rs)
    lab, ne, _ = _components_case(env, rs, num, den, abs_max)
    edges = oth.threshold_edges(tri, rs.lengths, num, den, abs_max)
    assert ne == len(edges)
    np.testing.assert_array_equal(lab, oth.components(rs.n, edges))


def test_components_with_long_reads_and_dense_triangle(env):
    """Reads longer than the systolic query limit take the general kernel's rows."""
    st = synth.Stream(808, 0)
    base = synth.random_codes(st, (900,))
    reads = []
    for k in range(60):
        L = int(st.integers(300, 900, ()))
        r = base[:L].copy()
        flip = st.integers(0, L - 1, (int(L * 0.03),))
        r[flip] = (r[flip] + 1) % 4
        reads.append("".join("ACGT"[c] for c in r))
    rs = synth.from_strings(reads)
    tri = oracle.all_pairs(rs)
    for kernel in ("auto", "general"):
        lab, ne, dense = _components_case(env, rs, 8, 100, 65535, kernel, want_tri=True)
        edges = oth.threshold_edges(tri, rs.lengths, 8, 100)
        np.testing.assert_array_equal(dense, tri)
        assert ne == len(edges)
        np.testing.assert_array_equal(lab, oth.components(rs.n, edges))


def test_components_tiny_sets(env):
    for strs in ([], ["ACGT"], ["ACGT", "ACGT"], ["ACGT", "TTTT", "ACGA"]):
        rs = synth.from_strings(strs)
        if rs.n == 0:
            continue
        lab, ne, _ = _components_case(env, rs, 1, 1, 1)
        tri = oracle.all_pairs(rs) if rs.n >= 2 else np.zeros(0, np.uint16)
        edges = oth.threshold_edges(tri, rs.lengths, 1, 1, 1)
        assert ne == len(edges)
        np.testing.assert_array_equal(lab, oth.components(rs.n, edges))


def test_tri_components_from_oracle_triangle(env):
    """Components from a triangle the oracle computed (uploaded), several thresholds on
    the same triangle."""
    gbd, torch = env
    rs = _clustered_set(500, 74)
    tri = oracle.all_pairs(rs)
    ctx = _ctx(gbd)
    s = ctx.load(rs)
    d_tri = torch.from_numpy(tri.view(np.int16)).cuda()
    labels = torch.empty(rs.n, dtype=torch.int32, device="cuda")
    edges = torch.empty(1, dtype=torch.int64, device="cuda")
    for num, den, abs_max in [(2, 100, 65535), (5, 100, 65535), (9, 100, 65535), (1, 1, 30)]:
        gbd.gbd_tri_components(ctx.handle, s.handle, d_tri, gbd.threshold(num, den, abs_max), labels, edges)
        torch.cuda.synchronize()
        e = oth.threshold_edges(tri, rs.lengths, num, den, abs_max)
        assert int(edges.cpu().numpy()[0]) == len(e)
        np.testing.assert_array_equal(labels.cpu().numpy().astype(np.int64), oth.components(rs.n, e))


def test_rect_hits_over_oracle_rectangle(env, ref_and_queries):
    """The epilogue alone over a rectangle the oracle computed (uploaded), two rules."""
    gbd, torch = env
    ref, ref_lab, qs, D = ref_and_queries
    ctx = _ctx(gbd)
    A, B = ctx.load(qs), ctx.load(ref)
    a0, a1, b0, b1 = 3, 80, 10, 490
    sub = np.ascontiguousarray(D[a0:a1, b0:b1])
    ld = b1 - b0
    d_rect = torch.from_numpy(sub.view(np.int16).ravel()).cuda()
    cap = sub.size
    hits = torch.empty(3 * cap, dtype=torch.int32, device="cuda")
    count = torch.empty(1, dtype=torch.int64, device="cuda")
    labs = torch.from_numpy(ref_lab).cuda()
    rows = torch.empty(a1 - a0, dtype=torch.int32, device="cuda")
    for num, den, abs_max in [(6, 100, 65535), (1, 1, 15)]:
        gbd.gbd_rect_hits(ctx.handle, A.handle, a0, a1, B.handle, b0, b1, d_rect, ld,
                          gbd.threshold(num, den, abs_max), hits, cap, count, labs, rows)
        torch.cuda.synchronize()
        n, got = _hits_of(torch, hits, count, cap)
        want = {(a0 + i, b0 + j, d) for i, j, d in oth.hits_rect(sub, qs.lengths[a0:a1], ref.lengths[b0:b1],
                                                                   num, den, abs_max)}
        assert n == len(want) and got == want
        ann = oth.annotate(sub, qs.lengths[a0:a1], ref.lengths[b0:b1], ref_lab[b0:b1], num, den, abs_max)
        np.testing.assert_array_equal(rows.cpu().numpy(), ann)


def _lengths_set(st, n, lo, hi):
    """Reads of random lengths in [lo, hi]; the epilogue reads only their lengths."""
    L = st.integers(lo, hi, (n,))
    return synth.from_strings(["A" * int(x) for x in L])


def _near_rule(st, shape, la, lb, num, den, abs_max, p_near):
    """Distances that sit on the decision boundary of the rule with probability p_near
    (the largest hit value plus -1, 0 or +1), else just above it or far above it."""
    L = np.maximum(la, lb).astype(np.int64)
    edge = np.minimum(np.minimum(num * L // den, abs_max), 65535)
    near = st.uniform(shape) < p_near
    off = st.integers(-1, 1, shape)
    above = edge + 1 + st.integers(0, 40, shape)
    far = st.uniform(shape) < 0.5
    d = np.where(near, edge + off, np.where(far, 65535, above))
    return np.clip(d, 0, 65535).astype(np.uint16)


@pytest.mark.parametrize("num,den,abs_max", [(7, 100, 65535), (1, 1, 25), (13, 50, 60)])
def test_rect_hits_long_rows_every_alignment(env, num, den, abs_max):
    """Rows longer than one work unit (20,003 columns), an odd row stride and a start two
    bytes past an alignment boundary, so every row begins at a different offset within
    16 bytes; distances on the rule's boundary.  Hit list and row labels exact."""
    gbd, torch = env
    st = synth.Stream(811, 0)
    nq, nr = 24, 20003
    qs, ref = _lengths_set(st, nq, 30, 700), _lengths_set(st, nr, 30, 700)
    D = _near_rule(st, (nq, nr), qs.lengths[:, None], ref.lengths[None, :], num, den, abs_max, 6e-5)
    ref_lab = st.integers(-1, 4, (nr,)).astype(np.int32)
    ld = nr + 3
    buf = np.full(1 + nq * ld, 7, np.uint16)
    buf[1:].reshape(nq, ld)[:, :nr] = D
    ctx = _ctx(gbd)
    A, B = ctx.load(qs), ctx.load(ref)
    d_buf = torch.from_numpy(buf.view(np.int16)).cuda()
    cap = 4096
    hits = torch.empty(3 * cap, dtype=torch.int32, device="cuda")
    count = torch.empty(1, dtype=torch.int64, device="cuda")
    rows = torch.empty(nq, dtype=torch.int32, device="cuda")
    gbd.gbd_rect_hits(ctx.handle, A.handle, 0, nq, B.handle, 0, nr, d_buf[1:], ld, gbd.threshold(num, den, abs_max),
                      hits, cap, count, torch.from_numpy(ref_lab).cuda(), rows)
    torch.cuda.synchronize()
    n, got = _hits_of(torch, hits, count, cap)
    want = oth.hits_rect(D, qs.lengths, ref.lengths, num, den, abs_max)
    assert 0 < len(want) < cap
    assert n == len(want) and got == want
    ann = oth.annotate(D, qs.lengths, ref.lengths, ref_lab, num, den, abs_max)
    np.testing.assert_array_equal(rows.cpu().numpy(), ann)


@pytest.mark.parametrize("num,den,abs_max", [(3, 100, 65535), (1, 1, 9)])
def test_tri_components_synthetic_triangle(env, num, den, abs_max):
    """A 3,001-read triangle of distances on the rule's boundary (random lengths): long
    rows, row ends inside a lane's eight entries, a partial last vector."""
    gbd, torch = env
    st = synth.Stream(812, 0)
    n = 3001
    rs = _lengths_set(st, n, 20, 900)
    iu, ju = np.triu_indices(n, 1)
    L = rs.lengths
    tri = _near_rule(st, (len(iu),), L[iu], L[ju], num, den, abs_max, 2e-4)
    ctx = _ctx(gbd)
    s = ctx.load(rs)
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    edges = torch.empty(1, dtype=torch.int64, device="cuda")
    gbd.gbd_tri_components(ctx.handle, s.handle, torch.from_numpy(tri.view(np.int16)).cuda(),
                           gbd.threshold(num, den, abs_max), labels, edges)
    torch.cuda.synchronize()
    e = oth.threshold_edges(tri, L, num, den, abs_max)
    assert len(e) > 100
    assert int(edges.cpu().numpy()[0]) == len(e)
    np.testing.assert_array_equal(labels.cpu().numpy().astype(np.int64), oth.components(n, e))


@pytest.mark.parametrize("band_entries", [1, 2000, 40000])
@pytest.mark.parametrize("num,den,abs_max", [(6, 100, 65535), (1, 1, 12)])
def test_components_in_bands(env, band_entries, num, den, abs_max):
    """Without a triangle the graph is built band by band (one row per band, a few rows,
    bands that grow towards the end); labels and edge count as the oracle's."""
    rs = _clustered_set(700, 75)
    tri = oracle.all_pairs(rs)
    lab, ne, _ = _components_case(env, rs, num, den, abs_max, band_entries=band_entries)
    edges = oth.threshold_edges(tri, rs.lengths, num, den, abs_max)
    assert len(edges) > 50
    assert ne == len(edges)
    np.testing.assert_array_equal(lab, oth.components(rs.n, edges))


def test_components_in_bands_long_reads_and_general_kernel(env):
    """Bands with rows longer than the systolic query limit (general kernel rows inside a
    band), and the general kernel for whole bands."""
    st = synth.Stream(809, 0)
    base = synth.random_codes(st, (900,))
    reads = []
    for _ in range(80):
        L = int(st.integers(300, 900, ()))
        r = base[:L].copy()
        flip = st.integers(0, L - 1, (int(L * 0.03),))
        r[flip] = (r[flip] + 1) % 4
        reads.append("".join("ACGT"[c] for c in r))
    rs = synth.from_strings(reads)
    tri = oracle.all_pairs(rs)
    edges = oth.threshold_edges(tri, rs.lengths, 8, 100)
    for kernel in ("auto", "general"):
        lab, ne, _ = _components_case(env, rs, 8, 100, 65535, kernel, band_entries=500)
        assert ne == len(edges)
        np.testing.assert_array_equal(lab, oth.components(rs.n, edges))


@pytest.mark.parametrize("banded", [False, True])
def test_components_edge_list_overflow(env, banded):
    """Every pair a hit (d <= max(la, lb) always holds): more than 64 Mi edges, so the
    edge list overflows and direct unions over the distances take over.  The graph is
    complete: one component labelled 0, n(n-1)/2 edges."""
    gbd, torch = env
    n = 12000
    st = synth.Stream(813, 0)
    rs = synth.from_strings(["".join("ACGT"[c] for c in synth.random_codes(st, (int(st.integers(8, 24, ())),)))
                             for _ in range(n)])
    m = n * (n - 1) // 2
    assert m > 64 << 20
    lab, ne, _ = _components_case(env, rs, 1, 1, 65535, want_tri=not banded)
    assert ne == m
    assert not lab.any()
