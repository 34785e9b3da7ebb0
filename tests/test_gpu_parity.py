"""CUDA path vs the CPU oracle, element by element (GPU).

Distances are integers, so the bar is bit-exact equality on every compared pair.
Every call goes through the C ABI (libgbd.so) via the thin binding.
"""
import numpy as np
import pytest

import oracle
from paper_1803_02272_gb300 import synth

pytestmark = pytest.mark.gpu

KERNELS = ["auto", "general", "systolic"]


@pytest.fixture(scope="module")
def gbd():
    import torch
    torch.cuda.set_device(0)
    from paper_1803_02272_gb300 import gbd as g
    return g


def _ctx(gbd, kernel="auto", **kw):
    k = {"auto": gbd.GBD_KERNEL_AUTO, "general": gbd.GBD_KERNEL_GENERAL,
         "systolic": gbd.GBD_KERNEL_SYSTOLIC}[kernel]
    return gbd.Context(0, kernel=k, **kw)


def _all_pairs(gbd, ctx, rs):
    import torch
    s = ctx.load(rs)
    out = ctx.all_pairs(s)
    torch.cuda.synchronize()
    return gbd.as_uint16(out)


@pytest.mark.parametrize("kernel", KERNELS)
def test_small_workload_all_pairs_exact(gbd, kernel):
    """150 reads (lengths 280-320): all 11,175 distances bit-exact."""
    rs = synth.workload_plain_small()
    got = _all_pairs(gbd, _ctx(gbd, kernel), rs)
    want = oracle.all_pairs(rs)
    assert got.shape == want.shape == (11175,)
    np.testing.assert_array_equal(got, want)


def _edge_reads():
    st = synth.Stream(4242, 0)
    reads = ["", "A", "C", "ACGT", "A" * 15, "A" * 16, "A" * 17, "T" * 31, "T" * 32, "T" * 33,
             "ACGT" * 8, "acgtACGT" * 3, "G" * 64]
    for L in [1, 2, 3, 15, 16, 17, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257,
              300, 449, 450, 511, 512, 513, 700]:
        reads.append("".join("ACGT"[c] for c in synth.random_codes(st, (L,))))
    base = "".join("ACGT"[c] for c in synth.random_codes(st, (400,)))
    reads += [base, base[:200], base[100:350], base[::-1]]
    return reads


@pytest.mark.parametrize("kernel", ["auto", "general"])
def test_edge_lengths_exact(gbd, kernel):
    """Empty reads, word-boundary lengths (15/16/17, 31/32/33...), homopolymers, a read
    inside another, lengths around 512 and beyond (those pairs go to the general kernel)."""
    rs = synth.from_strings(_edge_reads())
    got = _all_pairs(gbd, _ctx(gbd, kernel), rs)
    np.testing.assert_array_equal(got, oracle.all_pairs(rs))


@pytest.mark.parametrize("n", [0, 1, 2, 3, 33])
def test_tiny_sets(gbd, n):
    rs = synth.workload_plain_small().subset(range(n))
    ctx = _ctx(gbd)
    got = _all_pairs(gbd, ctx, rs) if n >= 2 else None
    if n >= 2:
        np.testing.assert_array_equal(got, oracle.all_pairs(rs))
    else:
        s = ctx.load(rs)
        assert s.n == n
        gbd.gbd_all_pairs(ctx.handle, s.handle, None, 0)


def test_tile_rectangle_exact(gbd):
    import torch
    rs = synth.workload_plain_10k(n=400)
    ctx = _ctx(gbd)
    A = ctx.load(rs.subset(range(0, 150)))
    B = ctx.load(rs.subset(range(150, 400)))
    out = ctx.tile(A, 7, 140, B, 3, 241, ld=250)
    torch.cuda.synchronize()
    got = gbd.as_uint16(out)[:, :238]
    want = oracle.rect(rs.subset(range(0, 150)), 7, 140, rs.subset(range(150, 400)), 3, 241)
    np.testing.assert_array_equal(got, want)


def test_symmetry_tile_both_orders(gbd):
    import torch
    rs = synth.workload_plain_10k(n=300)
    ctx = _ctx(gbd)
    A = ctx.load(rs.subset(range(0, 120)))
    B = ctx.load(rs.subset(range(120, 300)))
    ab = gbd.as_uint16(ctx.tile(A, 0, 120, B, 0, 180))
    ba = gbd.as_uint16(ctx.tile(B, 0, 180, A, 0, 120))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ab, ba.T)


def test_invalid_byte_rejected(gbd):
    ctx = _ctx(gbd)
    rs = synth.from_strings(["ACGT", "ACNT", "GG"])
    with pytest.raises(gbd.GbdError) as ei:
        ctx.load(rs)
    assert ei.value.code == gbd.GBD_EINVAL
    assert "position 6" in gbd.gbd_last_error()


def test_wrong_triangle_length_rejected(gbd):
    import torch
    ctx = _ctx(gbd)
    s = ctx.load(synth.workload_plain_small().subset(range(10)))
    out = torch.empty(44, dtype=torch.int16, device="cuda:0")
    with pytest.raises(gbd.GbdError) as ei:
        gbd.gbd_all_pairs(ctx.handle, s.handle, out, 44)
    assert ei.value.code == gbd.GBD_EINVAL


def test_device_input_pointers(gbd):
    """Reads given as device tensors (torch) instead of host arrays."""
    import torch
    rs = synth.workload_plain_small().subset(range(40))
    ctx = _ctx(gbd)
    seq = torch.from_numpy(rs.seq).cuda()
    off = torch.from_numpy(rs.offsets.astype(np.int64)).cuda()
    s = ctx.load_reads(seq, off)
    tri = gbd.as_uint16(ctx.all_pairs(s))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(tri, oracle.all_pairs(rs))


@pytest.mark.parametrize("scores", [(2, -3, 2), (1, -2, 3)])
def test_other_scores_raw_score_mode(gbd, scores):
    m, x, g = scores
    rs = synth.workload_plain_small().subset(range(30))
    ctx = _ctx(gbd, "auto", match=m, mismatch=x, gap=g, conversion=gbd.GBD_CONV_SCORE)
    got = _all_pairs(gbd, ctx, rs)
    n = rs.n
    pi, pj = np.triu_indices(n, 1)
    want = oracle.pair_scores(rs, pi, pj, match=m, mismatch=x, gap=g)
    np.testing.assert_array_equal(got.astype(np.int64), want)


@pytest.mark.parametrize("scores", [(1, -1, 1, 2), (2, -3, 1, 3), (1, -2, 2, 1)])
def test_affine_gaps_exact(gbd, scores):
    """Affine gaps (gap_open > 0) on the general kernel against the oracle's Gotoh mode:
    distances of the 150-read workload, and raw scores of edge-length reads."""
    import torch
    m, x, g, go = scores
    rs = synth.workload_plain_small()
    ctx = _ctx(gbd, "auto", match=m, mismatch=x, gap=g, gap_open=go)
    got = _all_pairs(gbd, ctx, rs)
    np.testing.assert_array_equal(got, oracle.all_pairs(rs, match=m, mismatch=x, gap=g, gap_open=go))
    edge = synth.from_strings(_edge_reads()[:30])
    ctx2 = _ctx(gbd, "auto", match=m, mismatch=x, gap=g, gap_open=go, conversion=gbd.GBD_CONV_SCORE)
    got2 = _all_pairs(gbd, ctx2, edge)
    pi, pj = np.triu_indices(edge.n, 1)
    want2 = oracle.pair_scores(edge, pi, pj, match=m, mismatch=x, gap=g, gap_open=go)
    np.testing.assert_array_equal(got2.astype(np.int64), want2)


def test_affine_gap_limits(gbd):
    _ctx(gbd, "systolic", gap_open=1000)            # the systolic kernel's largest opening
    with pytest.raises(gbd.GbdError):
        _ctx(gbd, "systolic", gap_open=1001)
    with pytest.raises(gbd.GbdError):
        _ctx(gbd, "auto", gap_open=-1)


@pytest.mark.parametrize("go", [2, 7])
def test_affine_systolic_batch_and_tile(gbd, go):
    """Affine gaps on the systolic kernel through the batched launch and a rectangle."""
    import torch
    samples = synth.workload_batched(n_samples=4, n_lo=20, n_hi=150)
    ctx = _ctx(gbd, "systolic", gap_open=go)
    sets = [ctx.load(s) for s in samples]
    outs = ctx.batch(sets)
    torch.cuda.synchronize()
    for rs, o in zip(samples, outs):
        np.testing.assert_array_equal(gbd.as_uint16(o), oracle.all_pairs(rs, gap_open=go))
    A, B = samples[0], samples[1]
    out = ctx.tile(sets[0], 0, A.n, sets[1], 0, B.n)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(gbd.as_uint16(out), oracle.rect(A, 0, A.n, B, 0, B.n, gap_open=go))


def test_batch_matches_per_sample(gbd):
    import torch
    samples = synth.workload_batched(n_samples=5, n_lo=20, n_hi=120)
    ctx = _ctx(gbd)
    sets = [ctx.load(s) for s in samples]
    outs = ctx.batch(sets)
    torch.cuda.synchronize()
    for rs, o in zip(samples, outs):
        np.testing.assert_array_equal(gbd.as_uint16(o), oracle.all_pairs(rs))


def test_batch_autotuner(gbd):
    """The first five calls time one candidate each (work-unit scales 1, 0.5, 2 with two
    streams, then the best scale with one and three streams), then the fastest is kept;
    every call's output is exact."""
    import torch
    samples = synth.workload_batched(n_samples=6, n_lo=50, n_hi=400)
    ctx = _ctx(gbd)
    sets = [ctx.load(s) for s in samples]
    outs = [torch.empty(max(s.n * (s.n - 1) // 2, 1), dtype=torch.int16, device="cuda") for s in samples]
    want = [oracle.all_pairs(rs) for rs in samples]
    states = []
    for call in range(8):
        for o in outs:
            o.fill_(-1)
        ctx.batch(sets, outs=outs)
        torch.cuda.synchronize()
        for rs, o, w in zip(samples, outs, want):
            np.testing.assert_array_equal(gbd.as_uint16(o[: rs.n * (rs.n - 1) // 2]), w)
        states.append(gbd.gbd_batch_tuning(ctx.handle))
    assert not states[0]["done"] and not states[4]["done"] and states[5]["done"] and states[7]["done"]
    assert states[0]["chosen"] == -1
    st = states[7]
    t = st["trial_ms"]
    assert len(t) == 5 and all(x > 0 for x in t)
    assert st["piece_scale"][:3] == [1.0, 0.5, 2.0] and st["streams"] == [2, 2, 2, 1, 3]
    best_scale = [1.0, 0.5, 2.0][int(np.argmin(t[:3]))]
    assert st["piece_scale"][3] == st["piece_scale"][4] == best_scale
    assert st["chosen"] == int(np.argmin(t))


def test_batch_graph_replay_and_recapture(gbd):
    """gbd_batch records its launch group as a CUDA graph: a second call with the same
    samples and outputs replays it, other outputs re-record it; results stay exact."""
    import torch
    samples = synth.workload_batched(n_samples=6, n_lo=30, n_hi=200)
    ctx = _ctx(gbd)
    sets = [ctx.load(s) for s in samples]
    outs = ctx.batch(sets)
    n0 = gbd.gbd_kernel_launches()
    for o in outs:
        o.fill_(-1)
    ctx.batch(sets, outs=outs)                 # replay
    torch.cuda.synchronize()
    assert gbd.gbd_kernel_launches() > n0
    for rs, o in zip(samples, outs):
        np.testing.assert_array_equal(gbd.as_uint16(o), oracle.all_pairs(rs))
    outs2 = ctx.batch(sets[::-1])              # different samples order: re-recorded
    torch.cuda.synchronize()
    for rs, o in zip(samples[::-1], outs2):
        np.testing.assert_array_equal(gbd.as_uint16(o), oracle.all_pairs(rs))


def test_10k_workload_sampled(gbd):
    """10^4 reads (5.0e7 pairs): the whole triangle on the GPU, 20,000 seeded pairs
    checked against the oracle, plus every pair of the first and last 40 reads."""
    import torch
    rs = synth.workload_plain_10k()
    n = rs.n
    ctx = _ctx(gbd)
    s = ctx.load(rs)
    tri = gbd.as_uint16(ctx.all_pairs(s))
    torch.cuda.synchronize()
    st = synth.Stream(5151, 0)
    i = st.integers(0, n - 2, (20000,))
    j = i + 1 + np.floor(st.uniform((20000,)) * (n - 1 - i)).astype(np.int64)
    k = i * n - i * (i + 1) // 2 + (j - i - 1)
    np.testing.assert_array_equal(tri[k], oracle.pairs(rs, i, j))
    for block in (range(0, 40), range(n - 40, n)):
        b = np.array(block)
        bi, bj = np.triu_indices(len(b), 1)
        ii, jj = b[bi], b[bj]
        kk = ii * n - ii * (ii + 1) // 2 + (jj - ii - 1)
        np.testing.assert_array_equal(tri[kk], oracle.pairs(rs, ii, jj))


@pytest.mark.parametrize("go", [0, 2, 9])
def test_systolic_every_rows_per_lane(go):
    """Query lengths 1..512 cover every rows-per-lane variant (R = 1..16) of the
    systolic kernel, with subjects shorter and longer than the query; linear gaps
    (go = 0) and affine gaps."""
    import torch
    from paper_1803_02272_gb300 import gbd as g
    st = synth.Stream(8080, 0)
    reads = []
    for L in list(range(1, 40)) + [63, 64, 65, 95, 96, 97] + list(range(100, 513, 29)) + [511, 512]:
        reads.append("".join("ACGT"[c] for c in synth.random_codes(st, (L,))))
    base = reads[-1]
    reads += [base[5:300], base[:128] + "ACGT" * 10, base[200:]]
    rs = synth.from_strings(reads)
    ctx = _ctx(g, "systolic", gap_open=go)
    got = _all_pairs(g, ctx, rs)
    np.testing.assert_array_equal(got, oracle.all_pairs(rs, gap_open=go))


@pytest.mark.parametrize("go", [0, 3])
def test_long_subject_rebases(go):
    """A 20,000-base subject streams past short queries: the DP values are rebased many
    times inside one subject."""
    import torch
    from paper_1803_02272_gb300 import gbd as g
    st = synth.Stream(9090, 0)
    long = "".join("ACGT"[c] for c in synth.random_codes(st, (20000,)))
    reads = [long[1000:1300], long[15000:15450], long[19900:], "ACGT" * 50, long]
    rs = synth.from_strings(reads)
    got = _all_pairs(g, _ctx(g, "auto", gap_open=go), rs)
    np.testing.assert_array_equal(got, oracle.all_pairs(rs, gap_open=go))
    if go:
        return
    ctx = _ctx(g, "auto")
    A = ctx.load(rs.subset([0, 1, 2, 3]))
    B = ctx.load(rs.subset([4, 4, 0]))
    out = ctx.tile(A, 0, 4, B, 0, 3)
    torch.cuda.synchronize()
    want = oracle.rect(rs.subset([0, 1, 2, 3]), 0, 4, rs.subset([4, 4, 0]), 0, 3)
    np.testing.assert_array_equal(g.as_uint16(out), want)


def test_systolic_rejects_other_scores(gbd):
    with pytest.raises(gbd.GbdError) as ei:
        gbd.Context(0, kernel=gbd.GBD_KERNEL_SYSTOLIC, match=2)
    assert ei.value.code == gbd.GBD_EINVAL


def _tile_pairs(n, r0, r1, c0, c1):
    """Every pair (i, j), i < j, of the block rows [r0, r1) x columns [c0, c1)."""
    ii, jj = np.meshgrid(np.arange(r0, r1), np.arange(c0, c1), indexing="ij")
    keep = ii < jj
    return ii[keep].astype(np.int64), jj[keep].astype(np.int64)


def test_paper_scale_sampled(gbd):
    """The paper-scale workload (10^5 reads, 5.0e9 pairs, the 10 GB triangle) in the launch
    configuration the benchmark times: 20,000 seeded pairs, the whole rows of three reads
    (first, middle, the longest) and four whole 64 x 1024 tiles of the triangle (the first,
    the last, one in the middle and the one of the longest read) checked against the
    oracle; the length bounds hold on every sampled pair."""
    import torch
    rs = synth.workload_paper_scale()
    n = rs.n
    ctx = _ctx(gbd)
    s = ctx.load(rs)
    tri = ctx.all_pairs(s)
    torch.cuda.synchronize()
    rng = np.random.default_rng(2026)
    i = rng.integers(0, n - 1, size=20000)
    j = i + 1 + (rng.random(20000) * (n - 1 - i)).astype(np.int64)
    idx = i * n - i * (i + 1) // 2 + (j - i - 1)
    got = gbd.as_uint16(tri[torch.from_numpy(idx).cuda()])
    want = oracle.pairs(rs, i, j)
    np.testing.assert_array_equal(got, want)
    L = rs.lengths.astype(np.int64)
    assert np.all(got >= np.abs(L[i] - L[j])) and np.all(got <= np.maximum(L[i], L[j]))
    longest = int(np.argmax(L[:-1]))
    for r in (0, n // 2, longest):
        k0 = r * n - r * (r + 1) // 2
        row = gbd.as_uint16(tri[k0:k0 + (n - 1 - r)])
        jj = np.arange(r + 1, n)
        np.testing.assert_array_equal(row, oracle.pairs(rs, np.full(len(jj), r), jj))
    lr = min(max(longest - 32, 0), n - 64)
    tiles = {"first": (0, 64, 1, 1025), "last": (n - 64, n, n - 1024, n),
             "middle": (n // 2, n // 2 + 64, n // 2 + 1, n // 2 + 1025),
             "longest read": (lr, lr + 64, lr + 1, min(lr + 1025, n))}
    for name, (r0, r1, c0, c1) in tiles.items():
        ti, tj = _tile_pairs(n, r0, r1, c0, c1)
        idx = ti * n - ti * (ti + 1) // 2 + (tj - ti - 1)
        got = gbd.as_uint16(tri[torch.from_numpy(idx).cuda()])
        np.testing.assert_array_equal(got, oracle.pairs(rs, ti, tj), err_msg=f"{name} tile")
    del tri


# ------------------------------------------------------------------ score-to-distance rules
# Section 2.2 leaves the conversion of the local score into a dissimilarity open; every
# reading behind gbd_params.conversion is compared with the oracle's mode of the same rule.

CONVERSIONS = ["min", "norm", "score"]


def _conv_codes(gbd, name):
    return {"max": (gbd.GBD_CONV_MAX, oracle.CONV_MAX), "min": (gbd.GBD_CONV_MIN, oracle.CONV_MIN),
            "score": (gbd.GBD_CONV_SCORE, oracle.CONV_SCORE), "norm": (gbd.GBD_CONV_NORM, oracle.CONV_NORM)}[name]


@pytest.mark.parametrize("conv", CONVERSIONS)
@pytest.mark.parametrize("kernel", ["systolic", "general"])
def test_conversions_all_pairs_exact(gbd, kernel, conv):
    """Each conversion on each kernel: the 150-read workload (all 11,175 pairs) and the
    edge-length reads (empty reads, a read inside another, lengths around every word and
    lane boundary and past 512), bit-exact."""
    cg, co = _conv_codes(gbd, conv)
    ctx = _ctx(gbd, kernel, conversion=cg)
    for rs in (synth.workload_plain_small(), synth.from_strings(_edge_reads())):
        got = _all_pairs(gbd, ctx, rs)
        np.testing.assert_array_equal(got, oracle.all_pairs(rs, conversion=co))


@pytest.mark.parametrize("conv", CONVERSIONS)
def test_conversions_affine_exact(gbd, conv):
    """The conversions with affine gaps: on the systolic kernel (open 2 and 9, extend 1)
    and on the general kernel (match 2, mismatch -3, extend 1, open 3)."""
    cg, co = _conv_codes(gbd, conv)
    rs = synth.workload_plain_small().subset(range(90))
    edge = synth.from_strings(_edge_reads()[:30])
    for go in (2, 9):
        ctx = _ctx(gbd, "systolic", gap_open=go, conversion=cg)
        for r in (rs, edge):
            np.testing.assert_array_equal(_all_pairs(gbd, ctx, r), oracle.all_pairs(r, gap_open=go, conversion=co))
    ctx = _ctx(gbd, "auto", match=2, mismatch=-3, gap=1, gap_open=3, conversion=cg)
    for r in (rs, edge):
        np.testing.assert_array_equal(_all_pairs(gbd, ctx, r),
                                      oracle.all_pairs(r, match=2, mismatch=-3, gap=1, gap_open=3, conversion=co))


@pytest.mark.parametrize("conv", CONVERSIONS)
def test_conversions_tile_and_batch_exact(gbd, conv):
    """The conversions through a rectangle (both kernels) and the batched launch."""
    import torch
    cg, co = _conv_codes(gbd, conv)
    rs = synth.workload_plain_10k(n=260)
    A, B = rs.subset(range(0, 100)), rs.subset(range(100, 260))
    for kernel in ("auto", "general"):
        ctx = _ctx(gbd, kernel, conversion=cg)
        out = ctx.tile(ctx.load(A), 3, 97, ctx.load(B), 0, B.n)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(gbd.as_uint16(out), oracle.rect(A, 3, 97, B, 0, B.n, conversion=co))
    samples = synth.workload_batched(n_samples=4, n_lo=20, n_hi=120)
    ctx = _ctx(gbd, "auto", conversion=cg)
    outs = ctx.batch([ctx.load(x) for x in samples])
    torch.cuda.synchronize()
    for x, o in zip(samples, outs):
        np.testing.assert_array_equal(gbd.as_uint16(o), oracle.all_pairs(x, conversion=co))


@pytest.mark.parametrize("kernel", ["auto", "general"])
def test_all_pairs_to_host_bands_exact(gbd, kernel):
    """The triangle computed band by band into host memory: many small bands (a few rows
    each, both staging buffers reused many times), one band, and reads longer than 512
    bases (general-kernel rows inside the bands); equal to the oracle and to the device
    triangle of gbd_all_pairs."""
    ctx = _ctx(gbd, kernel)
    for rs in (synth.workload_plain_small(), synth.from_strings(_edge_reads())):
        s = ctx.load(rs)
        m = rs.n * (rs.n - 1) // 2
        want = oracle.all_pairs(rs)
        for band in (rs.n - 1, 700, 0):
            host = np.full(m, 0xFFFF, dtype=np.uint16)
            gbd.gbd_all_pairs_to_host(ctx.handle, s.handle, host, m, band)
            np.testing.assert_array_equal(host, want)
        np.testing.assert_array_equal(_all_pairs(gbd, ctx, rs), want)


def test_all_pairs_to_host_pinned_10k(gbd):
    """10^4 reads into a page-locked host triangle with 2^22-entry bands (twelve bands):
    identical to the device triangle."""
    import torch
    rs = synth.workload_plain_10k()
    ctx = _ctx(gbd)
    s = ctx.load(rs)
    m = rs.n * (rs.n - 1) // 2
    host = torch.empty(m, dtype=torch.int16, pin_memory=True)
    gbd.gbd_all_pairs_to_host(ctx.handle, s.handle, host, m, 1 << 22)
    dev = gbd.as_uint16(ctx.all_pairs(s))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host.numpy().view(np.uint16), dev)
    with pytest.raises(gbd.GbdError) as ei:
        gbd.gbd_all_pairs_to_host(ctx.handle, s.handle, host, m - 1, 0)
    assert ei.value.code == gbd.GBD_EINVAL
