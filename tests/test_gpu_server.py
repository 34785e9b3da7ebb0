"""Serving (continuous batching over a resident reference set) vs the oracle (GPU)."""
import numpy as np
import pytest

import oracle
from paper_1803_02272_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    torch.cuda.set_device(0)
    from paper_1803_02272_gb300 import gbd
    ref_rs = synth.workload_plain_10k(n=3000)
    ctx = gbd.Context(0)
    ref = ctx.load(ref_rs)
    return gbd, ctx, ref, ref_rs


def _queries(seed, sizes):
    reqs = synth.workload_served_queries(len(sizes), rate_per_s=100.0, seed=seed, nq_hi=8)
    out = []
    for q, n in zip(reqs, sizes):
        st = synth.Stream(seed, n)
        anc = synth.random_codes(st, (3, 450))
        out.append(synth.reads_from_ancestors(st, anc, n, 250, 450, 0.05, 0.015))
    return out


def test_single_request_matches_oracle(env):
    import torch
    gbd, ctx, ref, ref_rs = env
    srv = gbd.Server(ctx, ref)
    q = _queries(1, [5])[0]
    t, out = srv.submit(q)
    srv.wait(t)
    torch.cuda.synchronize()
    got = gbd.as_uint16(out)
    cols = np.arange(0, ref_rs.n, 7)
    want = oracle.rect(q, 0, q.n, ref_rs.subset(cols), 0, len(cols))
    np.testing.assert_array_equal(got[:, cols], want)
    srv.close()


@pytest.mark.parametrize("conv", ["min", "norm"])
def test_server_conversions_match_oracle(env, conv):
    """A server of a context with another score-to-distance rule returns that rule's rows."""
    import torch
    gbd, _, _, ref_rs = env
    cg, co = {"min": (gbd.GBD_CONV_MIN, oracle.CONV_MIN), "norm": (gbd.GBD_CONV_NORM, oracle.CONV_NORM)}[conv]
    ctx = gbd.Context(0, conversion=cg)
    sub = ref_rs.subset(range(0, 600))
    srv = gbd.Server(ctx, ctx.load(sub))
    q = _queries(5, [7])[0]
    t, out = srv.submit(q)
    srv.wait(t)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(gbd.as_uint16(out), oracle.rect(q, 0, q.n, sub, 0, sub.n, conversion=co))
    srv.close()


def test_rows_identical_alone_and_mixed(env):
    """Each request's rows are byte-identical whether it runs alone or among others."""
    import torch
    gbd, ctx, ref, ref_rs = env
    qs = _queries(2, [1, 17, 3, 64, 9, 2])
    srv = gbd.Server(ctx, ref)
    alone = []
    for q in qs:
        t, out = srv.submit(q)
        srv.wait(t)
        alone.append(gbd.as_uint16(out).copy())
    tickets = [srv.submit(q) for q in qs]             # all at once: admitted together
    done = [False] * len(qs)
    while not all(done):
        for i, (t, _) in enumerate(tickets):
            if not done[i]:
                done[i] = srv.poll(t)
    torch.cuda.synchronize()
    for a, (_, out) in zip(alone, tickets):
        np.testing.assert_array_equal(gbd.as_uint16(out), a)
    # and every row against the regular rectangle entry point
    for q, a in zip(qs, alone):
        qs_h = ctx.load(q)
        ref_rows = gbd.as_uint16(ctx.tile(qs_h, 0, q.n, ref, 0, ref.n))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(a, ref_rows)
    srv.close()


def test_budget_rejects_and_queues(env):
    import torch
    gbd, _, _, ref_rs = env
    per_query = ref_rs.n * 2
    ctx = gbd.Context(0, hbm_budget=int(per_query * 40))
    ref = ctx.load(ref_rs)
    srv = gbd.Server(ctx, ref)
    big = _queries(3, [64])[0]                        # 64 rows never fit a 40-row budget
    with pytest.raises(gbd.GbdError) as ei:
        srv.submit(big)
    assert ei.value.code == gbd.GBD_EBUDGET
    small = _queries(4, [30, 30, 30])                 # fit one at a time: they queue
    tk = [srv.submit(q) for q in small]
    for t, _ in tk:
        srv.wait(t)
    torch.cuda.synchronize()
    for q, (_, out) in zip(small, tk):
        cols = np.arange(0, ref_rs.n, 97)
        want = oracle.rect(q, 0, q.n, ref_rs.subset(cols), 0, len(cols))
        np.testing.assert_array_equal(gbd.as_uint16(out)[:, cols], want)
    srv.close()


def test_wait_timeout_then_completion(env):
    """A wait with a tiny limit returns ETIMEDOUT (host-side bound), the ticket stays
    valid and the request completes later."""
    import torch
    gbd, _, _, ref_rs = env
    ctx = gbd.Context(0, timeout_us=1)
    ref = ctx.load(ref_rs)
    srv = gbd.Server(ctx, ref)
    q = _queries(5, [256])[0]
    t, out = srv.submit(q)
    with pytest.raises(gbd.GbdError) as ei:
        srv.wait(t)
    assert ei.value.code == gbd.GBD_ETIMEDOUT
    while not srv.poll(t):
        pass
    with pytest.raises(gbd.GbdError) as ei:           # a finished ticket is reported once
        srv.poll(t)
    assert ei.value.code == gbd.GBD_ENOTFOUND
    torch.cuda.synchronize()
    srv.close()


def test_bad_request_rejected(env):
    gbd, ctx, ref, _ = env
    srv = gbd.Server(ctx, ref)
    with pytest.raises(gbd.GbdError) as ei:
        srv.submit(synth.from_strings(["ACGTN"]))
    assert ei.value.code == gbd.GBD_EINVAL
    srv.close()


def test_affine_server_rows_match_oracle(env):
    """A server on a context with affine gaps (systolic kernel, gap open 3)."""
    import torch
    gbd, _, _, ref_rs = env
    ctx = gbd.Context(0, gap_open=3)
    sub = ref_rs.subset(range(400))
    ref = ctx.load(sub)
    srv = gbd.Server(ctx, ref)
    q = _queries(11, [6])[0]
    t, out = srv.submit(q)
    srv.wait(t)
    torch.cuda.synchronize()
    got = gbd.as_uint16(out)
    want = oracle.rect(q, 0, q.n, sub, 0, sub.n, gap_open=3)
    np.testing.assert_array_equal(got, want)
    srv.close()


def test_full_reference_sampled():
    """A request against the paper-scale resident reference (10^5 reads): sampled rows and
    columns against the oracle."""
    import torch
    from paper_1803_02272_gb300 import gbd
    ref_rs = synth.workload_paper_scale()
    ctx = gbd.Context(0)
    ref = ctx.load(ref_rs)
    srv = gbd.Server(ctx, ref)
    q = synth.workload_served_queries(1, 1.0, seed=1005, nq_hi=64)[0].reads
    t, out = srv.submit(q)
    srv.wait(t)
    torch.cuda.synchronize()
    got = gbd.as_uint16(out)
    rng = np.random.default_rng(7)
    rows = rng.integers(0, q.n, size=min(q.n, 4))
    cols = rng.integers(0, ref_rs.n, size=500)
    for r in rows:
        want = oracle.pairs(q, np.full(len(cols), r), cols, ref_rs)
        np.testing.assert_array_equal(got[r, cols], want)
    srv.close()
