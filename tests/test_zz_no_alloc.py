"""The allocation-free entry point gbd_tile_noalloc, for callers that cannot call
cudaMalloc (their device memory belongs to another allocator, or the code path must not
allocate).  Its output must equal the regular gbd_tile entry point's on two calls in a
row -- the scratch array is shared between calls, so the second call (smaller, other
reads) would expose state left over from the first.  Distances are integers: the bar is
exact equality.  After a first call on the device (which looks up the array's address),
a call must leave the device's free memory and torch's reserved memory unchanged.
This file is collected last on purpose."""
import gc

import numpy as np
import pytest

from paper_1803_02272_gb300 import synth

pytestmark = pytest.mark.gpu


def _device_reads(torch, rs):
    seq = torch.from_numpy(rs.seq if rs.seq.size else np.zeros(1, np.uint8)).cuda()
    off = torch.from_numpy(rs.offsets.view(np.int64).copy()).cuda()
    return seq, off


def test_noalloc_matches_tile_on_two_calls():
    import torch
    torch.cuda.set_device(0)
    from paper_1803_02272_gb300 import gbd
    ctx = gbd.Context(0)
    work = synth.workload_plain_10k(n=700)
    cases = [(work.subset(range(0, 300)), work.subset(range(300, 700))),
             (work.subset(range(650, 700)), synth.from_strings(["", "ACGT", "acgtac"] +
                                                               [work.read(i) for i in range(5)]))]
    calls = 0
    for A, B in cases + cases[:1]:
        nA, nB = A.n, B.n
        ld = nB + 3
        seqA, offA = _device_reads(torch, A)
        seqB, offB = _device_reads(torch, B)
        out = torch.full((nA * ld,), -1, dtype=torch.int16, device="cuda:0")
        max_len = int(max(A.lengths.max(), B.lengths.max()))
        torch.cuda.synchronize()
        gc.collect()
        gc.disable()                                   # no set is freed while memory is measured
        try:
            free0, reserved0 = torch.cuda.mem_get_info(0)[0], torch.cuda.memory_reserved(0)
            gbd.gbd_tile_noalloc(ctx.handle, seqA, offA, nA, seqB, offB, nB, max_len, out, ld)
            torch.cuda.synchronize()
            free1, reserved1 = torch.cuda.mem_get_info(0)[0], torch.cuda.memory_reserved(0)
        finally:
            gc.enable()
        if calls:                                      # the first call on a device may set up
            assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"
            assert reserved1 == reserved0
        calls += 1
        ref = ctx.tile(ctx.load(A), 0, nA, ctx.load(B), 0, nB)
        torch.cuda.synchronize()
        got = gbd.as_uint16(out).reshape(nA, ld)
        np.testing.assert_array_equal(got[:, :nB], gbd.as_uint16(ref))
        assert np.all(got[:, nB:] == 0xFFFF)          # columns past nB are left untouched


def test_noalloc_rejects_oversized_and_bad_input():
    import torch
    torch.cuda.set_device(0)
    from paper_1803_02272_gb300 import gbd
    ctx = gbd.Context(0)
    A = synth.from_strings(["ACGTACGT", "ACG"])
    seqA, offA = _device_reads(torch, A)
    out = torch.empty(4, dtype=torch.int16, device="cuda:0")
    with pytest.raises(gbd.GbdError) as ei:            # read longer than max_len
        gbd.gbd_tile_noalloc(ctx.handle, seqA, offA, 2, seqA, offA, 2, 4, out, 2)
    assert ei.value.code == gbd.GBD_EINVAL
    bad = synth.from_strings(["ACGT", "ACNT"])
    seqX, offX = _device_reads(torch, bad)
    with pytest.raises(gbd.GbdError) as ei:            # non-ACGT byte
        gbd.gbd_tile_noalloc(ctx.handle, seqX, offX, 2, seqA, offA, 2, 8, out, 2)
    assert ei.value.code == gbd.GBD_EINVAL
    with pytest.raises(gbd.GbdError) as ei:            # more than the 32 MiB array holds
        gbd.gbd_tile_noalloc(ctx.handle, seqA, offA, 2, seqA, offA, 600000, 65535, out, 600000)
    assert ei.value.code == gbd.GBD_EINVAL


def test_noalloc_rejects_bad_offsets_and_null_reads():
    """Decreasing offsets are rejected before any kernel reads the bytes with them, and a
    NULL read buffer is rejected on the host."""
    import torch
    torch.cuda.set_device(0)
    from paper_1803_02272_gb300 import gbd
    ctx = gbd.Context(0)
    A = synth.from_strings(["ACGTACGT", "ACG", "TTT"])
    seqA, offA = _device_reads(torch, A)
    bad_off = torch.from_numpy(np.array([0, 8, 2, 14], dtype=np.int64)).cuda()   # read 1 runs backwards
    out = torch.empty(9, dtype=torch.int16, device="cuda:0")
    with pytest.raises(gbd.GbdError) as ei:
        gbd.gbd_tile_noalloc(ctx.handle, seqA, bad_off, 3, seqA, offA, 3, 16, out, 3)
    assert ei.value.code == gbd.GBD_EINVAL
    assert "read 1 of A" in gbd.gbd_last_error()
    with pytest.raises(gbd.GbdError) as ei:
        gbd.gbd_tile_noalloc(ctx.handle, seqA, offA, 3, None, offA, 3, 16, out, 3)
    assert ei.value.code == gbd.GBD_EINVAL
    # the entry point is still usable after the rejections
    gbd.gbd_tile_noalloc(ctx.handle, seqA, offA, 3, seqA, offA, 3, 16, out, 3)
    ref = ctx.tile(ctx.load(A), 0, 3, ctx.load(A), 0, 3)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(gbd.as_uint16(out).reshape(3, 3), gbd.as_uint16(ref))
