"""The bounds-checked debug build (libgbd_check.so, compiled with -DGBD_BOUNDS_CHECK=1).

It replaces the memory checker that cannot run on this hardware's pool: every distance
store, every index into the general kernel's boundary rows and every shared-memory access
window of the systolic kernel is checked against its buffer, an out-of-range access is
skipped and the smallest such index is recorded.  The tests run the checked library on the
small workload, edge-length reads and a rectangle (results exact, nothing recorded), then
cap the output extent below the real one and check that exactly the stores past the cap
are skipped and that the cap itself is the recorded index.  Nothing here faults: the
checked build never performs the out-of-range stores."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1803_02272_gb300 import synth

pytestmark = pytest.mark.gpu

NONE = (1 << 64) - 1
SITE_SYSTOLIC_OUT, SITE_GENERAL_OUT = 1, 3


@pytest.fixture(scope="module")
def chk():
    import torch
    torch.cuda.set_device(0)
    from paper_1803_02272_gb300 import build, gbd
    return gbd, gbd.load_library(build.build(check=True))


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _ctx(gbd, lib, **kw):
    p = gbd.GbdParams()
    lib.gbd_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    assert lib.gbd_create(ctypes.byref(h), 0, ctypes.byref(p)) == 0, lib.gbd_last_error()
    return h.value


def _load(lib, ctx, rs):
    seq = rs.seq if rs.seq.size else np.zeros(1, np.uint8)
    off = np.ascontiguousarray(rs.offsets, dtype=np.uint64)
    h = ctypes.c_void_p()
    assert lib.gbd_load_reads(ctx, seq.ctypes.data, off.ctypes.data, rs.n, ctypes.byref(h), _stream()) == 0
    return h.value


def _violation(lib):
    v = ctypes.c_uint64()
    assert lib.gbd_bounds_check(ctypes.byref(v)) == 0, lib.gbd_last_error()
    return v.value


def _all_pairs(gbd, lib, ctx, rs):
    import torch
    m = rs.n * (rs.n - 1) // 2
    tri = torch.full((m,), -1, dtype=torch.int16, device="cuda:0")
    assert lib.gbd_all_pairs(ctx, _load(lib, ctx, rs), tri.data_ptr(), m, _stream()) == 0, lib.gbd_last_error()
    torch.cuda.synchronize()
    return gbd.as_uint16(tri)


def _edge_reads():
    st = synth.Stream(4343, 0)
    reads = ["", "A", "ACGT", "T" * 33]
    for L in (15, 16, 17, 31, 32, 33, 300, 511, 512, 513, 700):
        reads.append("".join("ACGT"[c] for c in synth.random_codes(st, (L,))))
    return reads


@pytest.mark.parametrize("kernel", ["auto", "general"])
def test_checked_build_is_exact_and_records_nothing(chk, kernel):
    import torch
    gbd, lib = chk
    k = gbd.GBD_KERNEL_AUTO if kernel == "auto" else gbd.GBD_KERNEL_GENERAL
    ctx = _ctx(gbd, lib, kernel=k)
    _violation(lib)                                    # start from a clear word
    for rs in (synth.workload_plain_small(), synth.from_strings(_edge_reads())):
        np.testing.assert_array_equal(_all_pairs(gbd, lib, ctx, rs), oracle.all_pairs(rs))
    rs = synth.workload_plain_10k(n=260)
    A, B = rs.subset(range(0, 100)), rs.subset(range(100, 260))
    ld = B.n + 5
    out = torch.full((A.n * ld,), -1, dtype=torch.int16, device="cuda:0")
    assert lib.gbd_tile(ctx, _load(lib, ctx, A), 0, A.n, _load(lib, ctx, B), 0, B.n, out.data_ptr(), ld,
                        _stream()) == 0
    torch.cuda.synchronize()
    got = gbd.as_uint16(out).reshape(A.n, ld)
    np.testing.assert_array_equal(got[:, :B.n], oracle.rect(A, 0, A.n, B, 0, B.n))
    assert _violation(lib) == NONE
    lib.gbd_destroy(ctx)


@pytest.mark.parametrize("kernel,site", [("auto", SITE_SYSTOLIC_OUT), ("general", SITE_GENERAL_OUT)])
def test_checked_build_skips_and_records_stores_past_the_extent(chk, kernel, site):
    """With the output extent capped 100 entries short of the triangle, the last 100
    entries are never written, the others are exact, and the recorded violation is the
    cap (the smallest skipped index) at the kernel's store site."""
    gbd, lib = chk
    k = gbd.GBD_KERNEL_AUTO if kernel == "auto" else gbd.GBD_KERNEL_GENERAL
    ctx = _ctx(gbd, lib, kernel=k)
    rs = synth.workload_plain_small().subset(range(60))      # lengths 280-320: systolic rows only
    m = rs.n * (rs.n - 1) // 2
    cap = m - 100
    _violation(lib)
    assert lib.gbd_debug_output_limit(ctx, cap) == 0
    got = _all_pairs(gbd, lib, ctx, rs)
    v = _violation(lib)
    assert v >> 56 == site and v & ((1 << 56) - 1) == cap
    np.testing.assert_array_equal(got[:cap], oracle.all_pairs(rs)[:cap])
    assert np.all(got[cap:] == 0xFFFF)                 # never written
    assert lib.gbd_debug_output_limit(ctx, 0) == 0     # the real extent again: nothing recorded
    np.testing.assert_array_equal(_all_pairs(gbd, lib, ctx, rs), oracle.all_pairs(rs))
    assert _violation(lib) == NONE
    lib.gbd_destroy(ctx)
