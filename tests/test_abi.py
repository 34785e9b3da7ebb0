"""The C-ABI library loads and exports every symbol include/gbd.h declares (CPU only:
no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbd.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(gbd_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1803_02272_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["gbd_create", "gbd_load_reads", "gbd_all_pairs", "gbd_tile", "gbd_batch",
                 "gbd_server_create", "gbd_server_submit", "gbd_server_poll",
                 "gbd_server_wait", "gbd_last_error"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_symbol():
    from paper_1803_02272_gb300 import gbd
    assert sorted(gbd.EXPORTS) == _declared()


def test_default_params_and_errors_without_gpu():
    from paper_1803_02272_gb300 import gbd
    assert gbd.gbd_params_size() == ctypes.sizeof(gbd.GbdParams)
    p = gbd.gbd_default_params()
    assert (p.match, p.mismatch, p.gap, p.conversion, p.kernel) == (1, -1, 1, 0, 0)
    assert (p.gap_open, p.band_entries, p.hbm_budget, p.timeout_us) == (0, 0, 0, 0)
    bad = gbd.gbd_default_params()
    bad.gap = -1
    with pytest.raises(gbd.GbdError) as ei:
        gbd.gbd_create(0, bad)
    assert ei.value.code == gbd.GBD_EINVAL
    assert "gap" in gbd.gbd_last_error()


def test_library_is_sm103a_only():
    from paper_1803_02272_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_probe_op_names_match_header():
    """The binding's probe names are the header's GBD_PROBE_* codes, in code order."""
    from paper_1803_02272_gb300 import gbd
    codes = {}
    for m in re.finditer(r"#define GBD_PROBE_(\w+)\s+(\d+)", open(HEADER).read()):
        codes[m.group(1)] = int(m.group(2))
    count = codes.pop("COUNT")
    assert sorted(codes.values()) == list(range(count))
    assert [name for name, _ in sorted(codes.items(), key=lambda kv: kv[1])] == gbd.PROBE_OPS


def test_default_build_has_no_bounds_checks():
    """The debug entry points exist in the default library and report that its kernels
    carry no checks (the checked library is a separate build)."""
    from paper_1803_02272_gb300 import gbd
    v = ctypes.c_uint64(0)
    assert gbd._lib.gbd_bounds_check(ctypes.byref(v)) == gbd.GBD_ENOTFOUND
    assert v.value == (1 << 64) - 1
    assert gbd._lib.gbd_debug_output_limit(None, 5) == gbd.GBD_EINVAL
