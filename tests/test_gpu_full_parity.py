"""Every pair of the 10^4-read workload (49,995,000 distances) against the oracle.

The oracle needs about ten minutes of all host cores for this triangle, so the test runs
only when GBD_FULL_PARITY=1 is set; it prints one summary line (pairs compared,
mismatches, oracle time and host threads).  Distances are integers: the bar is exact
equality on every pair."""
import os
import time

import numpy as np
import pytest

import oracle
from paper_1803_02272_gb300 import synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("GBD_FULL_PARITY") != "1",
                                 reason="full-size oracle comparison: set GBD_FULL_PARITY=1")]


def test_10k_workload_every_pair():
    import torch
    torch.cuda.set_device(0)
    from paper_1803_02272_gb300 import gbd
    rs = synth.workload_plain_10k()
    n = rs.n
    ctx = gbd.Context(0)
    tri = gbd.as_uint16(ctx.all_pairs(ctx.load(rs)))
    torch.cuda.synchronize()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    want = oracle.all_pairs(rs, nthreads=cores)
    dt = time.perf_counter() - t0
    bad = int(np.count_nonzero(tri != want))
    print(f"\nFULL_PARITY workload=10k reads={n} pairs={len(want)} mismatches={bad} "
          f"cells={rs.total_cells():.4e} oracle_s={dt:.1f} host_threads={cores}")
    assert len(want) == n * (n - 1) // 2 and bad == 0
