"""Host-side logic that needs no GPU: the seeded input generator and the benchmark's
reference arm (the oracle timed on the host cores, one JSON line)."""
import json
import os
import subprocess
import sys

import numpy as np

from paper_1803_02272_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_splitmix64_reference_outputs():
    # the first outputs of SplitMix64 (Steele, Lea and Flood's generator as given in
    # Vigna's reference C code) started at seed 1234567
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(x) for x in synth.splitmix64_sequence(1234567, 5)] == want


def test_streams_are_reproducible_and_distinct():
    a = synth.Stream(7, 0).u64((1000,))
    assert np.array_equal(a, synth.Stream(7, 0).u64((1000,)))
    assert not np.array_equal(a, synth.Stream(7, 1).u64((1000,)))
    u = synth.Stream(7, 2).uniform((200000,))
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005
    x = synth.Stream(7, 3).integers(250, 450, (200000,))
    assert x.min() == 250 and x.max() == 450


def test_paper_scale_recipe_shape():
    rs = synth.workload_paper_scale(n=2000)
    L = rs.lengths
    assert rs.n == 2000 and L.min() >= 250 and L.max() <= 450
    assert set(np.unique(rs.seq).tolist()) <= set(b"ACGT")


def test_bench_reference_arm_prints_one_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "300",
                          "--steps", "1", "--warmup", "1", "--cpu-seconds", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["value"] > 0 and rec["higher_is_better"] is True
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] >= 1
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["d2h_bytes_per_step"] == 0
    assert rec["config"]["n_reads"] == 300


def test_bench_triangle_write_and_traffic_figures():
    sys.path.insert(0, ROOT)
    import bench
    tw = bench.triangle_write(10**9, 2.0)
    assert tw["algorithmic_gbs"] == 1.0
    per_pair = bench.traffic_value("dram_bytes_per_pair")
    if per_pair is not None:          # the kernel sources still match the profiled ones
        assert per_pair >= 2.0 and bench.traffic_per_launch(10) == per_pair * 10
        assert tw["dram_bytes_per_pair"] >= 2.0
