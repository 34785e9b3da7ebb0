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
        # the written bytes per pair: the 2 B output, less what a capture leaves in L2
        assert 1.5 <= tw["dram_bytes_per_pair"] <= per_pair


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_cpu_baseline_leg_checks_what_it_is_given():
    """The bench's oracle leg: timing figures, and the spot check it runs on the GPU's
    values (here the oracle's own values, then one planted error)."""
    import oracle
    from oracle import threshold as oth
    bench = _bench()
    rs = synth.workload_plain_small()
    n = rs.n

    def exact(i, j):
        return oracle.pairs(rs, i, j)

    def one_wrong(i, j):
        d = oracle.pairs(rs, i, j).copy()
        d[0] ^= 1
        return d

    for fn, want in ((exact, 0), (one_wrong, 1)):
        out = bench.cpu_oracle_sample(rs, 0.05, gpu_pairs=fn)
        assert out["kind"] == "oracle" and out["value"] > 0 and out["check"]["mismatches"] == want
        # the check grows past the timed sample to the requested number of pairs
        out = bench.cpu_oracle_sample(rs, 0.05, gpu_pairs=fn, min_check=6000)
        assert out["check"]["pairs_checked"] >= 6000 and out["check"]["mismatches"] == want

    i = np.arange(0, 40)
    j = np.arange(1, 41)
    got = oracle.pairs(rs, i, j)
    assert bench.cpu_baseline_pairs(rs, i, j, got=got)["check"]["mismatches"] == 0
    got[3] += 1
    assert bench.cpu_baseline_pairs(rs, i, j, got=got)["check"]["mismatches"] == 1

    # the batched workload's check: all pairs of small samples, sampled pairs of the others
    samples = [rs.subset(range(0, 30)), rs.subset(range(30, 150))]

    def got_ok(s, i, j):
        return oracle.pairs(samples[s], i, j)

    def got_bad(s, i, j):
        d = oracle.pairs(samples[s], i, j).copy()
        d[-1] ^= 1
        return d

    b = bench.cpu_baseline_batch(samples, got_ok, all_pairs_upto=40, per_sample=100)
    assert b["kind"] == "oracle" and b["check"] == {"pairs_checked": 435 + 100, "mismatches": 0}
    assert bench.cpu_baseline_batch(samples, got_bad, all_pairs_upto=40, per_sample=100)["check"]["mismatches"] == 2

    th = type("T", (), {"num": 6, "den": 100, "abs_max": 65535})()
    tri = oracle.all_pairs(rs)
    labels = oth.components(n, oth.threshold_edges(tri, rs.lengths, 6, 100))
    iu, ju = np.triu_indices(n, 1)
    c = bench.cpu_baseline_components(rs, iu[:500], ju[:500], th, labels)["check"]
    assert c["hit_pairs_split"] == 0 and c["labels_are_roots"]
    bad = labels.copy()
    bad[bad == 0] = 1                 # read 0 loses its root
    assert not bench.cpu_baseline_components(rs, iu[:50], ju[:50], th, bad)["check"]["labels_are_roots"]

    ref = rs.subset(range(20, 150))
    ref_lab = (np.arange(ref.n) % 3).astype(np.int32)
    qs = rs.subset(range(0, 20))
    D = oracle.rect(qs, 0, qs.n, ref, 0, ref.n)
    want_rows = oth.annotate(D, qs.lengths, ref.lengths, ref_lab, 6, 100)
    a = bench.cpu_baseline_annotate(qs, ref, ref_lab, th, want_rows)
    assert a["check"] == {"rows_checked": 20, "mismatches": 0}


def test_cpu_baseline_mds_runs_on_a_small_sample():
    out = _bench().cpu_baseline_mds(1000, 16, 4, 1, n_sample=200)
    assert out["kind"] == "oracle" and out["unit"] == "s" and out["value"] > 0
