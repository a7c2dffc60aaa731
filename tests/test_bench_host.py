"""Host-side helpers of the benchmark, on CPU: stream statistics read from the block headers agree with
the oracle's parse, the workload generators honour their stated distributions, and the serving arrival
schedule is seeded and Poisson-shaped."""
import numpy as np

import bench
import oracle
import synth


def test_stream_stats_agree_with_the_oracle_parse():
    x = synth.make("text", 2_500_000, 7)
    comp = oracle.encode(x, block_log2=18, min_emit=6)
    st = bench.stream_stats(comp)
    r, L, s, _ = oracle.parse(comp)[:4]
    assert st["N"] == x.size and st["C"] == comp.size
    assert st["lit_bytes"] == int(r.sum()) and st["match_bytes"] == int(L.sum())
    assert st["n_match"] == int((L > 0).sum())
    assert st["max_depth"] == int(oracle.depths(comp).max())
    assert st["n_blocks"] == (x.size + (1 << 18) - 1) >> 18


def test_kernel_bytes_are_the_stated_formulas():
    """The method's bytes per launch (stream read once, output written once, match sources read once); the
    wavefront path's own per-match records are reported apart."""
    st = dict(C=100, N=1000, match_bytes=600, lit_bytes=400, n_match=50)
    assert bench.kernel_bytes("k_flat", st) == 100 + 1000 + 600
    assert bench.kernel_bytes("k_parse", st) == 100 + 1000
    assert bench.kernel_bytes("k_flow", st) == 2 * 600
    assert bench.kernel_bytes("k_wave", st) == 2 * 600
    assert bench.kernel_bytes("unknown", st) == 0.0
    assert bench.metadata_bytes("k_flow", st) == 28 * 50 and bench.metadata_bytes("k_flat", st) == 0.0


def test_batch_and_reference_configs_agree():
    """Both arms of the bench print the same config for a workload; the batch's decoded bytes come from
    the payload sizes alone."""
    specs, which, N = bench.batch_plan_specs(0)
    assert len(which) == bench.BATCH_STREAMS and len(specs) == bench.BATCH_UNIQUE
    assert N == sum(specs[u][1] for u in which)
    assert all(enc == bench.FLAT[k] for k, _, _, enc in specs)
    assert bench.batch_config(1, N)["decoded_bytes"] == N
    assert set(bench.EXTRAS) <= set(bench.WORKLOADS)


def test_reference_sample_uses_the_oracle_only():
    """The reference arm's sample is encoded by the oracle, with the workload's parameters, and is the
    workload's own input (a block-aligned prefix): it decodes back to it."""
    import argparse
    import sys
    args = argparse.Namespace(workload="small", gpus=1, size=0, batch_streams=4096)
    pool, cfg, sample = bench._reference_sample(args)
    assert cfg == bench.single_config(args, 1)
    (x, comp), = pool
    assert np.array_equal(oracle.decode(comp), x)
    assert np.array_equal(x, synth.make("markov", x.size, bench.stream_seed("markov", 0)))
    # in a process of its own, the reference arm's sampling never imports the product package
    import subprocess
    code = ("import argparse, sys, bench; "
            "bench._reference_sample(argparse.Namespace(workload='small', gpus=1, size=0, batch_streams=4096)); "
            "assert 'paper_2606_04268_gb300' not in sys.modules, 'product imported'")
    r = subprocess.run([sys.executable, "-c", code], cwd=bench.ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]


def test_batch_mix_follows_its_distribution():
    mix = synth.batch_mix(4096, seed=4000)
    sizes = np.array([n for _, n, _ in mix])
    kinds = [k for k, _, _ in mix]
    assert sizes.min() >= 4096 and sizes.max() <= 64 << 20
    assert abs(np.median(sizes) / (1 << 20) - 1.0) < 0.1          # median 1 MiB
    assert 6.5 < sizes.sum() / 2**30 < 9.5                          # ~8 GiB over 4096 streams
    share = {k: kinds.count(k) / len(kinds) for k in ("text", "fastq", "random")}
    assert abs(share["random"] - 0.08) < 0.02 and abs(share["text"] - 0.46) < 0.04
    assert len({sd for _, _, sd in mix}) == len(mix)                # every stream its own seed


def test_serve_mix_and_schedule():
    mix = synth.serve_mix(2000, seed=5000)
    sizes = np.array([n for _, n, _ in mix])
    assert sizes.min() >= 64 * 1024 and sizes.max() <= 256 << 20
    lg = np.log(sizes)
    assert abs(np.median(lg) - (np.log(64 * 1024) + np.log(256 << 20)) / 2) < 0.3   # log-uniform
    assert {k for k, _, _ in mix} == {"text", "fastq", "rle7"}
    a1, w1 = bench._serve_schedule(5000, 32, 1000.0, 9)
    a2, w2 = bench._serve_schedule(5000, 32, 1000.0, 9)
    assert np.array_equal(a1, a2) and np.array_equal(w1, w2)        # seeded
    gaps = np.diff(a1)
    assert a1[0] == 0 and (gaps >= 0).all()
    assert abs(gaps.mean() - 1e-3) < 1e-4                            # rate 1000 per second
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1                 # exponential gaps
    assert w1.min() >= 0 and w1.max() < 32


def test_parallel_cpu_baseline_legs():
    """The bench's block-parallel CPU figures: one queue over a batch of streams, and streams one at a time;
    both decode the streams exactly (the batch leg checks its first pass against the inputs)."""
    xs = [synth.make(k, n, 60 + i) for i, (k, n) in enumerate([("text", 300_000), ("fastq", 200_000),
                                                               ("random", 5_000), ("rle7", 0)])]
    cs = [oracle.encode(x, block_log2=16, tile_log2=12, flatten=2, min_emit=6) for x in xs]
    for batch in (True, False):
        line = bench._cpu_par_line(cs, xs, 0.2, "test streams", batch=batch)
        assert line["value"] > 0 and line["cores"] >= 1 and line["unit"] == "GB/s"
        assert ("queue" in line["kind"]) == batch
