"""Pre-scan CPU/GPU choice on the GPU machine: for streams the rule sends either way (measured CPU rate of
the block-parallel CPU decoder on this host), both decodes -- GPU through the C ABI, CPU through the
block-parallel decoder -- reproduce the input byte for byte, whichever the rule picked."""
import os
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2606_04268_gb300 as ax
import synth
from gpu_util import gpu_decode

pytestmark = pytest.mark.gpu


def test_both_choices_decode_exactly():
    ax.build()
    oracle.build()
    cases = [("fastq", 24 << 20, dict(flatten=2, min_emit=12, long_bits=20, chain_limit=4)),   # large, shallow
             ("text", 3 << 20, dict(block_log2=12, tile_log2=8)),                              # deep chains
             ("rle7", 20_000, dict(flatten=2))]                                                # tiny
    # measured CPU rate: the block-parallel decoder on all host cores (best of three, after a first call
    # that loads the decoder)
    x0 = synth.make("text", 8 << 20, 1)
    c0 = oracle.encode(x0, flatten=2, min_emit=6)
    assert oracle.cpupar_decode_rc(c0, threads=os.cpu_count())[0] == 0
    best = float("inf")
    for _ in range(3):
        t = time.perf_counter()
        assert oracle.cpupar_decode_rc(c0, threads=os.cpu_count())[0] == 0
        best = min(best, time.perf_counter() - t)
    cpu_gbps = x0.size / best / 1e9
    picks = []
    for kind, n, kw in cases:
        x = synth.make(kind, n, 9)
        comp = oracle.encode(x, **kw)
        info = ax.peek_header(comp[:64])
        which, tc, tg = ax.choose_device(info, cpu_gbps)
        assert which == ("gpu" if tg < tc else "cpu") and tc == pytest.approx(x.size / (cpu_gbps * 1e9))
        picks.append(which)
        rc, got = gpu_decode(comp, x.size)
        assert rc == 0 and np.array_equal(got, x), kind
        rc2, got2 = oracle.cpupar_decode_rc(comp, threads=os.cpu_count())
        assert rc2 == 0 and np.array_equal(got2, x), kind
    # 20 KB: the fixed GPU overhead (30 us) dominates at any CPU rate above 20 KB / 30 us
    assert cpu_gbps < 0.7 or picks[2] == "cpu", cpu_gbps
    assert picks[0] == "gpu", cpu_gbps  # 24 MiB one-pass: the GPU unless the host decodes at > 260 GB/s
