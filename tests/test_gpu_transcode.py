"""On-device transcoding into a globally chain-flattened stream (chain flattening §3.3 applied to an existing
stream): the GPU result equals the oracle's transcode byte for byte (integer and byte work: exact), decodes
to the input on the one-pass path, and a malformed stream is rejected with the oracle's status."""
import random

import numpy as np
import pytest
import torch

import oracle
import paper_2606_04268_gb300 as ax
import synth
from gpu_util import first_diff, gpu_decode, to_dev
from test_oracle_brute import random_parse

pytestmark = pytest.mark.gpu

CASES = [
    ("text", 3_000_000, dict()),                                      # deep chains, several blocks
    ("text", 1_500_000, dict(block_log2=12, tile_log2=8)),            # small blocks and tiles, ragged tail
    ("fastq", 2_000_000, dict(depth_cap=4, min_emit=12, long_bits=20)),
    ("rle7", 700_001, dict()),                                        # self-overlapping repeats
    ("markov", 900_000, dict(flatten=1, block_log2=14, tile_log2=10)),  # block-mode flattened input
    ("text", 800_000, dict(flatten=2)),                               # already flattened: a fixed point
    ("random", 300_000, dict()),                                      # few or no matches
    ("text", 1, dict()), ("text", 17, dict()), ("fastq", 0, dict()),
    ("text", 600_000, dict(min_match=1, block_log2=10, tile_log2=4)),  # every match length allowed
    ("text", 400_000, dict(tile_log2=13, block_log2=16)),             # tiles larger than the one-pass kernel's
]


def _check(comp, x):
    want = oracle.transcode_flat(comp)
    got = ax.transcode_flat(to_dev(comp)).cpu().numpy()
    assert got.size == want.size and np.array_equal(got, want), first_diff(got, want)
    rc, dec = gpu_decode(got, x.size)
    assert rc == 0 and np.array_equal(dec, x)
    info = ax.peek_header(got[:64])
    assert info.max_depth <= 1 and info.flatten == 2
    return got


@pytest.mark.parametrize("i", range(len(CASES)), ids=[f"{k}-{n}" for k, n, _ in CASES])
def test_transcode_matches_oracle(i):
    kind, n, kw = CASES[i]
    x = synth.make(kind, n, 300 + i)
    _check(oracle.encode(x, **kw), x)


def test_transcode_of_random_parses():
    """Arbitrary legal parses (not greedy ones), min_match 1..3, blocks of 16 bytes."""
    rng = random.Random(11)
    for t in range(60):
        n = rng.randint(20, 400)
        s = bytes(rng.choice(b"aabc") for _ in range(n))
        mm = 1 + t % 3
        parse = [m for m in random_parse(s, 16, rng) if m[2] >= mm]
        a = np.frombuffer(s, dtype=np.uint8)
        comp = oracle.serialize(a, [m[0] for m in parse], [m[1] for m in parse], [m[2] for m in parse],
                                block_log2=4, tile_log2=2, min_match=mm)
        _check(comp, a)


def test_transcode_rejects_malformed_stream_like_oracle():
    x = synth.make("text", 500_000, 3)
    comp = oracle.encode(x)
    bad = comp.copy()
    b0 = int.from_bytes(bytes(bad[64:72]), "little")
    bad[b0 + 32 + 20 + 4] ^= 3      # a sync entry's cmd offset
    rc_o = oracle.transcode_flat_rc(bad)[0]
    assert rc_o != 0
    with pytest.raises(ax.AceapexError) as e:
        ax.transcode_flat(to_dev(bad))
    assert e.value.code == rc_o


def test_transcode_then_one_pass_decode_is_faster_path():
    """The transcoded deep stream takes the one-pass kernel (the library's path choice by max_depth)."""
    x = synth.make("text", 2_000_000, 8)
    comp = oracle.encode(x)
    assert oracle.peek(comp).max_depth > 1
    t = ax.transcode_flat(to_dev(comp))
    info = ax.peek_header(t[:64].cpu().numpy())
    assert info.max_depth == 1 and info.tile_log2 <= 12
    out = torch.empty(x.size, dtype=torch.uint8, device="cuda")
    ax.profile(True)
    ax.decode(t, out)
    prof = ax.profile_read()
    ax.profile(False)
    assert torch.equal(out.cpu(), torch.from_numpy(x))
    assert prof.get("k_flat", (0, 0))[1] >= 1 and prof.get("k_flow", (0, 0))[1] == 0
