"""The block-parallel CPU decoder (threads over blocks in stream order, paper §3.1) against the oracle's
sequential decode, byte for byte, on every generator and encoder mode, with block sizes that give many
blocks and chains that cross blocks; and on the degenerate cases (empty, one byte, one block)."""
import numpy as np
import pytest

import oracle
import synth

KINDS = ["markov", "text", "fastq", "random", "rle7"]
MODES = [dict(), dict(flatten=1), dict(flatten=2, min_emit=6), dict(depth_cap=4, min_emit=6),
         dict(flatten=2, min_emit=12, long_bits=16, chain_limit=4)]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mode", MODES, ids=lambda m: "-".join(f"{k}{v}" for k, v in m.items()) or "plain")
def test_parallel_decode_equals_oracle(kind, mode):
    x = synth.make(kind, 700_000, 23)
    for bl, tl in ((14, 10), (16, 12), (20, 12)):
        comp = oracle.encode(x, block_log2=bl, tile_log2=tl, **mode)
        ref = oracle.decode(comp)
        for threads in (1, 3, 8, 64):
            rc, got = oracle.cpupar_decode_rc(comp, threads=threads)
            assert rc == 0 and np.array_equal(got, ref), (bl, threads, rc)


def test_deep_cross_block_chains():
    """Unflattened text with tiny blocks: most matches read earlier blocks that other threads decode."""
    x = synth.make("text", 2_000_000, 5)
    comp = oracle.encode(x, block_log2=10, tile_log2=6)
    assert oracle.peek(comp).max_depth > 50
    for threads in (2, 16):
        rc, got = oracle.cpupar_decode_rc(comp, threads=threads)
        assert rc == 0 and np.array_equal(got, x)


@pytest.mark.parametrize("n", [0, 1, 3, 16, 4096, 4097])
def test_tiny_and_empty(n):
    x = synth.make("rle7", n, 2)
    comp = oracle.encode(x, block_log2=12, tile_log2=6)
    rc, got = oracle.cpupar_decode_rc(comp, threads=4)
    assert rc == 0 and np.array_equal(got, x)


def test_rejects_wrong_size_and_bad_stream():
    x = synth.make("text", 50_000, 1)
    comp = oracle.encode(x, block_log2=12)
    assert oracle.cpupar_decode_rc(comp, out_len=x.size + 1, threads=2)[0] == -3
    bad = comp.copy()
    bad[0] ^= 1
    assert oracle.cpupar_decode_rc(bad, out_len=x.size, threads=2)[0] == -2
    # a match whose source does not precede it
    r, L, s, _ = oracle.parse(comp)
    b0 = int.from_bytes(bytes(comp[64:72]), "little")
    w = int(comp[b0 + 20])
    n_tiles = int.from_bytes(bytes(comp[b0 + 28:b0 + 32]), "little")
    cmd_bytes = int.from_bytes(bytes(comp[b0 + 12:b0 + 16]), "little")
    len_bytes = int.from_bytes(bytes(comp[b0 + 16:b0 + 20]), "little")
    a16 = lambda v: (v + 15) & ~15
    o_off = b0 + a16(a16(a16(32 + 20 * n_tiles) + cmd_bytes) + len_bytes)
    bad2 = comp.copy()
    bad2[o_off:o_off + w] = np.frombuffer(min(int(r[0]) + 1, (1 << (8 * w)) - 1).to_bytes(w, "little"), np.uint8)
    assert oracle.cpupar_decode_rc(bad2, threads=2)[0] == -4
