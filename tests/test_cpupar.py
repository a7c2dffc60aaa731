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
    assert oracle.cpupar_decode_rc(_bad_source_stream(comp), threads=2)[0] == -4


def _bad_source_stream(comp):
    """The stream with block 0's first match given a source that does not precede it."""
    r, L, s, _ = oracle.parse(comp)
    b0 = int.from_bytes(bytes(comp[64:72]), "little")
    w = int(comp[b0 + 20])
    n_tiles = int.from_bytes(bytes(comp[b0 + 28:b0 + 32]), "little")
    cmd_bytes = int.from_bytes(bytes(comp[b0 + 12:b0 + 16]), "little")
    len_bytes = int.from_bytes(bytes(comp[b0 + 16:b0 + 20]), "little")
    a16 = lambda v: (v + 15) & ~15
    o_off = b0 + a16(a16(a16(32 + 20 * n_tiles) + cmd_bytes) + len_bytes)
    bad = comp.copy()
    bad[o_off:o_off + w] = np.frombuffer(min(int(r[0]) + 1, (1 << (8 * w)) - 1).to_bytes(w, "little"), np.uint8)
    return bad


def _batch_pool(seed):
    """Streams of every generator and several encoder modes, many of one or two blocks, some of many, plus
    empty and one-byte streams: (inputs, streams)."""
    rng = np.random.default_rng(seed)
    xs, cs = [], []
    for i in range(40):
        kind = KINDS[i % len(KINDS)]
        mode = MODES[(i // len(KINDS)) % len(MODES)]
        n = int(rng.choice([0, 1, 3000, 60_000, 200_000, 900_000]))
        x = synth.make(kind, n, 100 + i)
        xs.append(x)
        cs.append(oracle.encode(x, block_log2=16, tile_log2=12, **mode))
    return xs, cs


@pytest.mark.parametrize("threads", [1, 4, 16, 64])
def test_batch_decode_equals_oracle(threads):
    xs, cs = _batch_pool(7)
    rc, st, outs = oracle.cpupar_decode_batch_rc(cs, [x.size for x in xs], threads=threads)
    assert rc == 0 and (st == 0).all(), st
    for c, x, o in zip(cs, xs, outs):
        assert np.array_equal(o, oracle.decode(c)) and np.array_equal(o, x)


def test_batch_of_deep_cross_block_streams():
    """Unflattened text with tiny blocks: waits inside each stream while other streams' blocks run."""
    xs = [synth.make("text", 400_000, 30 + k) for k in range(6)]
    cs = [oracle.encode(x, block_log2=10, tile_log2=6) for x in xs]
    rc, st, outs = oracle.cpupar_decode_batch_rc(cs, [x.size for x in xs], threads=16)
    assert rc == 0 and (st == 0).all()
    for x, o in zip(xs, outs):
        assert np.array_equal(o, x)


def test_batch_errors_per_stream_and_first_error_returned():
    x = synth.make("text", 50_000, 1)
    good = oracle.encode(x, block_log2=12)
    bad_magic = good.copy()
    bad_magic[0] ^= 1
    cs = [good, bad_magic, good, good]
    lens = [x.size, x.size, x.size + 1, x.size]
    rc, st, outs = oracle.cpupar_decode_batch_rc(cs, lens, threads=8)
    # the same statuses as one-at-a-time decodes, the good streams still decoded
    assert list(st) == [oracle.cpupar_decode_rc(c, m, threads=2)[0] for c, m in zip(cs, lens)] == [0, -2, -3, 0]
    assert rc == -2
    assert np.array_equal(outs[0], x) and np.array_equal(outs[3], x)


def test_batch_stream_failing_in_its_first_block_does_not_stall_the_others():
    """Block 0 of the middle stream fails; its later blocks, which wait on block 0, are released and
    skipped, and the streams around it decode."""
    x = synth.make("text", 50_000, 1)
    good = oracle.encode(x, block_log2=12)
    cs = [good, _bad_source_stream(good), good]
    for threads in (2, 8):
        rc, st, outs = oracle.cpupar_decode_batch_rc(cs, [x.size] * 3, threads=threads)
        assert rc == -4 and list(st) == [0, -4, 0]
        assert np.array_equal(outs[0], x) and np.array_equal(outs[2], x)


def test_empty_batch():
    rc, st, outs = oracle.cpupar_decode_batch_rc([], [], threads=4)
    assert rc == 0 and st.size == 0 and outs == []
