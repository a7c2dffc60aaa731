"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* round trip: decode(encode(x)) == x for every generator, flatten mode and depth cap;
* agreement with the textbook relative-distance LZ77 decoder (§2) on the same parse (§3.1 equivalence);
* brute force: every legal parse of every tiny string decodes to that string (separate file);
* invariants the paper fixes: sources precede destinations (§3.1), flattened sources are literal bytes
  (§3.3, global and within-block), depth cap honoured (§7.4), header depths equal an independent depth
  computation (§7.1); every return code of oracle_check is made to fire by a planted violation;
* a stream whose depth fields understate its matches' depths is rejected by the decoder (ERR_DEPTH);
* malformed streams are rejected with the error code the stream format assigns (format §5).
"""
import numpy as np
import pytest

import oracle
import synth
from stream_edit import block_offsets, lower_depths, set_depths

KINDS = ["markov", "text", "fastq", "random", "rle7"]
MODES = [dict(flatten=0), dict(flatten=1), dict(flatten=2), dict(depth_cap=4), dict(depth_cap=1),
         dict(flatten=2, min_emit=6), dict(depth_cap=4, min_emit=6)]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mode", MODES, ids=lambda m: "-".join(f"{k}{v}" for k, v in m.items()))
def test_round_trip_and_invariants(kind, mode):
    x = synth.make(kind, 300_000, 17)
    for bl, tl in ((20, 14), (12, 6), (16, 16)):
        comp = oracle.encode(x, block_log2=bl, tile_log2=tl, **mode)
        assert np.array_equal(oracle.decode(comp), x)
        assert oracle.check(comp) == 0
        dep = oracle.depths(comp)
        info = oracle.peek(comp)
        assert info.max_depth == (int(dep.max()) if dep.size else 0)
        if mode.get("flatten") == 2:
            assert info.max_depth <= 1
        if mode.get("depth_cap"):
            assert info.max_depth <= mode["depth_cap"]


@pytest.mark.parametrize("kind", KINDS)
def test_relative_decoder_agrees(kind):
    x = synth.make(kind, 200_000, 5)
    comp = oracle.encode(x, block_log2=14, tile_log2=9)
    r, L, s, lits = oracle.parse(comp)
    d = np.cumsum(r + L) - L
    dist = np.where(L > 0, d - s, 0)
    assert np.all(s[L > 0] < d[L > 0])
    assert np.array_equal(oracle.lz77_rel_decode(r, L, dist, lits, x.size), x)


def _explicit_depths(r, L, s):
    """Depth as the longest path in the explicit dependency DAG (match -> matches writing its source)."""
    spans, pos = [], 0
    for ri, li, si in zip(r.tolist(), L.tolist(), s.tolist()):
        pos += ri
        if li:
            spans.append((pos, pos + li, si))
            pos += li
    memo = {}

    def depth(i):
        if i in memo:
            return memo[i]
        d0, d1, si = spans[i]
        eff_end = si + min(d1 - d0, d0 - si)
        writers = [j for j in range(i) if spans[j][0] < eff_end and si < spans[j][1]]
        memo[i] = 1 + max((depth(j) for j in writers), default=0)
        return memo[i]

    return [depth(i) for i in range(len(spans))]


@pytest.mark.parametrize("kind", ["markov", "rle7", "text"])
def test_depth_equals_dag_longest_path(kind):
    x = synth.make(kind, 6000, 3)
    comp = oracle.encode(x, block_log2=10, tile_log2=4)
    r, L, s, _ = oracle.parse(comp)
    assert list(oracle.depths(comp)) == _explicit_depths(r, L, s)


def test_flatten_invariant_detects_violation():
    """A stream flagged as globally flattened whose match reads a match byte breaks invariant 4."""
    x = np.frombuffer(b"abcdabcdabcdXabcd", dtype=np.uint8)
    # match 1 copies bytes 4..7 (written by match 0): depth 2 under the 'global' flag
    comp = oracle.serialize(x, [4, 13], [0, 4], [8, 4], flatten=2, block_log2=6, tile_log2=3)
    assert oracle.check(comp) == 4
    ok = oracle.serialize(x, [4, 13], [0, 0], [8, 4], flatten=2, block_log2=6, tile_log2=3)
    assert oracle.check(ok) == 0 and np.array_equal(oracle.decode(ok), x)


def test_depth_cap_violation_detected():
    x = np.frombuffer(b"abab" * 8, dtype=np.uint8)
    comp = oracle.serialize(x, [2], [0], [30], depth_cap=1, block_log2=6, tile_log2=3)
    assert oracle.check(comp) == 0                               # overlap on literals: depth 1
    comp2 = oracle.serialize(x, [2, 16], [0, 8], [14, 16], depth_cap=1, block_log2=6, tile_log2=3)
    assert oracle.check(comp2) == 6                              # second match reads depth-1 bytes


def test_empty_and_tiny():
    for n in (0, 1, 2, 3, 4, 5, 15, 16, 17):
        x = synth.make("rle7", n, 1)
        comp = oracle.encode(x, block_log2=4, tile_log2=2)
        assert np.array_equal(oracle.decode(comp), x)
        assert oracle.check(comp) == 0


def _good():
    x = synth.make("text", 5000, 9)
    return x, oracle.encode(x, block_log2=11, tile_log2=8)


def _mut(comp, off, width, value):
    c = comp.copy()
    c[off:off + width] = np.frombuffer(int(value).to_bytes(width, "little"), np.uint8)
    return c


def test_malformed_streams_rejected():
    x, comp = _good()
    info = oracle.peek(comp)
    assert oracle.decode_rc(comp)[0] == 0
    assert oracle.decode_rc(_mut(comp, 0, 4, 0x12345678))[0] == -2          # magic
    assert oracle.decode_rc(_mut(comp, 4, 2, 2))[0] == -2                   # version
    assert oracle.decode_rc(_mut(comp, 6, 2, 3))[0] == -2                   # flags
    assert oracle.decode_rc(_mut(comp, 8, 1, 30))[0] == -2                  # block_log2
    assert oracle.decode_rc(comp, out_len=x.size + 1)[0] == -3              # out_len != N
    assert oracle.decode_rc(comp[:-16])[0] == -3                            # truncated
    assert oracle.decode_rc(_mut(comp, 24, 8, info.n_blocks + 1))[0] == -2  # n_blocks
    b1 = int.from_bytes(bytes(comp[72:80]), "little")
    assert oracle.decode_rc(_mut(comp, 72, 8, b1 + 16))[0] == -2            # block index
    b0 = int.from_bytes(bytes(comp[64:72]), "little")
    assert oracle.decode_rc(_mut(comp, b0 + 20, 1, 9))[0] == -2             # off width
    assert oracle.decode_rc(_mut(comp, b0 + 32 + 20 + 16, 4, 1))[0] == -2   # sync entry 1 out_pos
    # a match whose absolute source does not precede it
    r, L, s, _ = oracle.parse(comp)
    w = comp[b0 + 20]
    n_tiles = int.from_bytes(bytes(comp[b0 + 28:b0 + 32]), "little")
    cmd_bytes = int.from_bytes(bytes(comp[b0 + 12:b0 + 16]), "little")
    len_bytes = int.from_bytes(bytes(comp[b0 + 16:b0 + 20]), "little")
    a16 = lambda v: (v + 15) & ~15
    o_off = b0 + a16(a16(a16(32 + 20 * n_tiles) + cmd_bytes) + len_bytes)
    d0 = int(r[0])
    bad = _mut(comp, o_off, int(w), min(d0 + 1, (1 << (8 * int(w))) - 1))
    assert oracle.decode_rc(bad)[0] == -4


# ---------------------------------------------------------------------------------------------- depth fields
_set_depths, lower_depths = set_depths, lower_depths


# two blocks of 16 bytes; block 0: (d 4, s 0, L 4) depth 1 and (d 9, s 0, L 4) depth 1; block 1: (d 20, s 4,
# L 4) reads match bytes of block 0, depth 2
_X2 = np.frombuffer(b"abcdabcdXabcdYYYZZZZabcdQQQQQQQQ", dtype=np.uint8)


def test_block_flatten_invariant_detects_violation():
    """Within-block flattening (§3.3): a match may read match bytes of an earlier block, never of its own."""
    ok = oracle.serialize(_X2, [4, 9, 20], [0, 0, 4], [4, 4, 4], flatten=1, block_log2=4, tile_log2=2)
    assert oracle.check(ok) == 0 and np.array_equal(oracle.decode(ok), _X2)
    assert list(oracle.depths(ok)) == [1, 1, 2]
    bad = oracle.serialize(_X2, [4, 9, 20], [0, 4, 4], [4, 4, 4], flatten=1, block_log2=4, tile_log2=2)
    assert oracle.check(bad) == 5
    assert np.array_equal(oracle.decode(bad), _X2)            # a valid stream, only the flag is wrong
    # the same parse under the global flag breaks invariant 4 first (the read from block 0's match)
    glob = oracle.serialize(_X2, [4, 9, 20], [0, 0, 4], [4, 4, 4], flatten=2, block_log2=4, tile_log2=2)
    assert oracle.check(glob) == 4


def test_header_depth_fields_checked():
    """Block max_depth fields must equal the recomputed depths (§7.1): over- and understatement."""
    comp = oracle.serialize(_X2, [4, 9, 20], [0, 0, 4], [4, 4, 4], block_log2=4, tile_log2=2)
    assert oracle.peek(comp).max_depth == 2 and oracle.check(comp) == 0
    over = _set_depths(comp, [1, 3], 3)
    assert oracle.check(over) == 2
    assert oracle.decode_rc(over)[0] == 0                      # overstating is harmless to a decoder
    over0 = _set_depths(comp, [2, 2], 2)
    assert oracle.check(over0) == 2
    under = _set_depths(comp, [1, 1], 1)
    assert oracle.check(under) == 2
    assert oracle.decode_rc(under)[0] == -8                    # ERR_DEPTH
    zero = _set_depths(comp, [0, 2], 2)                        # block 0 has matches, field says none
    assert oracle.decode_rc(zero)[0] == -8
    # the stream field must still be the largest block field, else the stream is malformed
    assert oracle.decode_rc(_set_depths(comp, [1, 2], 1))[0] == -2


def test_depth_lie_reported_after_other_errors():
    """ERR_DEPTH is the last check of a stream: a format error anywhere else wins."""
    x = synth.make("text", 40_000, 4)
    comp = oracle.encode(x, block_log2=12, tile_log2=8)
    assert oracle.peek(comp).max_depth >= 2
    lie = lower_depths(comp, 1)
    assert oracle.decode_rc(lie)[0] == -8
    offs = block_offsets(lie)
    bad = _mut(lie, offs[-1] + 32 + 20 + 16, 4, 1)             # last block, sync entry 1 out_pos
    assert oracle.decode_rc(bad)[0] == -2


@pytest.mark.parametrize("kind", ["text", "markov", "rle7"])
def test_depth_lie_on_generated_streams(kind):
    """Depth-2 streams (cap 2) whose fields are lowered to 1 are rejected; cap-1 streams are not."""
    x = synth.make(kind, 200_000, 6)
    comp = oracle.encode(x, block_log2=14, tile_log2=10, depth_cap=2)
    assert oracle.peek(comp).max_depth == 2
    assert oracle.decode_rc(lower_depths(comp, 1))[0] == -8
    flat = oracle.encode(x, block_log2=14, tile_log2=10, flatten=2)
    assert oracle.decode_rc(lower_depths(flat, 1))[0] == 0
