"""Pins of the oracle's transcoder (global chain flattening of an existing stream, paper §3.3).

The transcoder traces every match byte to its root (the literal byte it ultimately copies) and rewrites
each match as the maximal runs of consecutive roots, each copying from its root; runs shorter than
min_match become literal bytes, and a self-overlapping match whose effective source is literal is kept.
Pinned by: hand-derived results on small streams (the expected parses are worked out in the comments),
the decoded bytes (oracle_decode, pinned on its own), the flattening invariant (oracle_check code 4 and
depth 1 everywhere), idempotence on streams that are already flattened, and -- on every legal parse of
tiny strings and random parses of longer ones -- root preservation, maximality and the length rule.
"""
import itertools
import random

import numpy as np
import pytest

import oracle
import synth
from test_oracle_brute import all_parses, random_parse


def _parse_list(comp):
    """Matches (d, s, L) of a stream, in destination order."""
    r, L, s, _ = oracle.parse(comp)
    d = np.cumsum(r + L) - L
    return [(int(d[i]), int(s[i]), int(L[i])) for i in range(len(r)) if L[i]]


def _stream(x: bytes, parse, block_log2=5, min_match=1):
    a = np.frombuffer(x, dtype=np.uint8)
    return oracle.serialize(a, [m[0] for m in parse], [m[1] for m in parse], [m[2] for m in parse],
                            block_log2=block_log2, tile_log2=2, min_match=min_match)


# hand-derived cases: (bytes, parse, block_log2, min_match, expected parse of the transcoded stream)
GOLDEN = [
    # a chain: [4,8) copies [0,4) (depth 1), [8,12) copies [4,8) (depth 2) -> both copy from 0
    (b"abcd" * 3, [(4, 0, 4), (8, 4, 4)], 5, 1, [(4, 0, 4), (8, 0, 4)]),
    # the same with blocks of 4 bytes: the roots are followed across blocks
    (b"abcd" * 3, [(4, 0, 4), (8, 4, 4)], 2, 4, [(4, 0, 4), (8, 0, 4)]),
    # a run: the self-overlapping match reads the literal 'a' only and is kept
    (b"a" * 10, [(1, 0, 9)], 5, 1, [(1, 0, 9)]),
    # period 2 over match bytes: [2,4) copies [0,2); [4,10) copies [2,4) with period 2 (roots 0,1,0,1,0,1):
    # a short period restarts from literal bytes -- [4,6) literal, then (6, 4, 4) reading them
    (b"ab" * 5, [(2, 0, 2), (4, 2, 6)], 5, 2, [(2, 0, 2), (6, 4, 4)]),
    # the same repeat too short to restart (3 - 2 < min_match 2): runs of roots 0,1 | 0 -> (4, 0, 2) and
    # one literal byte
    (b"abababa", [(2, 0, 2), (4, 2, 3)], 5, 2, [(2, 0, 2), (4, 0, 2)]),
    # roots 0..5 after "abcdef": [6,9)<-0, [9,12)<-3 (depth 1); [12,16)<-7 reads roots 1,2 | 3,4 of two writers,
    # consecutive -> one match from 1; [16,22)<-6 reads roots 0..5 -> from 0; [22,26)<-10 reads roots 4,5 | 1,2
    # -> two runs of two bytes
    (b"abcdef" b"abc" b"def" b"bcde" b"abcdef" b"efbc",
     [(6, 0, 3), (9, 3, 3), (12, 7, 4), (16, 6, 6), (22, 10, 4)], 5, 2,
     [(6, 0, 3), (9, 3, 3), (12, 1, 4), (16, 0, 6), (22, 4, 2), (24, 1, 2)]),
    # the same with min_match 3: the two-byte runs become literal bytes
    (b"abcdef" b"abc" b"def" b"bcde" b"abcdef" b"efbc",
     [(6, 0, 3), (9, 3, 3), (12, 7, 4), (16, 6, 6), (22, 10, 4)], 5, 3,
     [(6, 0, 3), (9, 3, 3), (12, 1, 4), (16, 0, 6)]),
]


@pytest.mark.parametrize("case", range(len(GOLDEN)))
def test_hand_derived_transcodes(case):
    x, parse, bl, mm, want = GOLDEN[case]
    comp = _stream(x, parse, bl, mm)
    t = oracle.transcode_flat(comp)
    assert _parse_list(t) == want
    assert bytes(oracle.decode(t)) == x
    info = oracle.peek(t)
    assert (info.flatten, info.depth_cap, info.block_log2, info.tile_log2, info.min_match) == (2, 0, bl, 2, mm)
    assert info.max_depth == (1 if want else 0)


def _roots(n, parse):
    """root[y]: y for a literal byte; for byte k of match (d, s, L), the root of s + (k mod (d - s))."""
    root = list(range(n))
    for d, s, L in parse:
        for k in range(L):
            root[d + k] = root[s + k % (d - s)]
    return root


def _check_transcode(x: bytes, parse, block_log2, min_match):
    comp = _stream(x, parse, block_log2, min_match)
    t = oracle.transcode_flat(comp)
    assert bytes(oracle.decode(t)) == x
    assert oracle.check(t) == 0
    new = _parse_list(t)
    assert all(int(v) == 1 for v in oracle.depths(t))
    root = _roots(len(x), parse)
    owner = {}
    for i, (d, s, L) in enumerate(parse):
        for k in range(L):
            owner[d + k] = i
    covered, restarted = set(), set()
    for d, s, L in new:
        assert L >= min_match
        i = owner[d]
        od, os_, oL = parse[i]
        assert d + L <= od + oL, "a rewritten match stays inside one original match"
        if (od, os_, oL) == (d, s, L) and d - s < L:
            # kept self-overlapping match: its effective source is literal
            assert all(root[y] == y for y in range(s, d))
        elif s == od and od - os_ < oL and (d, L) == (2 * od - os_, oL - (od - os_)):
            # a short repeat restarted from literal bytes: the original's first period, then the rest
            assert od - os_ <= 32
            assert not any(y in covered for y in range(od, d))
            restarted.add(i)
        else:
            assert d - s >= L and all(root[d + k] == s + k for k in range(L)), "roots preserved"
            # maximal: the neighbours inside the same original match do not continue the run
            if d > od:
                assert root[d - 1] + 1 != root[d]
            if d + L < od + oL:
                assert root[d + L] != root[d + L - 1] + 1
        covered.update(range(d, d + L))
    # every original match byte left literal lies in a run of consecutive roots shorter than min_match
    for i, (od, os_, oL) in enumerate(parse):
        if i in restarted:
            continue
        k = 0
        while k < oL:
            k1 = k + 1
            while k1 < oL and root[od + k1] == root[od + k1 - 1] + 1:
                k1 += 1
            run = range(od + k, od + k1)
            if not any(y in covered for y in run):
                assert k1 - k < min_match
            k = k1
    return t


@pytest.mark.parametrize("alphabet,max_len", [("ab", 6), ("abc", 5)])
@pytest.mark.parametrize("block_log2", [2, 3])
def test_every_parse_of_tiny_strings(alphabet, max_len, block_log2):
    count = 0
    for n in range(1, max_len + 1):
        for tup in itertools.product(alphabet, repeat=n):
            s = "".join(tup).encode()
            for parse in all_parses(s, 1 << block_log2, limit=400):
                _check_transcode(s, parse, block_log2, 1)
                count += 1
    assert count > 1000


@pytest.mark.parametrize("min_match", [1, 2, 3])
def test_random_parses_of_longer_strings(min_match):
    rng = random.Random(min_match)
    done = 0
    while done < 300:
        n = rng.randint(8, 60)
        s = bytes(rng.choice(b"aab") for _ in range(n))
        parse = [m for m in random_parse(s, 16, rng) if m[2] >= min_match]
        _check_transcode(s, parse, 4, min_match)
        done += 1


GEN = [("text", 300_000, dict()), ("markov", 200_000, dict(block_log2=14, tile_log2=8)),
       ("fastq", 250_000, dict(depth_cap=3)), ("rle7", 150_000, dict()), ("random", 40_000, dict()),
       ("text", 120_000, dict(flatten=1, block_log2=12, tile_log2=6)), ("text", 1, dict()), ("fastq", 0, dict())]


@pytest.mark.parametrize("spec", GEN, ids=[f"{k}-{n}-{i}" for i, (k, n, _) in enumerate(GEN)])
def test_generated_streams(spec):
    kind, n, kw = spec
    x = synth.make(kind, n, 77)
    c = oracle.encode(x, **kw)
    t = oracle.transcode_flat(c)
    assert np.array_equal(oracle.decode(t), x)
    assert oracle.check(t) == 0
    info, ic = oracle.peek(t), oracle.peek(c)
    assert info.max_depth <= 1 and info.flatten == 2
    assert (info.block_log2, info.tile_log2, info.min_match) == (ic.block_log2, ic.tile_log2, ic.min_match)
    assert np.array_equal(oracle.transcode_flat(t), t), "a flattened stream transcodes to itself"


@pytest.mark.parametrize("kind", ["text", "fastq", "rle7", "markov"])
def test_flattened_encoder_output_is_a_fixed_point(kind):
    x = synth.make(kind, 200_000, 5)
    c = oracle.encode(x, flatten=2)
    assert np.array_equal(oracle.transcode_flat(c), c)


def test_malformed_input_is_reported():
    x = synth.make("text", 50_000, 1)
    c = oracle.encode(x)
    bad = c.copy()
    bad[0] ^= 1
    assert oracle.transcode_flat_rc(bad)[0] == oracle.decode_rc(bad)[0] != 0
