"""Pins of the oracle's entropy container (format §6; the paper's entropy stage, §6 of the paper).

Pinned by: Huffman optimality against brute force over every length assignment of small alphabets,
closed-form lengths of dyadic distributions, completeness of unlimited codes (Kraft sum exactly 1) and the
12-bit limit, the entropy bound, a container written out by hand from the format (bit order, lanes,
nibbles, alignment), every malformation the format names, and round trips of generated streams."""
import itertools
import math
import struct

import numpy as np
import pytest

import oracle
import synth


def _lengths(counts_by_symbol: dict) -> dict:
    c = np.zeros(256, dtype=np.uint64)
    for s, v in counts_by_symbol.items():
        c[s] = v
    L = oracle.huff_lengths(c)
    return {s: int(L[s]) for s in range(256) if L[s]}


def test_dyadic_distributions_get_exact_lengths():
    assert _lengths({0: 8, 1: 4, 2: 2, 3: 1, 4: 1}) == {0: 1, 1: 2, 2: 3, 3: 4, 4: 4}
    assert _lengths({s: 5 for s in range(16)}) == {s: 4 for s in range(16)}
    assert _lengths({7: 100}) == {7: 1}
    assert _lengths({}) == {}


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_huffman_is_optimal_against_brute_force(k):
    rng = np.random.default_rng(k)
    for _ in range(40):
        counts = [int(v) for v in rng.integers(1, 50, k)]
        got = _lengths(dict(enumerate(counts)))
        cost = sum(counts[s] * got[s] for s in range(k))
        best = min(sum(c * l for c, l in zip(counts, ls))
                   for ls in itertools.product(range(1, k + 1), repeat=k) if sum(2.0 ** -l for l in ls) <= 1)
        assert cost == best
        assert sum(2.0 ** -got[s] for s in range(k)) == 1.0  # Huffman codes are complete


def test_limit_and_entropy_bound():
    # Fibonacci weights make an unlimited Huffman tree 30 levels deep
    fib = [1, 1]
    while len(fib) < 30:
        fib.append(fib[-1] + fib[-2])
    L = _lengths(dict(enumerate(fib)))
    assert max(L.values()) == 12 and sum(2 ** (12 - v) for v in L.values()) <= 4096
    rng = np.random.default_rng(1)
    for _ in range(20):
        counts = rng.integers(0, 1000, 256) * (rng.random(256) < 0.5)
        n = int(counts.sum())
        L = _lengths({s: int(v) for s, v in enumerate(counts) if v})
        bits = sum(int(counts[s]) * L[s] for s in L)
        H = -sum(v * math.log2(v / n) for v in counts if v)
        assert H <= bits + 1e-6 and bits <= H + n  # Huffman: at most one bit per symbol above the entropy


def _hand_container():
    """4000 bytes, 3000 'a' then 1000 'b' (not a stream: one coded segment).  Code: 'a' (97) and 'b' (98)
    both of length 1, canonical 'a' = 0, 'b' = 1.  Lane l codes bytes l, l+32, ...: 125 codes, 125 bits,
    16 bytes; its codes are 1 from byte 3000 on, i.e. from its code i0 = ceil((3000 - l) / 32)."""
    raw = b"a" * 3000 + b"b" * 1000
    nib = bytearray(128)
    nib[48] = 1 << 4  # symbol 97 = 2*48 + 1: high nibble of byte 48
    nib[49] = 1       # symbol 98 = 2*49: low nibble of byte 49
    lanes = b""
    for l in range(32):
        bits = [0 if l + 32 * i < 3000 else 1 for i in range(125)] + [0] * 3
        lanes += bytes(int("".join(map(str, bits[8 * j:8 * j + 8])), 2) for j in range(16))
    payload = bytes([1, 0, 0, 0]) + struct.pack("<I", 0) + bytes(nib) + struct.pack("<32H", *([16] * 32)) + lanes
    payload += bytes(-len(payload) % 16)
    e_off = 64 + 16 * 1 + 0  # align16(80) = 80
    e_len = e_off + len(payload)
    hdr = struct.pack("<IHHIIQQQ", 0x45454341, 1, 0, 0, 12, len(raw), 1, e_len) + bytes(24)
    return raw, hdr + struct.pack("<QQ", 0, e_off) + payload


def test_hand_written_container():
    raw, e = _hand_container()
    assert bytes(oracle.entropy_encode(np.frombuffer(raw, np.uint8))) == e
    assert bytes(oracle.entropy_decode(np.frombuffer(e, np.uint8))) == raw


def _field(e, off, fmt, value):
    b = bytearray(e)
    struct.pack_into(fmt, b, off, value)
    return np.frombuffer(bytes(b), np.uint8)


def test_every_malformation_is_rejected():
    raw, e = _hand_container()
    E = np.frombuffer(e, np.uint8)
    bad = {
        "magic": (_field(e, 0, "<I", 0x45454342), -2),
        "version": (_field(e, 4, "<H", 2), -2),
        "max_len": (_field(e, 12, "<I", 13), -2),
        "e_len field": (_field(e, 32, "<Q", len(e) + 16), -3),
        "n_seg zero with data": (_field(e, 24, "<Q", 0), -2),
        "first payload offset": (_field(e, 72, "<Q", 96), -2),
        "mode": (_field(e, 80, "<B", 2), -2),
        "table ahead": (_field(e, 84, "<I", 1), -2),
        "code length 13": (_field(e, 80 + 8 + 48, "<B", 13 << 4), -2),
        "kraft": (_field(e, 80 + 8 + 50, "<B", 1), -2),          # a third code of length 1
        "lane too short": (_field(e, 80 + 136, "<H", 15), -2),    # lane 0 ends before its 125th code
        "lanes beyond payload": (_field(e, 80 + 136, "<H", 4000), -2),
    }
    for name, (b, code) in bad.items():
        assert oracle.entropy_decode_rc(b, len(raw))[0] == code, name
    assert oracle.entropy_decode_rc(E[:-16], len(raw))[0] == -3  # truncated: e_len differs
    assert oracle.entropy_decode_rc(E, len(raw) + 1)[0] == -3


GEN = [("text", 2_000_000, dict(flatten=2, min_emit=6)), ("fastq", 1_500_000, dict(flatten=2, min_emit=12, long_bits=20)),
       ("text", 700_000, dict()), ("random", 300_000, dict(flatten=2)), ("rle7", 400_001, dict(flatten=2)),
       ("markov", 333_333, dict(block_log2=14, tile_log2=8)), ("text", 1, dict()), ("fastq", 0, dict())]


@pytest.mark.parametrize("spec", GEN, ids=[f"{k}-{n}" for k, n, _ in GEN])
def test_round_trip_of_generated_streams(spec):
    kind, n, kw = spec
    x = synth.make(kind, n, 21)
    c = oracle.encode(x, **kw)
    e = oracle.entropy_encode(c)
    assert np.array_equal(oracle.entropy_decode(e), c)
    assert np.array_equal(oracle.decode(oracle.entropy_decode(e)), x)
    assert e.size % 16 == 0
    if n >= 1_000_000 and kind != "random":
        assert e.size < 0.8 * c.size  # the sections of text and FASTQ compress
