"""Brute force: every legal parse of every tiny string must decode to that string.

A parse is any sequence of literals and matches (absolute source s < destination d, length >= 1 with
min_match = 1, never leaving the destination block) whose byte-sequential copy reproduces the string.
All parses are enumerated for strings over {a,b} up to 6 bytes and over {a,b,c} up to 5 bytes, with
blocks of 4 and 8 bytes; longer strings use random legal parses.  Each parse is serialized, decoded by
the oracle and by the textbook relative decoder, and its depths are compared with the longest path of the
explicit dependency graph.
"""
import itertools
import random

import numpy as np
import pytest

import oracle
from test_oracle_pins import _explicit_depths


def all_parses(s: bytes, B: int, limit: int = 10**6):
    n = len(s)
    out = []

    def rec(p, acc):
        if len(out) >= limit:
            return
        if p == n:
            out.append(list(acc))
            return
        rec(p + 1, acc)
        bend = min((p // B + 1) * B, n)
        for src in range(p):
            per = p - src
            for L in range(1, bend - p + 1):
                if s[p + L - 1] != s[src + (L - 1) % per]:
                    break
                acc.append((p, src, L))
                rec(p + L, acc)
                acc.pop()

    rec(0, [])
    return out


def random_parse(s: bytes, B: int, rng: random.Random):
    n, p, acc = len(s), 0, []
    while p < n:
        bend = min((p // B + 1) * B, n)
        opts = []
        for src in range(p):
            per = p - src
            L = 0
            while p + L < bend and s[p + L] == s[src + L % per]:
                L += 1
            if L:
                opts.append((src, L))
        if opts and rng.random() < 0.7:
            src, L = rng.choice(opts)
            L = rng.randint(1, L)
            acc.append((p, src, L))
            p += L
        else:
            p += 1
    return acc


def check_parse(s: bytes, parse, block_log2: int):
    x = np.frombuffer(s, dtype=np.uint8)
    d = [m[0] for m in parse]
    src = [m[1] for m in parse]
    L = [m[2] for m in parse]
    comp = oracle.serialize(x, d, src, L, block_log2=block_log2, tile_log2=2, min_match=1)
    assert bytes(oracle.decode(comp)) == s
    r, Ls, ss, lits = oracle.parse(comp)
    dst = np.cumsum(r + Ls) - Ls
    dist = np.where(Ls > 0, dst - ss, 0)
    assert bytes(oracle.lz77_rel_decode(r, Ls, dist, lits, len(s))) == s
    assert list(oracle.depths(comp)) == _explicit_depths(r, Ls, ss)
    assert oracle.check(comp) == 0


@pytest.mark.parametrize("alphabet,max_len", [("ab", 6), ("abc", 5)])
@pytest.mark.parametrize("block_log2", [2, 3])
def test_every_parse_of_tiny_strings(alphabet, max_len, block_log2):
    count = 0
    for n in range(1, max_len + 1):
        for t in itertools.product(alphabet, repeat=n):
            s = "".join(t).encode()
            for parse in all_parses(s, 1 << block_log2):
                check_parse(s, parse, block_log2)
                count += 1
    assert count > 1000


@pytest.mark.parametrize("block_log2", [2, 3, 4])
def test_random_parses_of_short_strings(block_log2):
    rng = random.Random(block_log2)
    for _ in range(400):
        n = rng.randint(7, 40)
        s = bytes(rng.choice(b"aab") for _ in range(n))
        check_parse(s, random_parse(s, 1 << block_log2, rng), block_log2)
