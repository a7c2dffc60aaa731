"""The oracle against streams assembled by hand in the ACEAPEX stream format, and the worked example of §3.1."""
import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "streams.json")) as f:
    GOLDEN = {k: v for k, v in json.load(f).items() if not k.startswith("_")}


def assemble(fx) -> np.ndarray:
    buf = bytearray(fx["comp_len"])
    for off, width, value in fx["ints"]:
        buf[off:off + width] = int(value).to_bytes(width, "little")
    for off, text in fx["bytes"]:
        buf[off:off + len(text)] = text.encode()
    return np.frombuffer(bytes(buf), dtype=np.uint8)


@pytest.mark.parametrize("name", sorted(GOLDEN))
def test_golden_decode(name):
    fx = GOLDEN[name]
    comp = assemble(fx)
    out = oracle.decode(comp)
    assert bytes(out) == fx["decoded"].encode()
    assert list(oracle.depths(comp)) == fx["depths"]
    assert oracle.check(comp) == 0


@pytest.mark.parametrize("name", sorted(GOLDEN))
def test_golden_serializer_reproduces_layout(name):
    """Re-serializing the hand-written parse gives the hand-assembled bytes (pins the writer's layout)."""
    fx = GOLDEN[name]
    comp = assemble(fx)
    info = oracle.peek(comp)
    r, L, s, _ = oracle.parse(comp)
    pos, d_list, s_list, l_list = 0, [], [], []
    for ri, li, si in zip(r.tolist(), L.tolist(), s.tolist()):
        pos += ri
        if li:
            d_list.append(pos); s_list.append(si); l_list.append(li)
            pos += li
    again = oracle.serialize(fx["decoded"].encode(), d_list, s_list, l_list, block_log2=info.block_log2,
                             tile_log2=info.tile_log2, min_match=info.min_match)
    assert bytes(again) == bytes(comp)


def test_paper_3_1_worked_example():
    """§3.1: bytes at position 5,000 are referenced as offset 5,000 from positions 5,100 and 5,300; in
    relative LZ77 the same references are distances 100 and 300."""
    rng = np.random.default_rng(31)
    data = rng.integers(0, 256, 6000, dtype=np.uint8)
    L = 40
    data[5100:5100 + L] = data[5000:5000 + L]
    data[5300:5300 + L] = data[5000:5000 + L]
    comp = oracle.serialize(data, [5100, 5300], [5000, 5000], [L, L], block_log2=12, tile_log2=8)
    r, Ls, s, lits = oracle.parse(comp)
    assert [int(x) for x in s[Ls > 0]] == [5000, 5000]          # the same absolute offset twice
    d = np.cumsum(r + Ls) - Ls                                  # destination of each match
    dist = np.where(Ls > 0, d - s, 0)
    assert [int(x) for x in dist[Ls > 0]] == [100, 300]         # two different relative distances
    out = oracle.decode(comp)
    assert np.array_equal(out, data)
    assert np.array_equal(oracle.lz77_rel_decode(r, Ls, dist, lits, data.size), data)
    # the match at 5,300 lies in block 1 (B = 4,096) and reads block 1 bytes: no positional context needed
    assert list(oracle.depths(comp)) == [1, 1]
