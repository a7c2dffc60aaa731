"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every symbol include/aceapex.h
declares, and its host-side pieces (header parse, CPU encoder) agree with the oracle.  No GPU call."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2606_04268_gb300 as ax
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    ax.build()
    return ax.lib()


def declared_functions():
    with open(os.path.join(ROOT, "include", "aceapex.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(aceapex_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(ax.SYMBOLS) == names


def test_strerror_names(lib):
    for code in range(0, -9, -1):
        assert ax.strerror(code)


@pytest.mark.parametrize("kw", [dict(), dict(flatten=2, min_emit=6), dict(block_log2=12, tile_log2=6, depth_cap=4)])
def test_peek_header_matches_oracle(lib, kw):
    x = synth.make("text", 200_000, 4)
    comp = oracle.encode(x, **kw)
    a, b = ax.peek_header(comp[:64]), oracle.peek(comp)
    for f in ("n_blocks", "comp_len", "n_match", "n_seq", "block_log2", "tile_log2", "min_match", "flatten",
              "depth_cap", "max_depth"):
        assert getattr(a, f) == getattr(b, f), f
    assert a.decoded_len == b.N
    with pytest.raises(ax.AceapexError) as e:
        bad = comp[:64].copy(); bad[0] ^= 1
        ax.peek_header(bad)
    assert e.value.code == ax.ERR_FORMAT


@pytest.mark.parametrize("kind", ["markov", "text", "fastq", "random", "rle7"])
@pytest.mark.parametrize("kw", [dict(), dict(flatten=1), dict(flatten=2, min_emit=6), dict(depth_cap=4, min_emit=6),
                                dict(block_log2=10, tile_log2=4, flatten=2), dict(depth_cap=1, chain_limit=4),
                                dict(flatten=2, min_emit=10, long_bits=16), dict(depth_cap=4, min_emit=10, long_bits=16),
                                dict(flatten=1, long_bits=12, long_chain=2), dict(long_bits=20, long_chain=16)])
def test_encoder_equals_oracle_encoder(lib, kind, kw):
    """The library's C++ encoder follows the same parse rules as the oracle's: identical streams."""
    x = synth.make(kind, 400_000, 8)
    a = oracle.encode(x, **kw)
    b = ax.encode(x, **kw)
    assert a.size == b.size and np.array_equal(a, b)
    assert np.array_equal(oracle.decode(b), x)
    assert oracle.check(b) == 0


def test_encoder_rejects_bad_params(lib):
    with pytest.raises(ax.AceapexError):
        ax.encode(b"abc", block_log2=30)
    with pytest.raises(ax.AceapexError):
        ax.encode(b"abc", chain_limit=64)
    with pytest.raises(ax.AceapexError):
        ax.encode(b"abc", long_bits=30)
    with pytest.raises(ax.AceapexError):
        ax.encode(b"abc", long_bits=16, long_chain=17)
    with pytest.raises(oracle.OracleError):
        oracle.encode(b"abc", long_bits=16, long_chain=0)


def test_batch_host_argument_and_header_errors_without_a_gpu(lib):
    """aceapex_decode_batch_host settles argument, size and header errors from host memory, before any device
    work: a batch with no stream left to decode returns without touching the GPU."""
    assert lib.aceapex_decode_batch_host(-1, None, None, None, None, None, None) == ax.ERR_ARG
    assert lib.aceapex_decode_batch_host(1, None, None, None, None, None, None) == ax.ERR_ARG
    assert lib.aceapex_decode_batch_host(0, None, None, None, None, None, None) == 0
    x = synth.make("text", 5000, 3)
    good = oracle.encode(x, block_log2=12, tile_log2=8, flatten=2)
    bad_magic = good.copy()
    bad_magic[0] ^= 0xFF
    rc_o, _ = oracle.decode_rc(bad_magic, out_len=x.size)
    empty = oracle.encode(np.zeros(0, np.uint8))
    comps = [good[:40].copy(), good, bad_magic, empty]
    outs = [np.empty(x.size, np.uint8), np.empty(x.size + 3, np.uint8), np.empty(x.size, np.uint8),
            np.zeros(0, np.uint8)]
    st = ax.decode_batch_host(comps, outs, stream=0)  # stream 0: no torch CUDA call
    assert list(st) == [ax.ERR_ARG, ax.ERR_SIZE, rc_o, 0]
    b = ax.HostBatch(comps, outs)
    assert ax.decode_batch_host_status(b, 0) == ax.ERR_ARG  # the first failing status in stream order
    assert ax.decode_batch_host([empty], [np.zeros(0, np.uint8)], stream=0).tolist() == [0]
