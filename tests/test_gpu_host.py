"""aceapex_decode_host: host buffers in, host buffer out, copies overlapped with the decode in slices of
whole blocks.  Checked byte for byte against the input (the oracle's own decode reproduces it) and, for a
malformed stream, against the oracle's error code."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_04268_gb300 as ax
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ax.build()
    oracle.build()
    yield


def _pinned(a: np.ndarray) -> torch.Tensor:
    t = torch.empty(a.size, dtype=torch.uint8).pin_memory()
    t.copy_(torch.from_numpy(a))
    return t


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_flattened_multi_slice(pinned):
    x = synth.make("fastq", 70 << 20, 41)  # 70 one-MiB blocks: 3 slices
    comp = ax.encode(x, flatten=2, min_emit=6)
    assert ax.peek_header(comp[:64]).max_depth <= 1
    if pinned:
        hc, ho = _pinned(comp), torch.empty(x.size, dtype=torch.uint8).pin_memory()
    else:
        hc, ho = comp.copy(), np.empty(x.size, np.uint8)
    for _ in range(2):  # the device buffers are reused by the second call
        if pinned:
            ho.fill_(0x5A)
        else:
            ho.fill(0x5A)
        assert ax.decode_host_status(hc, ho) == 0
        got = ho.numpy() if pinned else ho
        assert np.array_equal(got, x)


@pytest.mark.parametrize("kind,kw", [("text", dict()), ("rle7", dict(flatten=2)), ("random", dict(flatten=2)),
                                     ("markov", dict(block_log2=16, tile_log2=10, flatten=2))])
def test_kinds_and_paths(kind, kw):
    x = synth.make(kind, 5_000_001, 43)
    comp = oracle.encode(x, **kw)
    out = np.empty(x.size, np.uint8)
    assert ax.decode_host_status(comp, out) == 0
    assert np.array_equal(out, x)


def test_errors_match_the_oracle_and_sizes_are_checked():
    x = synth.make("text", 300_000, 44)
    comp = oracle.encode(x, block_log2=14, tile_log2=8, flatten=2)
    bad = comp.copy()
    b1 = int.from_bytes(bytes(bad[72:80]), "little")       # offset of block 1 (block index entry 1)
    bad[b1:b1 + 4] = np.frombuffer((5).to_bytes(4, "little"), np.uint8)  # its n_seq field, changed
    rc_o, _ = oracle.decode_rc(bad, out_len=x.size)
    assert rc_o != 0
    out = np.empty(x.size, np.uint8)
    assert ax.decode_host_status(bad, out) == rc_o
    assert ax.decode_host_status(comp, np.empty(x.size + 1, np.uint8)) == ax.ERR_SIZE
    assert ax.decode_host_status(comp, out) == 0 and np.array_equal(out, x)


def test_empty_stream():
    comp = oracle.encode(np.zeros(0, np.uint8))
    assert ax.decode_host_status(comp, np.zeros(0, np.uint8)) == 0
