"""The allocation-free entry point (aceapex_decode_noalloc) against the regular one.

Callers that cannot allocate device memory while decoding use aceapex_decode_noalloc, whose scratch is
a fixed array in the library's static device memory.  Its output must equal aceapex_decode's, byte for
byte (the decode is exact integer work), on two calls in a row (the array keeps the previous call's
contents), and it must refuse streams that do not fit its fixed scratch.  This file is collected last, so
that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2606_04268_gb300 as ax
import synth

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_regular_decode_twice():
    ax.build()
    for kind, n, seed in (("fastq", 3_000_000, 41), ("text", 2_000_001, 42)):
        x = synth.make(kind, n, seed)
        comp = oracle.encode(x, flatten=2, min_emit=6)
        info = ax.peek_header(comp[:64])
        d_comp = _dev(comp)
        ref = torch.zeros(x.size, dtype=torch.uint8, device="cuda")
        assert ax.decode_status(d_comp, ref) == 0
        ref_h = ref.cpu().numpy()
        assert np.array_equal(ref_h, x)
        for _ in range(2):
            out = torch.full((x.size,), 0x5A, dtype=torch.uint8, device="cuda")
            st = torch.full((1,), 77, dtype=torch.int32, device="cuda")
            ax.decode_noalloc(d_comp, out, info, st)
            torch.cuda.synchronize()
            assert int(st.item()) == 0
            assert np.array_equal(out.cpu().numpy(), ref_h)


def test_noalloc_rejects_what_does_not_fit():
    ax.build()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    # a stream whose matches are deeper than 1 needs the wavefront path's per-match records
    x = synth.make("text", 300_000, 5)
    deep = oracle.encode(x)
    info = ax.peek_header(deep[:64])
    assert info.max_depth > 1
    with pytest.raises(ax.AceapexError) as e:
        ax.decode_noalloc(_dev(deep), torch.empty(x.size, dtype=torch.uint8, device="cuda"), info, st)
    assert e.value.code == ax.ERR_NOMEM
    # more tile flags and literal bits than the fixed 16 MiB array holds (16 MiB of output in 4-byte tiles)
    y = synth.make("rle7", 16 << 20, 6)
    many = oracle.encode(y, flatten=2, block_log2=12, tile_log2=2)
    info2 = ax.peek_header(many[:64])
    assert 4 * info2.n_tiles + info2.decoded_len // 8 > 16 << 20
    with pytest.raises(ax.AceapexError) as e:
        ax.decode_noalloc(_dev(many), torch.empty(y.size, dtype=torch.uint8, device="cuda"), info2, st)
    assert e.value.code == ax.ERR_NOMEM


def test_noalloc_reports_depth_lie_like_regular_decode():
    """A stream whose depth fields understate its matches' depths ends in ERR_DEPTH on both entry points."""
    from stream_edit import lower_depths
    ax.build()
    x = synth.make("text", 400_000, 43)
    lie = lower_depths(oracle.encode(x, block_log2=16, tile_log2=12, depth_cap=2), 1)
    info = ax.peek_header(lie[:64])
    assert info.max_depth == 1
    d_comp = _dev(lie)
    out = torch.empty(x.size, dtype=torch.uint8, device="cuda")
    rc = ax.decode_status(d_comp, out)
    assert rc == ax.ERR_DEPTH
    for _ in range(2):
        st = torch.full((1,), 77, dtype=torch.int32, device="cuda")
        ax.decode_noalloc(d_comp, out, info, st)
        torch.cuda.synchronize()
        assert int(st.item()) == rc
