"""aceapex_decode_batch_host: n streams in host memory decoded into host buffers, in groups whose copies in,
decodes and copies out overlap.  Outputs are checked byte for byte against the inputs (which the oracle's
decode reproduces), error statuses against the oracle's codes and the library's own argument checks, and the
bytes around every output (host gaps, guard bytes) for writes outside the outputs."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_04268_gb300 as ax
import synth

pytestmark = pytest.mark.gpu

POISON = 0xA5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ax.build()
    oracle.build()
    yield


def _mixed(count, seed, big=1 << 20):
    """(input, stream) pairs: flattened FASTQ / text / RLE / random, deep text (wavefront path), tiny and
    empty streams, sizes from a few bytes to a few MiB."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        kind = ["fastq", "text", "rle7", "random", "deep", "tiny", "empty"][i % 7]
        n = int(rng.integers(big // 2, 3 * big))
        if kind == "empty":
            x = np.zeros(0, np.uint8)
            c = oracle.encode(x)
        elif kind == "tiny":
            x = synth.make("text", int(rng.integers(1, 200)), seed + i)
            c = oracle.encode(x, block_log2=12, tile_log2=6, flatten=2)
        elif kind == "deep":
            x = synth.make("text", n, seed + i)
            c = ax.encode(x)
            assert ax.peek_header(c[:64]).max_depth > 1
        else:
            x = synth.make(kind, n, seed + i)
            c = ax.encode(x, flatten=2, min_emit=6)
        out.append((x, c))
    return out


def _contiguous(pairs, pinned):
    """One host buffer holding every stream back to back (16-byte offsets) and one holding every output back
    to back, with poisoned guard bytes before and after."""
    c_off = np.cumsum([0] + [c.size for _, c in pairs])
    o_off = np.cumsum([0] + [x.size for x, _ in pairs])
    G = 64
    if pinned:
        hc = torch.empty(int(c_off[-1]) + 16, dtype=torch.uint8).pin_memory().numpy()
        ho = torch.empty(int(o_off[-1]) + 2 * G, dtype=torch.uint8).pin_memory().numpy()
    else:
        hc = np.empty(int(c_off[-1]) + 16, np.uint8)
        ho = np.empty(int(o_off[-1]) + 2 * G, np.uint8)
    for i, (_, c) in enumerate(pairs):
        hc[c_off[i]:c_off[i + 1]] = c
    ho.fill(POISON)
    comps = [hc[c_off[i]:c_off[i + 1]] for i in range(len(pairs))]
    outs = [ho[G + o_off[i]:G + o_off[i + 1]] for i in range(len(pairs))]
    return hc, ho, comps, outs, G


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_contiguous_batch_exact_and_guards_untouched(pinned):
    pairs = _mixed(35, 900)  # ~60 MiB: several groups
    hc, ho, comps, outs, G = _contiguous(pairs, pinned)
    for rep in range(2):  # the second call reuses the library's device buffers
        ho.fill(POISON)
        st = ax.decode_batch_host(comps, outs)
        assert (st == 0).all(), st
        for (x, _), o in zip(pairs, outs):
            assert np.array_equal(o, x)
        assert (ho[:G] == POISON).all() and (ho[ho.size - G:] == POISON).all()


def test_scattered_unaligned_buffers_and_gaps_kept():
    """Streams at odd host addresses and with gaps (small and large) between them; outputs with gaps that
    must keep their bytes."""
    pairs = _mixed(21, 901, big=256 << 10)
    rng = np.random.default_rng(7)
    gaps_c = [int(g) for g in rng.choice([0, 3, 16, 100, 70_000, 200_000], size=len(pairs))]
    gaps_o = [int(g) for g in rng.choice([0, 1, 5, 4096], size=len(pairs))]
    hc = np.zeros(sum(c.size for _, c in pairs) + sum(gaps_c) + 64, np.uint8)
    ho = np.full(sum(x.size for x, _ in pairs) + sum(gaps_o) + 64, POISON, np.uint8)
    comps, outs, at_c, at_o = [], [], 5, 7
    for (x, c), gc, go in zip(pairs, gaps_c, gaps_o):
        at_c += gc
        hc[at_c:at_c + c.size] = c
        comps.append(hc[at_c:at_c + c.size])
        at_c += c.size
        at_o += go
        outs.append(ho[at_o:at_o + x.size])
        at_o += x.size
    mask = np.ones(ho.size, bool)
    for o in outs:
        a = o.ctypes.data - ho.ctypes.data
        mask[a:a + o.size] = False
    st = ax.decode_batch_host(comps, outs)
    assert (st == 0).all(), st
    for (x, _), o in zip(pairs, outs):
        assert np.array_equal(o, x)
    assert (ho[mask] == POISON).all()


def test_errors_per_stream_match_the_oracle_and_the_device_batch():
    pairs = _mixed(14, 902, big=128 << 10)
    x = synth.make("text", 300_000, 44)
    good = oracle.encode(x, block_log2=14, tile_log2=8, flatten=2)
    bad = good.copy()
    b1 = int.from_bytes(bytes(bad[72:80]), "little")  # offset of block 1 (block index entry 1)
    bad[b1:b1 + 4] = np.frombuffer((5).to_bytes(4, "little"), np.uint8)  # its n_seq field, changed
    rc_o, _ = oracle.decode_rc(bad, out_len=x.size)
    assert rc_o != 0
    comps = [c for _, c in pairs] + [bad, good, good[:40].copy(), good]
    outs = [np.empty(xx.size, np.uint8) for xx, _ in pairs] + [np.empty(x.size, np.uint8), np.empty(x.size, np.uint8),
                                                               np.empty(x.size, np.uint8), np.empty(x.size + 1, np.uint8)]
    st = ax.decode_batch_host(comps, outs)
    k = len(pairs)
    assert (st[:k] == 0).all(), st
    assert st[k] == rc_o
    assert st[k + 1] == 0 and np.array_equal(outs[k + 1], x)
    assert st[k + 2] == ax.ERR_ARG
    assert st[k + 3] == ax.ERR_SIZE
    for (xx, _), o in zip(pairs, outs[:k]):
        assert np.array_equal(o, xx)
    # the device-pointer batch gives the same statuses (streams long enough to copy to the device)
    dc = [torch.from_numpy(c).cuda() for c in comps[:k + 2]] + [torch.from_numpy(comps[k + 3]).cuda()]
    do = [torch.empty(o.size, dtype=torch.uint8, device="cuda") for o in outs[:k + 2]] + \
         [torch.empty(outs[k + 3].size, dtype=torch.uint8, device="cuda")]
    sd = ax.decode_batch(dc, do)
    assert list(sd) == list(st[:k + 2]) + [st[k + 3]]


def test_first_error_returned_and_prepared_batch_reused():
    pairs = _mixed(9, 903, big=64 << 10)
    _, _, comps, outs, _ = _contiguous(pairs, True)
    b = ax.HostBatch(comps, outs)
    for _ in range(3):
        assert ax.decode_batch_host_status(b) == 0
        assert (b.statuses[:b.n] == 0).all()
    for (x, _), o in zip(pairs, outs):
        assert np.array_equal(o, x)
    short = [comps[0][:10].copy()] + comps[1:]
    bb = ax.HostBatch(short, outs)
    assert ax.decode_batch_host_status(bb) == ax.ERR_ARG
    assert bb.statuses[0] == ax.ERR_ARG and (bb.statuses[1:bb.n] == 0).all()


def test_empty_batch_and_all_empty_streams():
    assert ax.decode_batch_host([], []).size == 0
    e = oracle.encode(np.zeros(0, np.uint8))
    st = ax.decode_batch_host([e, e.copy()], [np.zeros(0, np.uint8), np.zeros(0, np.uint8)])
    assert (st == 0).all()
