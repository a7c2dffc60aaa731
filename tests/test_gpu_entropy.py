"""GPU decoder of the entropy container (format §6): the wrapped stream it produces equals the oracle's,
byte for byte, for containers of generated streams, a hand-written one and every malformation the oracle
pins (the same status); the wrapped stream then decodes to the input."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_04268_gb300 as ax
import synth
from gpu_util import to_dev
from test_oracle_entropy import _hand_container, _field

pytestmark = pytest.mark.gpu

GEN = [("text", 3_000_000, dict(flatten=2, min_emit=6)), ("fastq", 2_000_000, dict(flatten=2, min_emit=12, long_bits=20)),
       ("text", 900_000, dict()), ("random", 500_000, dict(flatten=2)), ("rle7", 400_001, dict(flatten=2)),
       ("markov", 777_777, dict(block_log2=12, tile_log2=6, flatten=2)), ("text", 1, dict()), ("fastq", 0, dict())]


def _gpu_raw(e: np.ndarray):
    info = ax.entropy_peek(e[:64])
    d = to_dev(e)
    raw = torch.full((int(info.raw_len) + 64,), 0xA5, dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ax.entropy_decode_async(d, info, raw[:int(info.raw_len)], st)
    torch.cuda.synchronize()
    host = raw.cpu().numpy()
    assert np.all(host[int(info.raw_len):] == 0xA5), "write past the wrapped stream"
    return int(st.item()), host[:int(info.raw_len)]


@pytest.mark.parametrize("spec", GEN, ids=[f"{k}-{n}" for k, n, _ in GEN])
def test_entropy_decode_matches_oracle(spec):
    kind, n, kw = spec
    x = synth.make(kind, n, 31)
    c = oracle.encode(x, **kw)
    e = oracle.entropy_encode(c)
    rc, raw = _gpu_raw(e)
    assert rc == 0 and np.array_equal(raw, oracle.entropy_decode(e)) and np.array_equal(raw, c)
    out = torch.empty(n, dtype=torch.uint8, device="cuda")
    ax.decode(ax.entropy_decode(to_dev(e)), out)
    assert np.array_equal(out.cpu().numpy(), x)


def test_hand_written_container_and_malformations():
    raw, e = _hand_container()
    rc, got = _gpu_raw(np.frombuffer(e, np.uint8))
    assert rc == 0 and bytes(got) == raw
    cases = [(80, "<B", 2), (84, "<I", 1), (80 + 8 + 48, "<B", 13 << 4), (80 + 8 + 50, "<B", 1), (80 + 136, "<H", 15),
             (80 + 136, "<H", 4000), (72, "<Q", 96)]
    for off, fmt, v in cases:
        b = _field(e, off, fmt, v)
        want = oracle.entropy_decode_rc(b, len(raw))[0]
        assert want == ax.ERR_FORMAT
        rc, _ = _gpu_raw(b)
        assert rc == want, (off, fmt, v)
    # header-level errors are found on the host
    for off, fmt, v, code in [(0, "<I", 0x45454342, ax.ERR_FORMAT), (12, "<I", 13, ax.ERR_FORMAT)]:
        with pytest.raises(ax.AceapexError) as ex:
            ax.entropy_peek(_field(e, off, fmt, v)[:64])
        assert ex.value.code == code


def test_entropy_of_many_segments_and_shared_codes():
    """A 24 MiB FASTQ stream: thousands of segments, most of them sharing their section's code."""
    x = synth.make("fastq", 24 << 20, 5)
    c = oracle.encode(x, flatten=2, min_emit=12, long_bits=22, chain_limit=4)
    e = oracle.entropy_encode(c)
    assert int(ax.entropy_peek(e[:64]).n_seg) > 4000
    rc, raw = _gpu_raw(e)
    assert rc == 0 and np.array_equal(raw, c)
