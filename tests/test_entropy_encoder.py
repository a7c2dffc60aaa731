"""The library's CPU encoder of the entropy container follows the same rules as the oracle's (format §6 and
the encoder choices there): its containers are byte-identical to the oracle's, and the oracle decodes them
back to the wrapped stream."""
import numpy as np
import pytest

import oracle
import paper_2606_04268_gb300 as ax
import synth

CASES = [("text", 2_000_000, dict(flatten=2, min_emit=6)), ("fastq", 1_000_000, dict(flatten=2, min_emit=12, long_bits=20)),
         ("text", 500_000, dict()), ("random", 200_000, dict(flatten=2)), ("rle7", 300_001, dict(flatten=2)),
         ("markov", 400_000, dict(block_log2=12, tile_log2=6)), ("text", 1, dict()), ("fastq", 0, dict())]


@pytest.mark.parametrize("spec", CASES, ids=[f"{k}-{n}" for k, n, _ in CASES])
def test_library_encoder_matches_oracle(spec):
    kind, n, kw = spec
    c = oracle.encode(synth.make(kind, n, 41), **kw)
    got = ax.entropy_encode(c)
    assert np.array_equal(got, oracle.entropy_encode(c))
    assert np.array_equal(oracle.entropy_decode(got), c)


def test_arbitrary_bytes_and_skewed_codes():
    rng = np.random.default_rng(3)
    for n in (1, 17, 4095, 4096, 4097, 70_000):
        # a steep distribution: Huffman depths beyond 12 bits, cut back to 12
        raw = np.minimum(rng.geometric(0.45, n) - 1, 255).astype(np.uint8)
        got = ax.entropy_encode(raw)
        assert np.array_equal(got, oracle.entropy_encode(raw))
        assert np.array_equal(oracle.entropy_decode(got), raw)
