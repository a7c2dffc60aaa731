"""Property test on CPU: for small random inputs and random encoder parameters, the library's C++ encoder
produces the same stream as the oracle's encoder, the oracle decodes it back to the input, and the
stream passes the oracle's invariant check (sources precede destinations, flattened sources are literal,
the depth cap holds, the recorded depths are the recomputed ones)."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
import paper_2606_04268_gb300 as ax  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _libs():
    oracle.build()
    ax.build()
    ax.lib()


def _data(seed: int, n: int, alphabet: int, motif: int) -> np.ndarray:
    """Random bytes over a small alphabet with repeated motifs (so that matches, overlaps and chains occur)."""
    rng = np.random.default_rng(seed)
    base = rng.integers(0, alphabet, max(motif, 1), dtype=np.uint8)
    out = np.empty(n, np.uint8)
    i = 0
    while i < n:
        if rng.random() < 0.5:
            k = int(rng.integers(1, 40))
            out[i:i + k] = np.resize(base, k)[: max(0, min(k, n - i))]
        else:
            k = int(rng.integers(1, 12))
            out[i:i + k] = rng.integers(0, alphabet, k, dtype=np.uint8)[: max(0, min(k, n - i))]
        i += k
    return out


@settings(max_examples=60, deadline=None)
@given(seed=st.integers(0, 2**31 - 1), n=st.integers(0, 6000), alphabet=st.sampled_from([2, 4, 26, 256]),
       motif=st.integers(1, 50), block_log2=st.sampled_from([6, 8, 12]), tile=st.integers(2, 6),
       min_match=st.integers(1, 6), flatten=st.sampled_from([0, 1, 2]), depth_cap=st.sampled_from([0, 1, 2, 5]),
       chain_limit=st.sampled_from([1, 4, 16]), use_first=st.sampled_from([0, 1]), min_emit=st.sampled_from([0, 6]),
       long_bits=st.sampled_from([0, 8, 12]), long_chain=st.sampled_from([1, 4, 16]))
def test_encoders_agree_and_round_trip(seed, n, alphabet, motif, block_log2, tile, min_match, flatten, depth_cap,
                                       chain_limit, use_first, min_emit, long_bits, long_chain):
    x = _data(seed, n, alphabet, motif)
    kw = dict(block_log2=block_log2, tile_log2=min(tile, block_log2), min_match=min_match, flatten=flatten,
              depth_cap=depth_cap, chain_limit=chain_limit, use_first=use_first, min_emit=min_emit,
              long_bits=long_bits, long_chain=long_chain)
    a = oracle.encode(x, **kw)
    b = ax.encode(x, **kw)
    assert np.array_equal(a, b)
    assert np.array_equal(oracle.decode(a), x)
    assert oracle.check(a) == 0
