"""Seeded synthetic inputs shaped like the paper's workloads (§4.2 datasets: text corpus, FASTQ reads).

This module holds no codec arithmetic: it only produces raw bytes (and, for the batched and served
workloads, seeded size and content mixes).  Both the CPU oracle's tests and the GPU decoder's tests and
benchmark take their inputs from here, so neither side depends on the other.

Recipes (seeds are fixed per workload):

* ``markov_text``  -- order-2 Markov bytes over 96 printable symbols (0x20-0x7E and newline), seeded
  skewed transition tables, interleaved with reuse of earlier words drawn Zipf(s=1.1).
* ``zipf_text``    -- English-like text: 200k generated words (length uniform 2-12, letters from a
  seeded unigram profile) drawn Zipf(s=1.0), 35 % bigram successors, sentences of 5-30 words,
  ~5 % invented markup tokens, paragraph breaks.
* ``fastq``        -- 150-base reads sampled from 64 seeded 1 Mb ACGT segments with 1 % substitutions,
  ``@SYNTH.<segment>.<id>`` headers with incrementing ids, ``+`` lines, Phred+33 qualities from a
  per-position Gaussian (mean 31 falling to 28, sd 3, clipped to [2, 41]).
* ``random_bytes`` -- uniform bytes (incompressible).
* ``rle7``         -- a seeded 7-byte motif repeated, 0.1 % of bytes mutated (self-overlapping matches).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile gen.c into libsynth.so next to it (plain gcc, host architecture)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, p, sz = ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t
            lib.synth_random.argtypes = [u64, p, sz]
            lib.synth_rle7.argtypes = [u64, p, sz]
            lib.synth_markov_text.argtypes = [u64, p, sz]
            lib.synth_zipf_text.argtypes = [u64, u64, p, sz]
            lib.synth_fastq.argtypes = [u64, u64, p, sz]
            for f in (lib.synth_random, lib.synth_rle7, lib.synth_markov_text, lib.synth_zipf_text, lib.synth_fastq):
                f.restype = None
            _lib = lib
    return _lib


def _buf(n: int) -> np.ndarray:
    return np.empty(int(n), dtype=np.uint8)


def random_bytes(n: int, seed: int) -> np.ndarray:
    a = _buf(n)
    _load().synth_random(seed, a.ctypes.data, a.size)
    return a


def rle7(n: int, seed: int) -> np.ndarray:
    a = _buf(n)
    _load().synth_rle7(seed, a.ctypes.data, a.size)
    return a


def markov_text(n: int, seed: int) -> np.ndarray:
    a = _buf(n)
    _load().synth_markov_text(seed, a.ctypes.data, a.size)
    return a


def zipf_text(n: int, seed: int, vocab_seed: int = 2000) -> np.ndarray:
    a = _buf(n)
    _load().synth_zipf_text(vocab_seed, seed, a.ctypes.data, a.size)
    return a


def fastq(n: int, seed: int, ref_seed: int = 3000) -> np.ndarray:
    a = _buf(n)
    _load().synth_fastq(ref_seed, seed, a.ctypes.data, a.size)
    return a


def make(kind: str, n: int, seed: int) -> np.ndarray:
    """Bytes of one content kind: 'text', 'markov', 'fastq', 'random', 'rle7'."""
    if kind == "text":
        return zipf_text(n, seed)
    if kind == "markov":
        return markov_text(n, seed)
    if kind == "fastq":
        return fastq(n, seed)
    if kind == "random":
        return random_bytes(n, seed)
    if kind == "rle7":
        return rle7(n, seed)
    raise ValueError(kind)


# ---------------------------------------------------------------------------------------------- workloads
MiB = 1 << 20
GiB = 1 << 30

# the small single-stream workload (4 MiB Markov text, 4 blocks) and the 1 GiB ones
SMALL_TEXT = dict(kind="markov", n=4 * MiB, seed=1000)
BIG_TEXT = dict(kind="text", n=1 * GiB, seed=2000)
BIG_FASTQ = dict(kind="fastq", n=1 * GiB, seed=3000)


def batch_mix(n_streams: int = 4096, seed: int = 4000, total_scale: float = 1.0):
    """Stream sizes and kinds of the batched workload.

    Sizes: lognormal with median 1 MiB and sigma 1.18 (mean ~2 MiB), clipped to [4 KiB, 64 MiB], then
    multiplied by ``total_scale`` (1.0 gives ~8 GiB over 4096 streams).  Kinds: 46 % text, 46 % FASTQ,
    8 % uniform random bytes.  Returns a list of (kind, size, seed).
    """
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.normal(np.log(MiB), 1.18, n_streams))
    sizes = np.clip(sizes, 4096, 64 * MiB) * total_scale
    sizes = np.maximum(sizes.astype(np.int64), 1)
    u = rng.random(n_streams)
    kinds = np.where(u < 0.46, "text", np.where(u < 0.92, "fastq", "random"))
    return [(str(k), int(s), seed * 100000 + i) for i, (k, s) in enumerate(zip(kinds, sizes))]


def serve_mix(n_requests: int, seed: int = 5000, lo: int = 64 * 1024, hi: int = 256 * MiB):
    """Request sizes (log-uniform in [lo, hi]) and kinds (text / FASTQ / period-7 RLE, equal shares)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), n_requests)).astype(np.int64)
    kinds = rng.choice(np.array(["text", "fastq", "rle7"]), n_requests)
    return [(str(k), int(s), seed * 100000 + i) for i, (k, s) in enumerate(zip(kinds, sizes))]
