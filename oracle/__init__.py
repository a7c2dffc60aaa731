"""CPU oracle for the ACEAPEX decoder -- TEST INFRASTRUCTURE ONLY.

Plain sequential C (``oracle.c``) restating the paper's method: the encoder (§3.1 absolute offsets,
§3.3 chain flattening, §7.4 depth cap), the decoder that defines the decoded bytes (§3.2), a textbook
relative-distance LZ77 decoder (§2), per-match depth (§7.1) and the stream invariants.  Beside it,
``cpupar.c``: the paper's block-parallel multi-threaded CPU decoder (§3.1), a CPU baseline, not the
oracle.  Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg use them; the
product package never imports them and shares no code with them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

FLAT_NONE, FLAT_BLOCK, FLAT_GLOBAL = 0, 1, 2
ERR = {0: "OK", -1: "ERR_ARG", -2: "ERR_FORMAT", -3: "ERR_SIZE", -4: "ERR_OFFSET", -7: "ERR_NOMEM", -8: "ERR_DEPTH"}


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {ERR.get(code, code)}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("block_log2", "tile_log2", "min_match", "hash_bits", "chain_limit", "flatten", "depth_cap", "use_first", "min_emit",
                 "long_bits", "long_chain")]


class Info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("N", "n_blocks", "comp_len", "n_match", "n_seq")] + \
               [(n, ctypes.c_uint32) for n in ("block_log2", "tile_log2", "min_match", "flatten", "depth_cap", "max_depth")]


_ENT_SRC = os.path.join(_HERE, "entropy.c")


def build(force: bool = False) -> str:
    """Compile oracle.c and entropy.c into liboracle.so next to them (plain gcc -O2), and the block-parallel
    CPU decoder."""
    srcs = [_SRC, _ENT_SRC]
    if force or not os.path.exists(_LIB_PATH) or any(os.path.getmtime(_LIB_PATH) < os.path.getmtime(p) for p in srcs):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp] + srcs)
        os.replace(tmp, _LIB_PATH)
    build_cpupar(force)
    return _LIB_PATH


_PAR_SRC = os.path.join(_HERE, "cpupar.c")
_PAR_PATH = os.path.join(_HERE, "libcpupar.so")
_par = None


def build_cpupar(force: bool = False) -> str:
    """Compile the block-parallel CPU decoder (cpupar.c, a CPU baseline, not the oracle) next to it."""
    if force or not os.path.exists(_PAR_PATH) or os.path.getmtime(_PAR_PATH) < os.path.getmtime(_PAR_SRC):
        tmp = _PAR_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp, _PAR_SRC])
        os.replace(tmp, _PAR_PATH)
    return _PAR_PATH


def _par_lib():
    global _par
    with _lock:
        if _par is None:
            lib = ctypes.CDLL(build_cpupar())
            lib.cpupar_decode.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int]
            lib.cpupar_decode.restype = ctypes.c_int
            lib.cpupar_decode_batch.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            lib.cpupar_decode_batch.restype = ctypes.c_int
            _par = lib
    return _par


def cpupar_decode_rc(comp, out_len: int | None = None, threads: int | None = None):
    """Block-parallel CPU decode (§3.1: threads over blocks in order): (status, bytes or None)."""
    c = _u8(comp)
    if out_len is None:
        out_len = int.from_bytes(bytes(c[16:24]), "little")
    out = np.zeros(max(out_len, 1), dtype=np.uint8)
    rc = _par_lib().cpupar_decode(c.ctypes.data, c.size, out.ctypes.data, out_len, int(threads or os.cpu_count() or 1))
    return rc, (out[:out_len] if rc == 0 else None)


def cpupar_decode_batch_rc(comps, out_lens=None, threads: int | None = None, outs=None):
    """Block-parallel CPU decode of n independent streams from one queue of (stream, block) units (§3.1
    per stream, §7.5 across streams): (first failing status or 0, per-stream statuses, outputs).  `outs`:
    optional preallocated uint8 arrays (one per stream) to decode into."""
    cs = [_u8(c) for c in comps]
    n = len(cs)
    if out_lens is None:
        out_lens = [int.from_bytes(bytes(c[16:24]), "little") if c.size >= 24 else 0 for c in cs]
    if outs is None:
        outs = [np.zeros(max(int(m), 1), dtype=np.uint8) for m in out_lens]
    cp = (ctypes.c_void_p * max(n, 1))(*[c.ctypes.data for c in cs])
    cl = (ctypes.c_uint64 * max(n, 1))(*[c.size for c in cs])
    op = (ctypes.c_void_p * max(n, 1))(*[o.ctypes.data for o in outs])
    ol = (ctypes.c_uint64 * max(n, 1))(*[int(m) for m in out_lens])
    st = np.zeros(max(n, 1), np.int32)
    rc = _par_lib().cpupar_decode_batch(n, cp, cl, op, ol, st.ctypes.data, int(threads or os.cpu_count() or 1))
    return rc, st[:n], [o[:int(m)] for o, m in zip(outs, out_lens)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p, u64, i64 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64
            pp = ctypes.POINTER(ctypes.c_void_p)
            lib.oracle_encode.argtypes = [p, u64, ctypes.POINTER(Params), pp]
            lib.oracle_encode.restype = i64
            lib.oracle_serialize.argtypes = [p, u64, p, p, p, u64, ctypes.POINTER(Params), pp]
            lib.oracle_serialize.restype = i64
            lib.oracle_free.argtypes = [p]
            lib.oracle_free.restype = None
            lib.oracle_decode.argtypes = [p, u64, p, u64]
            lib.oracle_decode.restype = ctypes.c_int
            lib.oracle_peek.argtypes = [p, u64, ctypes.POINTER(Info)]
            lib.oracle_peek.restype = ctypes.c_int
            lib.oracle_parse.argtypes = [p, u64, p, p, p, p, u64]
            lib.oracle_parse.restype = i64
            lib.oracle_lz77_rel_decode.argtypes = [u64, p, p, p, p, p, u64]
            lib.oracle_lz77_rel_decode.restype = ctypes.c_int
            lib.oracle_depths.argtypes = [p, u64, p, u64]
            lib.oracle_depths.restype = i64
            lib.oracle_check.argtypes = [p, u64]
            lib.oracle_huff_lengths.argtypes = [p, p]
            lib.oracle_huff_lengths.restype = ctypes.c_int
            lib.oracle_entropy_encode.argtypes = [p, u64, pp]
            lib.oracle_entropy_encode.restype = i64
            lib.oracle_entropy_peek.argtypes = [p, u64, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
            lib.oracle_entropy_peek.restype = ctypes.c_int
            lib.oracle_entropy_decode.argtypes = [p, u64, p, u64]
            lib.oracle_entropy_decode.restype = ctypes.c_int
            lib.oracle_transcode_flat.restype = ctypes.c_int64
            lib.oracle_transcode_flat.argtypes = [p, u64, pp]
            lib.oracle_check.restype = ctypes.c_int
            _lib = lib
    return _lib


def params(block_log2=20, tile_log2=12, min_match=4, hash_bits=20, chain_limit=16, flatten=FLAT_NONE,
           depth_cap=0, use_first=1, min_emit=0, long_bits=0, long_chain=4) -> Params:
    return Params(block_log2, tile_log2, min_match, hash_bits, chain_limit, flatten, depth_cap, use_first, min_emit,
                  long_bits, long_chain)


def _u8(a) -> np.ndarray:
    a = np.ascontiguousarray(np.frombuffer(a, dtype=np.uint8) if isinstance(a, (bytes, bytearray)) else a)
    assert a.dtype == np.uint8
    return a


def _take(ptr: ctypes.c_void_p, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint8)
    ctypes.memmove(out.ctypes.data, ptr, n)
    _load().oracle_free(ptr)
    return out


def encode(data, **kw) -> np.ndarray:
    """Encode bytes into an ACEAPEX stream (uint8 array)."""
    a = _u8(data)
    prm = params(**kw)
    ptr = ctypes.c_void_p()
    n = _load().oracle_encode(a.ctypes.data, a.size, ctypes.byref(prm), ctypes.byref(ptr))
    if n < 0:
        raise OracleError(n, "oracle_encode")
    return _take(ptr, n)


def serialize(data, d, s, L, **kw) -> np.ndarray:
    """Serialize a given parse: matches (d, s, L) sorted by d; every other byte of ``data`` is literal."""
    a = _u8(data)
    d = np.ascontiguousarray(d, dtype=np.uint64)
    s = np.ascontiguousarray(s, dtype=np.uint64)
    L = np.ascontiguousarray(L, dtype=np.uint32)
    prm = params(**kw)
    ptr = ctypes.c_void_p()
    n = _load().oracle_serialize(a.ctypes.data, a.size, d.ctypes.data, s.ctypes.data, L.ctypes.data, d.size,
                                 ctypes.byref(prm), ctypes.byref(ptr))
    if n < 0:
        raise OracleError(n, "oracle_serialize")
    return _take(ptr, n)


def peek(comp) -> Info:
    c = _u8(comp)
    info = Info()
    rc = _load().oracle_peek(c.ctypes.data, c.size, ctypes.byref(info))
    if rc:
        raise OracleError(rc, "oracle_peek")
    return info


def decode_rc(comp, out_len: int | None = None):
    """Returns (status, decoded bytes or None)."""
    c = _u8(comp)
    if out_len is None:
        try:
            out_len = peek(c).N
        except OracleError as e:
            return e.code, None
    out = np.zeros(max(out_len, 1), dtype=np.uint8)
    rc = _load().oracle_decode(c.ctypes.data, c.size, out.ctypes.data, out_len)
    return rc, (out[:out_len] if rc == 0 else None)


def decode(comp, out_len: int | None = None) -> np.ndarray:
    rc, out = decode_rc(comp, out_len)
    if rc:
        raise OracleError(rc, "oracle_decode")
    return out


def parse(comp):
    """Every sequence of the stream: (r, L, s, literal bytes); L = 0 for a sequence without match."""
    c = _u8(comp)
    info = peek(c)
    ns = int(info.n_seq)
    r = np.zeros(max(ns, 1), np.uint64)
    L = np.zeros(max(ns, 1), np.uint64)
    s = np.zeros(max(ns, 1), np.uint64)
    lits = np.zeros(max(int(info.N), 1), np.uint8)
    n = _load().oracle_parse(c.ctypes.data, c.size, r.ctypes.data, L.ctypes.data, s.ctypes.data, lits.ctypes.data, ns)
    if n < 0:
        raise OracleError(n, "oracle_parse")
    n_lit = int(r[:n].sum())
    return r[:n], L[:n], s[:n], lits[:n_lit]


def lz77_rel_decode(r, L, dist, lits, out_len: int) -> np.ndarray:
    r = np.ascontiguousarray(r, np.uint64)
    L = np.ascontiguousarray(L, np.uint64)
    dist = np.ascontiguousarray(dist, np.uint64)
    lits = np.ascontiguousarray(lits, np.uint8)
    out = np.zeros(max(out_len, 1), np.uint8)
    rc = _load().oracle_lz77_rel_decode(r.size, r.ctypes.data, L.ctypes.data, dist.ctypes.data,
                                        lits.ctypes.data if lits.size else None, out.ctypes.data, out_len)
    if rc:
        raise OracleError(rc, "oracle_lz77_rel_decode")
    return out[:out_len]


def depths(comp) -> np.ndarray:
    """Per-match dependency depth (§7.1), in stream order."""
    c = _u8(comp)
    nm = int(peek(c).n_match)
    out = np.zeros(max(nm, 1), np.uint32)
    n = _load().oracle_depths(c.ctypes.data, c.size, out.ctypes.data, nm)
    if n < 0:
        raise OracleError(n, "oracle_depths")
    return out[:n]


def check(comp) -> int:
    """0 when every invariant holds; see oracle_check in oracle.c for the codes."""
    c = _u8(comp)
    return _load().oracle_check(c.ctypes.data, c.size)


def transcode_flat_rc(comp):
    """Global chain flattening of an existing stream (oracle_transcode_flat): (0, stream) or (status, None)."""
    c = _u8(comp)
    ptr = ctypes.c_void_p()
    n = _load().oracle_transcode_flat(c.ctypes.data, c.size, ctypes.byref(ptr))
    if n < 0:
        return int(n), None
    return 0, _take(ptr, n)


def transcode_flat(comp) -> np.ndarray:
    rc, out = transcode_flat_rc(comp)
    if rc:
        raise OracleError(rc, "oracle_transcode_flat")
    return out


def huff_lengths(counts) -> np.ndarray:
    """Code lengths (at most 12) of the entropy container's code for 256 symbol counts."""
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    assert c.size == 256
    out = np.zeros(256, dtype=np.uint8)
    _load().oracle_huff_lengths(c.ctypes.data, out.ctypes.data)
    return out


def entropy_encode(raw) -> np.ndarray:
    """Wrap a stream in the entropy container (format §6)."""
    a = _u8(raw)
    ptr = ctypes.c_void_p()
    n = _load().oracle_entropy_encode(a.ctypes.data, a.size, ctypes.byref(ptr))
    if n < 0:
        raise OracleError(n, "oracle_entropy_encode")
    return _take(ptr, n)


def entropy_decode_rc(e, raw_len: int | None = None):
    """(status, wrapped stream or None) of an entropy container."""
    c = _u8(e)
    if raw_len is None:
        rl, ns = ctypes.c_uint64(), ctypes.c_uint64()
        rc = _load().oracle_entropy_peek(c.ctypes.data, c.size, ctypes.byref(rl), ctypes.byref(ns))
        if rc:
            return rc, None
        raw_len = int(rl.value)
    out = np.zeros(max(raw_len, 1), dtype=np.uint8)
    rc = _load().oracle_entropy_decode(c.ctypes.data, c.size, out.ctypes.data, raw_len)
    return rc, (out[:raw_len] if rc == 0 else None)


def entropy_decode(e) -> np.ndarray:
    rc, out = entropy_decode_rc(e)
    if rc:
        raise OracleError(rc, "oracle_entropy_decode")
    return out
