"""GB300 ACEAPEX stream decoder: Python binding of libaceapex.so (C ABI in include/aceapex.h).

Argument marshalling only: every step of the decode runs in the library's CUDA kernels, and the encoder
in its C++ code.  PyTorch supplies device memory and streams.  Importing this module never falls back to
anything: if the shared library is missing, calls raise.

    import paper_2606_04268_gb300 as ax
    comp = ax.encode(data_bytes, flatten=2)            # numpy uint8 stream (CPU encoder)
    d_comp = torch.from_numpy(comp).cuda()
    d_out = torch.empty(n, dtype=torch.uint8, device="cuda")
    ax.decode(d_comp, d_out)                           # raises AceapexError on a bad stream
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
LIB_PATH = os.path.join(_HERE, "libaceapex.so")
_SOURCES = ["decode.cu", "api.cpp", "encoder.cpp", "serve.cpp", "transcode.cu", "entropy.cu", "entropy_enc.cpp"]
_HEADERS = ["decode.h", "layout.h", "device_common.cuh", "tile.cuh", "warp_tile.cuh", "onepass.cuh", "wave.cuh"]
NVCC_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

OK, ERR_ARG, ERR_FORMAT, ERR_SIZE, ERR_OFFSET, ERR_TIMEOUT, ERR_CUDA, ERR_NOMEM, ERR_DEPTH = 0, -1, -2, -3, -4, -5, -6, -7, -8
STATUS_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_FORMAT", -3: "ERR_SIZE", -4: "ERR_OFFSET", -5: "ERR_TIMEOUT",
                -6: "ERR_CUDA", -7: "ERR_NOMEM", -8: "ERR_DEPTH"}
FLAT_NONE, FLAT_BLOCK, FLAT_GLOBAL = 0, 1, 2
HIST_MAX = 4096


class AceapexError(RuntimeError):
    def __init__(self, code: int, what: str = "aceapex"):
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)}")
        self.code = code


# ---------------------------------------------------------------------------------------------- build
def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(_CSRC, f) for f in _SOURCES + _HEADERS] + [os.path.join(_INCLUDE, "aceapex.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libaceapex.so for sm_103a in-tree (nvcc, one -gencode, translation units in parallel)."""
    if not force and not _stale():
        return LIB_PATH
    nvcc = _nvcc()
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    objdir = os.path.join(_HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    common = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", f"-I{_INCLUDE}"] + NVCC_ARCH

    def compile_one(src: str) -> str:
        obj = os.path.join(objdir, src + f".{os.getpid()}.o")
        cmd = [nvcc] + common + ["-c", os.path.join(_CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(_SOURCES)) as ex:
        objs = list(ex.map(compile_one, _SOURCES))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    link = [nvcc] + NVCC_ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + \
        ["-Xlinker", f"-rpath,{cuda_lib}"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    for o in objs:
        os.remove(o)
    return LIB_PATH


# ---------------------------------------------------------------------------------------------- ctypes
class Info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("decoded_len", "n_blocks", "comp_len", "n_match", "n_seq", "n_tiles")] + \
               [(n, ctypes.c_uint32) for n in ("block_log2", "tile_log2", "min_match", "flatten", "depth_cap", "max_depth")]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("decoded_len", "comp_len", "n_match", "n_tiles")] + \
               [(n, ctypes.c_uint32) for n in ("max_depth", "one_pass", "n_levels", "hist_len")] + \
               [("level_hist", ctypes.c_uint64 * HIST_MAX), ("phase_cycles", ctypes.c_uint64 * 8)]


class EntropyInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("raw_len", "n_seg", "e_len")]


class DeviceModel(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("cpu_gbps", "gpu_one_pass_gbps", "gpu_wave_gbps", "gpu_level_us", "gpu_fixed_us", "link_gbps")]


class EncParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ("block_log2", "tile_log2", "min_match", "hash_bits", "chain_limit", "flatten", "depth_cap",
                 "use_first", "min_emit", "long_bits", "long_chain")]


# every exported symbol of include/aceapex.h
SYMBOLS = ["aceapex_peek_header", "aceapex_workspace_size", "aceapex_decode", "aceapex_decode_async",
           "aceapex_decode_noalloc",
           "aceapex_decode_batch", "aceapex_batch_plan_create", "aceapex_batch_plan_launch",
           "aceapex_batch_plan_statuses", "aceapex_batch_plan_statuses_device", "aceapex_batch_plan_destroy", "aceapex_set_launch_config",
           "aceapex_decode_host", "aceapex_decode_batch_host", "aceapex_get_launch_config", "aceapex_set_wave_scheduler", "aceapex_set_force_wavefront", "aceapex_set_wait_limit", "aceapex_profile",
           "aceapex_profile_read", "aceapex_get_stats", "aceapex_strerror",
           "aceapex_server_create", "aceapex_server_submit", "aceapex_server_step", "aceapex_server_poll",
           "aceapex_server_release", "aceapex_server_destroy",
           "aceapex_encode", "aceapex_free", "aceapex_choose_device",
           "aceapex_transcode_create", "aceapex_transcode_write", "aceapex_transcode_info", "aceapex_transcode_destroy",
           "aceapex_entropy_peek", "aceapex_entropy_decode", "aceapex_entropy_encode"]

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libaceapex.so; raises if it has not been built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_2606_04268_gb300.build() first")
            L = ctypes.CDLL(LIB_PATH)
            p, sz, i32, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64
            L.aceapex_peek_header.argtypes = [p, sz, ctypes.POINTER(Info)]
            L.aceapex_workspace_size.argtypes = [ctypes.POINTER(Info)]
            L.aceapex_workspace_size.restype = sz
            L.aceapex_decode.argtypes = [p, sz, p, sz, p]
            L.aceapex_decode_async.argtypes = [p, sz, p, sz, ctypes.POINTER(Info), p, sz, p, p]
            L.aceapex_decode_noalloc.argtypes = [p, sz, p, sz, ctypes.POINTER(Info), p, p]
            L.aceapex_decode_batch.argtypes = [i32, p, p, p, p, p, p]
            L.aceapex_batch_plan_create.argtypes = [i32, p, p, p, p, p, ctypes.POINTER(p)]
            L.aceapex_batch_plan_launch.argtypes = [p, i32, p]
            L.aceapex_batch_plan_statuses.argtypes = [p, p, p]
            L.aceapex_batch_plan_destroy.argtypes = [p]
            L.aceapex_batch_plan_statuses_device.argtypes = [p, p, p]
            L.aceapex_set_launch_config.argtypes = [i32, i32]
            L.aceapex_get_launch_config.argtypes = [ctypes.POINTER(ctypes.c_int)] * 2
            L.aceapex_set_force_wavefront.argtypes = [i32]
            L.aceapex_decode_host.argtypes = [p, sz, p, sz, p]
            L.aceapex_decode_batch_host.argtypes = [i32, p, p, p, p, p, p]
            L.aceapex_set_wave_scheduler.argtypes = [i32]
            L.aceapex_set_wait_limit.argtypes = [u64, u64]
            L.aceapex_profile.argtypes = [i32]
            L.aceapex_profile_read.argtypes = [i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_uint64)]
            L.aceapex_get_stats.argtypes = [ctypes.POINTER(Stats)]
            L.aceapex_strerror.argtypes = [i32]
            L.aceapex_strerror.restype = ctypes.c_char_p
            L.aceapex_server_create.argtypes = [sz, i32, u64, ctypes.POINTER(p)]
            L.aceapex_server_submit.argtypes = [p, p, sz, ctypes.POINTER(Info)]
            L.aceapex_server_submit.restype = ctypes.c_int64
            L.aceapex_server_step.argtypes = [p, p]
            L.aceapex_server_poll.argtypes = [p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(p)]
            L.aceapex_server_release.argtypes = [p, ctypes.c_int64, p]
            L.aceapex_server_destroy.argtypes = [p]
            L.aceapex_entropy_peek.argtypes = [p, sz, ctypes.POINTER(EntropyInfo)]
            L.aceapex_entropy_encode.argtypes = [p, sz, ctypes.POINTER(p), ctypes.POINTER(sz)]
            L.aceapex_entropy_decode.argtypes = [p, sz, ctypes.POINTER(EntropyInfo), p, sz, p, p]
            L.aceapex_transcode_create.argtypes = [p, sz, ctypes.POINTER(p), ctypes.POINTER(sz), p]
            L.aceapex_transcode_write.argtypes = [p, p, sz, p]
            L.aceapex_transcode_info.argtypes = [p, ctypes.POINTER(u64), ctypes.POINTER(u64)]
            L.aceapex_transcode_destroy.argtypes = [p]
            L.aceapex_choose_device.argtypes = [ctypes.POINTER(Info), ctypes.POINTER(DeviceModel),
                                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            L.aceapex_encode.argtypes = [p, sz, ctypes.POINTER(EncParams), ctypes.POINTER(p)]
            L.aceapex_encode.restype = ctypes.c_int64
            L.aceapex_free.argtypes = [p]
            L.aceapex_free.restype = None
            _lib = L
    return _lib


def _check(rc: int, what: str) -> int:
    if rc != 0:
        raise AceapexError(rc, what)
    return rc


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dev_ptr(t) -> int:
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.uint8 and t.is_contiguous(), \
        "expected a contiguous uint8 CUDA tensor"
    return t.data_ptr()


# ---------------------------------------------------------------------------------------------- API
def strerror(code: int) -> str:
    return lib().aceapex_strerror(code).decode()


def peek_header(prefix) -> Info:
    a = np.ascontiguousarray(np.frombuffer(prefix, np.uint8) if isinstance(prefix, (bytes, bytearray)) else prefix)
    info = Info()
    _check(lib().aceapex_peek_header(a.ctypes.data, a.size, ctypes.byref(info)), "aceapex_peek_header")
    return info


def workspace_size(info: Info) -> int:
    return lib().aceapex_workspace_size(ctypes.byref(info))


def decode_status(comp, out, stream=None) -> int:
    """Decode device stream `comp` into device buffer `out` (blocking); returns the status code."""
    return lib().aceapex_decode(_dev_ptr(comp), comp.numel(), _dev_ptr(out) if out.numel() else None,
                                out.numel(), _stream_ptr(stream))


def decode(comp, out, stream=None):
    _check(decode_status(comp, out, stream), "aceapex_decode")
    return out


def _host_ptr(a) -> tuple[int, int]:
    """(address, byte length) of a contiguous host numpy array or CPU tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"] and a.dtype == np.uint8
        return a.ctypes.data, a.size
    assert not a.is_cuda and a.is_contiguous() and a.element_size() == 1
    return a.data_ptr(), a.numel()


def decode_host_status(comp, out, stream=None) -> int:
    """Decode a stream in host memory into a host buffer (aceapex_decode_host); returns the status code.
    comp/out: uint8 numpy arrays or CPU tensors (pinned memory lets the copies overlap the decode)."""
    cp, cn = _host_ptr(comp)
    op, on = _host_ptr(out)
    return lib().aceapex_decode_host(cp, cn, op if on else None, on, _stream_ptr(stream))


def decode_host(comp, out, stream=None):
    _check(decode_host_status(comp, out, stream), "aceapex_decode_host")
    return out


def decode_async(comp, out, info: Info, workspace, status, stream=None) -> None:
    """Enqueue a decode with no host synchronisation; `workspace` is a zero-filled uint8 CUDA tensor of at
    least workspace_size(info) bytes, `status` an int32 CUDA tensor of one element."""
    import torch
    assert status.is_cuda and status.dtype == torch.int32
    _check(lib().aceapex_decode_async(_dev_ptr(comp), comp.numel(), _dev_ptr(out) if out.numel() else None,
                                      out.numel(), ctypes.byref(info), _dev_ptr(workspace), workspace.numel(),
                                      status.data_ptr(), _stream_ptr(stream)), "aceapex_decode_async")


def decode_noalloc(comp, out, info: Info, status, stream=None) -> None:
    """Decode without allocating: the library's static device scratch replaces the workspace (see
    aceapex_decode_noalloc).  For callers that cannot allocate device memory while decoding."""
    import torch
    assert status.is_cuda and status.dtype == torch.int32
    _check(lib().aceapex_decode_noalloc(_dev_ptr(comp), comp.numel(), _dev_ptr(out) if out.numel() else None,
                                        out.numel(), ctypes.byref(info), status.data_ptr(), _stream_ptr(stream)),
           "aceapex_decode_noalloc")


def _arrays(comps, outs):
    n = len(comps)
    cp = (ctypes.c_void_p * n)(*[_dev_ptr(c) for c in comps])
    op = (ctypes.c_void_p * n)(*[_dev_ptr(o) if o.numel() else None for o in outs])
    cl = (ctypes.c_size_t * n)(*[c.numel() for c in comps])
    ol = (ctypes.c_size_t * n)(*[o.numel() for o in outs])
    return n, cp, cl, op, ol


def decode_batch(comps, outs, stream=None) -> np.ndarray:
    """Decode many streams (blocking); returns the per-stream status codes."""
    n, cp, cl, op, ol = _arrays(comps, outs)
    st = np.zeros(max(n, 1), np.int32)
    lib().aceapex_decode_batch(n, cp, cl, op, ol, st.ctypes.data, _stream_ptr(stream))
    return st[:n]


class HostBatch:
    """Pointer and length arrays of n host-memory streams and their host outputs, for decode_batch_host.
    comps/outs: uint8 numpy arrays or CPU tensors (pinned memory lets the copies overlap the decodes).
    Built once, the arrays serve every later call on the same buffers."""

    def __init__(self, comps, outs):
        assert len(comps) == len(outs)
        self._keep = (list(comps), list(outs))
        n = len(comps)
        c = [_host_ptr(x) for x in comps]
        o = [_host_ptr(x) for x in outs]
        self.n = n
        self.cp = (ctypes.c_void_p * max(n, 1))(*[a for a, _ in c])
        self.cl = (ctypes.c_size_t * max(n, 1))(*[b for _, b in c])
        self.op = (ctypes.c_void_p * max(n, 1))(*[a if b else None for a, b in o])
        self.ol = (ctypes.c_size_t * max(n, 1))(*[b for _, b in o])
        self.statuses = np.zeros(max(n, 1), np.int32)


def decode_batch_host_status(batch: "HostBatch", stream=None) -> int:
    """Decode the streams of a HostBatch from host memory into its host outputs (aceapex_decode_batch_host:
    copies in, decodes and copies out overlapped).  Returns the first failing status (0: all decoded); the
    per-stream statuses are in batch.statuses[:batch.n]."""
    return lib().aceapex_decode_batch_host(batch.n, batch.cp, batch.cl, batch.op, batch.ol,
                                           batch.statuses.ctypes.data, _stream_ptr(stream))


def decode_batch_host(comps, outs, stream=None) -> np.ndarray:
    """Decode many streams held in host memory into host buffers (blocking); returns the per-stream
    status codes."""
    b = HostBatch(comps, outs)
    decode_batch_host_status(b, stream)
    return b.statuses[:b.n].copy()


class BatchPlan:
    """Decode plan over fixed buffers: headers read once; launches optionally replayed as a CUDA graph."""

    def __init__(self, comps, outs, stream=None):
        self._keep = (list(comps), list(outs))
        n, cp, cl, op, ol = _arrays(comps, outs)
        self.n = n
        self._h = ctypes.c_void_p()
        _check(lib().aceapex_batch_plan_create(n, cp, cl, op, ol, _stream_ptr(stream), ctypes.byref(self._h)),
               "aceapex_batch_plan_create")

    def launch(self, graph: bool = False, stream=None) -> None:
        _check(lib().aceapex_batch_plan_launch(self._h, int(graph), _stream_ptr(stream)), "aceapex_batch_plan_launch")

    def statuses(self, stream=None) -> np.ndarray:
        st = np.zeros(max(self.n, 1), np.int32)
        lib().aceapex_batch_plan_statuses(self._h, st.ctypes.data, _stream_ptr(stream))
        return st[:self.n]

    def statuses_device(self, out, stream=None) -> None:
        """Write the per-stream statuses into the device int32 tensor out (stream-ordered, no host sync)."""
        _check(lib().aceapex_batch_plan_statuses_device(self._h, out.data_ptr(), _stream_ptr(stream)),
               "aceapex_batch_plan_statuses_device")

    def close(self) -> None:
        if self._h:
            lib().aceapex_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching decode server (aceapex_server_*): submit device-resident streams, call step()
    repeatedly; each step admits what fits the HBM budget and advances every admitted request by a slice of
    its tiles in one shared launch."""

    def __init__(self, hbm_budget: int = 64 << 30, max_slots: int = 64, tiles_per_step: int = 65536):
        self._h = ctypes.c_void_p()
        _check(lib().aceapex_server_create(int(hbm_budget), int(max_slots), int(tiles_per_step), ctypes.byref(self._h)),
               "aceapex_server_create")
        self._keep = {}

    def submit(self, comp, info: Info | None = None) -> int:
        if info is None:
            info = peek_header(comp[:64].cpu().numpy())
        rid = lib().aceapex_server_submit(self._h, _dev_ptr(comp), comp.numel(), ctypes.byref(info))
        if rid < 0:
            raise AceapexError(int(rid), "aceapex_server_submit")
        self._keep[rid] = (comp, info)
        return int(rid)

    def step(self, stream=None) -> int:
        rc = lib().aceapex_server_step(self._h, _stream_ptr(stream))
        if rc < 0:
            raise AceapexError(rc, "aceapex_server_step")
        return rc

    def poll(self, rid: int):
        """None while pending, else (status, device pointer of the output)."""
        st = ctypes.c_int32()
        ptr = ctypes.c_void_p()
        rc = lib().aceapex_server_poll(self._h, int(rid), ctypes.byref(st), ctypes.byref(ptr))
        if rc < 0:
            raise AceapexError(rc, "aceapex_server_poll")
        return None if rc == 0 else (int(st.value), ptr.value)

    def output(self, rid: int):
        """Copy of a finished request's output as a uint8 CUDA tensor."""
        import torch
        res = self.poll(rid)
        assert res is not None, "request not finished"
        n = int(self._keep[rid][1].decoded_len)
        out = torch.empty(n, dtype=torch.uint8, device="cuda")
        if n:
            out.copy_(_wrap_ptr(res[1], n))
        return out

    def release(self, rid: int, stream=None) -> None:
        _check(lib().aceapex_server_release(self._h, int(rid), _stream_ptr(stream)), "aceapex_server_release")
        self._keep.pop(rid, None)

    def close(self) -> None:
        if self._h:
            lib().aceapex_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _wrap_ptr(ptr: int, n: int):
    """A uint8 CUDA tensor view of n bytes at a raw device pointer (no ownership)."""
    import torch

    class _Holder:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "|u1", "data": (ptr, False), "version": 3}
    return torch.as_tensor(_Holder(), device="cuda")


def set_launch_config(warps_per_cta: int = 4, ctas_per_sm: int = 0) -> None:
    """Launch shape of the one-pass kernel: warps per CTA (2, 4 or 8) and CTAs per SM (0 = as many as fit)."""
    _check(lib().aceapex_set_launch_config(int(warps_per_cta), int(ctas_per_sm)), "aceapex_set_launch_config")


def get_launch_config():
    w, c = ctypes.c_int(), ctypes.c_int()
    _check(lib().aceapex_get_launch_config(ctypes.byref(w), ctypes.byref(c)), "get_launch_config")
    return w.value, c.value


def choose_device(info: Info, cpu_gbps: float, link_gbps: float = 0.0, **model) -> tuple:
    """Pre-scan choice between a CPU and a GPU decode from the stream's header (aceapex_choose_device):
    returns ("gpu" or "cpu", estimated CPU seconds, estimated GPU seconds).  model: gpu_one_pass_gbps,
    gpu_wave_gbps, gpu_level_us, gpu_fixed_us (0 = the library's GB300 defaults)."""
    m = DeviceModel(cpu_gbps, model.get("gpu_one_pass_gbps", 0.0), model.get("gpu_wave_gbps", 0.0),
                    model.get("gpu_level_us", 0.0), model.get("gpu_fixed_us", 0.0), link_gbps)
    tc, tg = ctypes.c_double(), ctypes.c_double()
    rc = lib().aceapex_choose_device(ctypes.byref(info), ctypes.byref(m), ctypes.byref(tc), ctypes.byref(tg))
    if rc < 0:
        raise AceapexError(rc, "aceapex_choose_device")
    return ("gpu" if rc == 1 else "cpu"), tc.value, tg.value


def entropy_encode(raw) -> np.ndarray:
    """Wrap a host stream in the entropy container with the library's CPU encoder (aceapex_entropy_encode)."""
    a = np.ascontiguousarray(raw, dtype=np.uint8)
    ptr, n = ctypes.c_void_p(), ctypes.c_size_t()
    _check(lib().aceapex_entropy_encode(a.ctypes.data if a.size else None, a.size, ctypes.byref(ptr), ctypes.byref(n)),
           "aceapex_entropy_encode")
    out = np.empty(n.value, np.uint8)
    ctypes.memmove(out.ctypes.data, ptr, n.value)
    lib().aceapex_free(ptr)
    return out


def entropy_peek(host_prefix) -> EntropyInfo:
    """Header of an entropy container (aceapex_entropy_peek) from its first 64 bytes in host memory."""
    b = np.ascontiguousarray(np.asarray(host_prefix, dtype=np.uint8)[:64])
    info = EntropyInfo()
    _check(lib().aceapex_entropy_peek(b.ctypes.data, b.size, ctypes.byref(info)), "aceapex_entropy_peek")
    return info


def entropy_decode_async(e, info: EntropyInfo, raw, status, stream=None) -> None:
    """Enqueue the decode of the device entropy container e into the device buffer raw (the wrapped stream);
    status: device int32 tensor receiving 0 or ERR_FORMAT."""
    _check(lib().aceapex_entropy_decode(e.data_ptr(), e.numel(), ctypes.byref(info), raw.data_ptr(), raw.numel(),
                                        status.data_ptr(), _stream_ptr(stream)), "aceapex_entropy_decode")


def entropy_decode(e, stream=None):
    """The wrapped stream of a device entropy container, as a new uint8 device tensor (blocking)."""
    import torch
    info = entropy_peek(e[:64].cpu().numpy())
    raw = torch.empty(max(int(info.raw_len), 16), dtype=torch.uint8, device=e.device)[:int(info.raw_len)]
    status = torch.zeros(1, dtype=torch.int32, device=e.device)
    entropy_decode_async(e, info, raw, status, stream)
    st = int(status.item())
    if st:
        raise AceapexError(st, "aceapex_entropy_decode")
    return raw


class Transcode:
    """Global chain flattening of a device-resident stream into a new stream whose matches all read literal
    bytes, so that the one-pass kernel decodes it (aceapex_transcode_*; chain flattening §3.3 applied to an
    existing stream).  Creating it runs the analysis on the GPU (decode, roots, rewritten matches, block
    layout); write() serializes the new stream into a device buffer of at least out_len bytes."""

    def __init__(self, comp, stream=None):
        import torch
        self._h = ctypes.c_void_p()
        n = ctypes.c_size_t()
        _check(lib().aceapex_transcode_create(comp.data_ptr(), comp.numel(), ctypes.byref(self._h), ctypes.byref(n),
                                              _stream_ptr(stream)), "aceapex_transcode_create")
        self.out_len = int(n.value)
        nm, ns = ctypes.c_uint64(), ctypes.c_uint64()
        lib().aceapex_transcode_info(self._h, ctypes.byref(nm), ctypes.byref(ns))
        self.n_match, self.n_seq = int(nm.value), int(ns.value)

    def write(self, out, stream=None) -> None:
        _check(lib().aceapex_transcode_write(self._h, out.data_ptr(), out.numel(), _stream_ptr(stream)),
               "aceapex_transcode_write")

    def close(self) -> None:
        if self._h:
            lib().aceapex_transcode_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def transcode_flat(comp, stream=None):
    """The globally flattened form of a device-resident stream, as a new uint8 device tensor."""
    import torch
    t = Transcode(comp, stream)
    try:
        out = torch.empty(max(t.out_len, 16), dtype=torch.uint8, device=comp.device)[:t.out_len]
        t.write(out, stream)
        return out
    finally:
        t.close()


def set_wave_scheduler(kind: int) -> None:
    """Scheduler of the wavefront path: 2 warp dataflow (default); 1 per-level queues with a grid barrier
    per level; 0 per-match dataflow."""
    _check(lib().aceapex_set_wave_scheduler(int(kind)), "aceapex_set_wave_scheduler")


def set_force_wavefront(on: bool) -> None:
    lib().aceapex_set_force_wavefront(int(on))


def set_wait_limit(ns: int = 0, withhold_tile: int | None = None) -> None:
    """Bounded-wait limit (0 = default 4 s) and the test hook that withholds one tile's flag."""
    lib().aceapex_set_wait_limit(int(ns), (1 << 64) - 1 if withhold_tile is None else int(withhold_tile))


def profile(enable: bool) -> None:
    """Start (clearing totals) or stop recording CUDA-event times around every library kernel."""
    lib().aceapex_profile(int(enable))


def profile_read() -> dict:
    """{kernel name: (total ms, launches)} accumulated since profile(True)."""
    k = 32
    names = (ctypes.c_char_p * k)()
    ms = (ctypes.c_double * k)()
    n = (ctypes.c_uint64 * k)()
    cnt = lib().aceapex_profile_read(k, names, ms, n)
    return {names[i].decode(): (ms[i], int(n[i])) for i in range(min(cnt, k))}


def get_stats() -> dict:
    s = Stats()
    _check(lib().aceapex_get_stats(ctypes.byref(s)), "aceapex_get_stats")
    return dict(decoded_len=s.decoded_len, comp_len=s.comp_len, n_match=s.n_match, n_tiles=s.n_tiles,
                max_depth=s.max_depth, one_pass=bool(s.one_pass), n_levels=s.n_levels,
                level_hist=np.array(s.level_hist[:s.hist_len], dtype=np.uint64),
                phase_cycles=dict(zip(PHASE_NAMES, list(s.phase_cycles))))


PHASE_NAMES = ["open", "parse", "literals", "store_publish", "wait", "matches", "store", "tiles"]


def encode(data, block_log2=20, tile_log2=12, min_match=4, hash_bits=20, chain_limit=16, flatten=FLAT_NONE,
           depth_cap=0, use_first=1, min_emit=0, long_bits=0, long_chain=4) -> np.ndarray:
    """Encode host bytes with the library's CPU encoder; returns the stream as a uint8 numpy array."""
    a = np.ascontiguousarray(np.frombuffer(data, np.uint8) if isinstance(data, (bytes, bytearray)) else data)
    assert a.dtype == np.uint8
    prm = EncParams(block_log2, tile_log2, min_match, hash_bits, chain_limit, flatten, depth_cap, use_first, min_emit,
                    long_bits, long_chain)
    ptr = ctypes.c_void_p()
    n = lib().aceapex_encode(a.ctypes.data if a.size else None, a.size, ctypes.byref(prm), ctypes.byref(ptr))
    if n < 0:
        raise AceapexError(int(n), "aceapex_encode")
    out = np.empty(n, np.uint8)
    ctypes.memmove(out.ctypes.data, ptr, n)
    lib().aceapex_free(ptr)
    return out


def encode_many(items, threads: int | None = None, **params):
    """Encode several inputs in parallel threads (the C++ encoder releases the GIL through ctypes)."""
    with ThreadPoolExecutor(max_workers=threads or os.cpu_count()) as ex:
        return list(ex.map(lambda x: encode(x, **params), items))
