"""Helpers shared by the GPU tests: device round trips through the C ABI with poisoned guard bytes."""
import numpy as np
import torch

import paper_2606_04268_gb300 as ax

POISON = 0xA5
GUARD = 64


def to_dev(comp: np.ndarray) -> torch.Tensor:
    t = torch.from_numpy(np.ascontiguousarray(comp)).cuda()
    assert t.data_ptr() % 16 == 0
    return t


def gpu_decode(comp: np.ndarray, n: int, offset: int = 0, stream=None):
    """Decode through aceapex_decode into a poisoned buffer at byte offset `offset`; returns (status, bytes).
    Asserts that no byte outside [offset, offset + n) was written."""
    d_comp = to_dev(comp)
    buf = torch.full((GUARD + offset + n + GUARD,), POISON, dtype=torch.uint8, device="cuda")
    out = buf[GUARD + offset: GUARD + offset + n]
    rc = ax.decode_status(d_comp, out, stream)
    torch.cuda.synchronize()
    host = buf.cpu().numpy()
    assert np.all(host[:GUARD + offset] == POISON), "write before the output buffer"
    assert np.all(host[GUARD + offset + n:] == POISON), "write after the output buffer"
    return rc, host[GUARD + offset: GUARD + offset + n]


def first_diff(a: np.ndarray, b: np.ndarray):
    if a.size != b.size:
        return f"size {a.size} != {b.size}"
    d = np.nonzero(a != b)[0]
    return None if d.size == 0 else f"{d.size} bytes differ, first at {int(d[0])}"
