"""Byte edits of ACEAPEX streams for tests (stream format §1.1, §2.1): rewrite the depth fields of the
block headers and the stream header.  No decoding logic."""
import numpy as np


def block_offsets(comp):
    nb = int.from_bytes(bytes(comp[24:32]), "little")
    return [int.from_bytes(bytes(comp[64 + 8 * b:72 + 8 * b]), "little") for b in range(nb)]


def block_depths(comp):
    return [int.from_bytes(bytes(comp[o + 24:o + 28]), "little") for o in block_offsets(comp)]


def set_depths(comp, block_depths_, stream_depth):
    """Overwrite the blocks' and the stream's max_depth fields."""
    c = comp.copy()
    for off, dep in zip(block_offsets(c), block_depths_):
        c[off + 24:off + 28] = np.frombuffer(int(dep).to_bytes(4, "little"), np.uint8)
    c[48:52] = np.frombuffer(int(stream_depth).to_bytes(4, "little"), np.uint8)
    return c


def lower_depths(comp, to=1):
    """Every depth field clipped to `to`: a stream whose headers understate its matches' depths."""
    deps = [min(d, to) for d in block_depths(comp)]
    return set_depths(comp, deps, max(deps, default=0))
