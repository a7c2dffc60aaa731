"""Serving: every request decoded by the continuous-batching server (admitted against an HBM budget, its
tiles advanced in shared launches while other requests arrive and run) equals the same request decoded
alone, byte for byte (the method is exact integer work: tolerance zero)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_04268_gb300 as ax
import synth
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def make_requests():
    spec = [("text", 900_000, dict(flatten=2, min_emit=6)), ("fastq", 2_500_000, dict(flatten=2, min_emit=6)),
            ("rle7", 1_300_001, dict(flatten=2)), ("text", 700_000, dict()),           # a deep (unflattened) stream
            ("random", 200_000, dict(flatten=2)), ("text", 5, dict(flatten=2)), ("fastq", 0, dict(flatten=2)),
            ("markov", 333_333, dict(flatten=2, block_log2=16, tile_log2=10)), ("fastq", 4_000_000, dict(depth_cap=4))]
    reqs = []
    for i, (kind, n, kw) in enumerate(spec):
        x = synth.make(kind, n, 900 + i)
        comp = oracle.encode(x, **kw)
        reqs.append((x, comp))
    return reqs


def alone(comp, n):
    d = to_dev(comp)
    out = torch.zeros(n, dtype=torch.uint8, device="cuda")
    assert ax.decode_status(d, out) == 0
    return out.cpu().numpy()


@pytest.mark.parametrize("tiles_per_step", [64, 4096])
def test_server_matches_alone(tiles_per_step):
    reqs = make_requests()
    refs = [alone(c, x.size) for x, c in reqs]
    for (x, _), r in zip(reqs, refs):
        assert np.array_equal(r, x)
    big = max(c.size + x.size for x, c in reqs)
    srv = ax.Server(hbm_budget=2 * big, max_slots=3, tiles_per_step=tiles_per_step)
    d_comps = [to_dev(c) for _, c in reqs]
    ids = []
    pending = list(range(len(reqs)))
    done = {}
    steps = 0
    # requests arrive a few at a time while earlier ones are running
    while pending or len(done) < len(reqs):
        for _ in range(2):
            if pending:
                k = pending.pop(0)
                ids.append((k, srv.submit(d_comps[k])))
        srv.step()
        steps += 1
        for k, rid in ids:
            if k in done:
                continue
            res = srv.poll(rid)
            if res is not None:
                st, _ = res
                assert st == 0, (k, ax.STATUS_NAMES.get(st))
                done[k] = srv.output(rid).cpu().numpy()
                srv.release(rid)
        assert steps < 100000
    for k, (x, _) in enumerate(reqs):
        assert np.array_equal(done[k], refs[k]), k
    srv.close()


def test_server_reports_bad_stream_and_continues():
    x = synth.make("text", 300_000, 3)
    good = oracle.encode(x, flatten=2)
    bad = good.copy()
    b0 = int.from_bytes(bytes(bad[64:72]), "little")
    bad[b0 + 32 + 20 + 16] ^= 1  # a sync entry of block 0
    srv = ax.Server(hbm_budget=1 << 30, max_slots=4, tiles_per_step=8)
    ra = srv.submit(to_dev(bad))
    rb = srv.submit(to_dev(good))
    res = {}
    for _ in range(10000):
        srv.step()
        for rid in (ra, rb):
            if rid not in res:
                p = srv.poll(rid)
                if p is not None:
                    res[rid] = p[0]
                    if rid == rb:
                        assert np.array_equal(srv.output(rid).cpu().numpy(), x)
        if len(res) == 2:
            break
    assert res[ra] == ax.ERR_FORMAT and res[rb] == 0
    srv.close()
