"""Full-size workloads on the GPU, in the launch configuration the bench times: 1 GiB of English-like text
with full-depth chains (wavefront path), 1 GiB of FASTQ chain-flattened (one-pass path) and depth-capped
at 4 (wavefront path).  Every decoded byte is checked against the input, and the oracle's sequential decode
of the same stream is checked against the input too (the two implementations share no code).  The
streams are encoded once per machine into a file cache that the bench reuses."""
import numpy as np
import pytest
import torch

import bench
import oracle
import paper_2606_04268_gb300 as ax

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GiB = 1 << 30
# the bench's single-stream workloads, with the bench's encoder parameters
FULL = [(bench.WORKLOADS[w][0], bench.WORKLOADS[w][1], bench.stream_seed(bench.WORKLOADS[w][0], 0), bench.WORKLOADS[w][2])
        for w in ("text", "fastq-flat", "fastq-cap4")]


@pytest.fixture(scope="module", autouse=True)
def _streams():
    ax.build()
    oracle.build()
    bench.warm_stream_cache(FULL)
    yield


@pytest.mark.parametrize("spec", FULL, ids=["text-full-depth", "fastq-flat", "fastq-cap4"])
def test_full_size_workload_decodes_exactly(spec):
    kind, n, seed, enc = spec
    x, comp, _ = bench.cached_stream(kind, n, seed, enc)
    info = ax.peek_header(comp[:64])
    assert info.decoded_len == n
    if enc.get("flatten"):
        assert info.max_depth <= 1
    if enc.get("depth_cap"):
        assert 1 < info.max_depth <= enc["depth_cap"]
    d_comp = torch.from_numpy(comp).cuda()
    out = torch.empty(n, dtype=torch.uint8, device="cuda")
    ws = torch.zeros(ax.workspace_size(info), dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    xt = torch.from_numpy(x).cuda()
    for _ in range(2):  # twice on the same workspace, as the bench's back-to-back steps do
        out.fill_(0xA5)
        ax.decode_async(d_comp, out, info, ws, st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0, ax.STATUS_NAMES.get(int(st.item()))
        assert torch.equal(out, xt)
    if info.max_depth > 1:
        ax.decode(d_comp, out)  # the blocking call also reads back the level statistics
        assert torch.equal(out, xt)
        stats = ax.get_stats()
        assert stats["n_levels"] == info.max_depth
        if info.max_depth < ax.HIST_MAX:
            assert int(np.asarray(stats["level_hist"][1:info.max_depth + 1]).sum()) == info.n_match
    rc, ref = oracle.decode_rc(comp, n)
    assert rc == 0 and np.array_equal(ref, x)


def test_full_size_batch_graph_replay():
    """The batched configuration at full size: 4096 streams (256 distinct payloads from the batched mix,
    each placed 16 times), ~8 GiB of output, one plan replayed as a CUDA graph twice."""
    specs, which, N = bench.batch_plan_specs(0)
    pool = bench.encode_pool(specs)
    c_off = np.cumsum([0] + [pool[u][1].size for u in which])
    o_off = np.cumsum([0] + [pool[u][0].size for u in which])
    assert o_off[-1] == N > 6 * GiB
    d_comp = torch.empty(int(c_off[-1]), dtype=torch.uint8, device="cuda")
    uniq = [torch.from_numpy(c).cuda() for _, c in pool]
    for i, u in enumerate(which):
        d_comp[c_off[i]:c_off[i + 1]].copy_(uniq[u])
    del uniq
    d_out = torch.empty(int(o_off[-1]), dtype=torch.uint8, device="cuda")
    comps = [d_comp[c_off[i]:c_off[i + 1]] for i in range(4096)]
    outs = [d_out[o_off[i]:o_off[i + 1]] for i in range(4096)]
    plan = ax.BatchPlan(comps, outs)
    try:
        for _ in range(2):
            d_out.fill_(0x5A)
            plan.launch(graph=True)
            assert (plan.statuses() == 0).all()
            xs = [torch.from_numpy(x).cuda() for x, _ in pool]
            for i, u in enumerate(which):
                assert torch.equal(outs[i], xs[u]), i
            del xs
    finally:
        plan.close()


def test_full_size_text_transcode_matches_oracle():
    """The 1 GiB deep text transcoded on the device into a globally flattened stream: byte-identical to the
    oracle's transcode, and decoded exactly by the one-pass path."""
    kind, n, seed, enc = FULL[0]
    x, comp, _ = bench.cached_stream(kind, n, seed, enc)
    got = ax.transcode_flat(torch.from_numpy(comp).cuda())
    want = oracle.transcode_flat(comp)
    assert got.numel() == want.size and np.array_equal(got.cpu().numpy(), want)
    info = ax.peek_header(want[:64])
    assert info.max_depth == 1
    out = torch.empty(n, dtype=torch.uint8, device="cuda")
    ax.decode(got, out)
    assert torch.equal(out, torch.from_numpy(x).cuda())
