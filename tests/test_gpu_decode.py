"""GPU decode through the C ABI against the CPU oracle, byte for byte (the method is exact integer work,
so the tolerance is zero).  Inputs are oracle-encoded; expected bytes are the original input, which the
oracle's own decode also reproduces."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_04268_gb300 as ax
import synth
from gpu_util import first_diff, gpu_decode, to_dev
from stream_edit import block_depths, lower_depths, set_depths

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ax.build()
    ax.set_force_wavefront(False)
    ax.set_wait_limit(0)
    yield
    ax.set_force_wavefront(False)
    ax.set_wait_limit(0)


def set_path(path: str):
    """auto: the one-pass kernel for the streams it takes (depth <= 1, tiles <= 4 KiB), warp dataflow for the
    others; w2 / w8: the same with 2 / 8 warps per CTA of the one-pass kernel; wave: level queues for every
    stream; flow: per-match dataflow for every stream; wflow: warp dataflow for every stream."""
    ax.set_force_wavefront(path in ("wave", "flow", "wflow"))
    ax.set_wave_scheduler({"flow": 0, "wave": 1}.get(path, 2))
    ax.set_launch_config({"w2": 2, "w8": 8}.get(path, 4), 0)


def check(x: np.ndarray, comp: np.ndarray, path: str = "auto", offset: int = 0):
    set_path(path)
    try:
        rc, got = gpu_decode(comp, x.size, offset)
    finally:
        set_path("auto")
    assert rc == 0, ax.STATUS_NAMES.get(rc, rc)
    assert first_diff(got, x) is None, first_diff(got, x)
    return got


def test_small_text_workload_matches_oracle():
    """4 MiB Markov text, 4 blocks of 1 MiB, greedy parse, min match 4, no flattening."""
    x = synth.markov_text(4 << 20, 1000)
    comp = oracle.encode(x, min_match=4)
    assert oracle.peek(comp).n_blocks == 4
    ref = oracle.decode(comp)
    assert np.array_equal(ref, x)
    for path in ("auto", "wave", "flow", "wflow"):
        got = check(x, comp, path)
        assert np.array_equal(got, ref)


KINDS = ["markov", "text", "fastq", "random", "rle7"]
MODES = {"plain": dict(), "block": dict(flatten=1), "global": dict(flatten=2, min_emit=6),
         "cap4": dict(depth_cap=4, min_emit=6), "cap1": dict(depth_cap=1)}
SHAPES = [(20, 14), (16, 10), (12, 6), (10, 2)]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"B{s[0]}T{s[1]}")
def test_kinds_modes_shapes(kind, mode, shape):
    n = 700_001 if shape[0] >= 16 else 90_001
    x = synth.make(kind, n, hash((kind, mode, shape)) & 0xFFFF)
    comp = oracle.encode(x, block_log2=shape[0], tile_log2=shape[1], **MODES[mode])
    for path in ("auto", "w2", "w8", "wave", "flow", "wflow"):
        check(x, comp, path)


@pytest.mark.parametrize("n", [1, 2, 15, 16, 17, 4095, 4096, 4097, (1 << 20) - 1, 1 << 20, (1 << 20) + 1,
                               (3 << 20) + 12345])
@pytest.mark.parametrize("kind", ["text", "rle7", "random"])
def test_sizes_and_ragged_tails(n, kind):
    x = synth.make(kind, n, n)
    for kw in (dict(), dict(flatten=2)):
        comp = oracle.encode(x, **kw)
        check(x, comp, "auto")
        check(x, comp, "w8")


def test_empty_stream():
    comp = oracle.encode(np.zeros(0, np.uint8))
    d = to_dev(comp)
    out = torch.empty(0, dtype=torch.uint8, device="cuda")
    assert ax.decode_status(d, out) == 0


@pytest.mark.parametrize("period", list(range(1, 34)))
def test_self_overlapping_periods(period):
    """Period-p data gives matches whose source overlaps their destination (RLE-like copies)."""
    rng = np.random.default_rng(period)
    motif = rng.integers(0, 256, period, dtype=np.uint8)
    x = np.tile(motif, 60_000 // period + 1)[:60_000].copy()
    x[rng.integers(0, x.size, 20)] = rng.integers(0, 256, 20, dtype=np.uint8)
    for kw in (dict(block_log2=14, tile_log2=8), dict(block_log2=14, tile_log2=8, flatten=2)):
        comp = oracle.encode(x, **kw)
        r, L, s, _ = oracle.parse(comp)
        d = np.cumsum(r + L) - L
        if period > 1:
            assert np.any((L > 0) & (d - s < L)), "expected self-overlapping matches"
        for path in ("auto", "w2", "w8", "wave", "flow", "wflow"):
            check(x, comp, path)


@pytest.mark.parametrize("offset", list(range(1, 16)))
def test_unaligned_output(offset):
    x = synth.make("text", 50_000, offset)
    comp = oracle.encode(x, block_log2=12, tile_log2=5, flatten=2)
    check(x, comp, "auto", offset=offset)
    check(x, comp, "wave", offset=offset)
    check(x, comp, "wflow", offset=offset)
    check(x, comp, "w2", offset=offset)


@pytest.mark.parametrize("path", ["auto", "wave", "flow", "wflow"])
def test_level_histogram_matches_oracle_depths(path):
    x = synth.make("text", 3 << 20, 77)
    comp = oracle.encode(x)
    dep = oracle.depths(comp)
    check(x, comp, path)
    st = ax.get_stats()
    assert not st["one_pass"] and st["max_depth"] == dep.max()
    hist = np.bincount(dep, minlength=int(dep.max()) + 1)
    assert np.array_equal(st["level_hist"][:hist.size].astype(np.int64), hist)
    assert st["n_levels"] == dep.max()


def _mut(comp, off, width, value):
    c = comp.copy()
    c[off:off + width] = np.frombuffer(int(value).to_bytes(width, "little"), np.uint8)
    return c


def malformed_cases():
    x = synth.make("text", 30_000, 9)
    comp = oracle.encode(x, block_log2=12, tile_log2=8)
    flat = oracle.encode(x, block_log2=12, tile_log2=8, flatten=2)
    b0 = int.from_bytes(bytes(comp[64:72]), "little")
    b1 = int.from_bytes(bytes(comp[72:80]), "little")
    nt = int.from_bytes(bytes(comp[b0 + 28:b0 + 32]), "little")
    cmd = int.from_bytes(bytes(comp[b0 + 12:b0 + 16]), "little")
    a16 = lambda v: (v + 15) & ~15
    o_cmd = b0 + a16(32 + 20 * nt)
    cases = {
        "magic": _mut(comp, 0, 4, 0x12345678), "version": _mut(comp, 4, 2, 7), "flags": _mut(comp, 6, 2, 3),
        "block_log2": _mut(comp, 8, 1, 25), "tile_gt_block": _mut(comp, 9, 1, 13), "n_blocks": _mut(comp, 24, 8, 99),
        "n_match": _mut(comp, 40, 8, 5), "n_seq": _mut(comp, 56, 8, 7), "max_depth": _mut(comp, 48, 4, 1),
        "index": _mut(comp, 72, 8, b1 + 16), "index_misaligned": _mut(comp, 72, 8, b1 + 4),
        "off_width": _mut(comp, b0 + 20, 1, 9), "n_tiles": _mut(comp, b0 + 28, 4, nt + 1),
        "sync_out": _mut(comp, b0 + 32 + 20 + 16, 4, 3), "sync_seq": _mut(comp, b0 + 32 + 20, 4, 1),
        "varint_run": _mut(comp, o_cmd, 4, 0xFFFFFFFF), "cmd_bytes": _mut(comp, b0 + 12, 4, cmd + 1),
        "flat_depth_lie": _mut(flat, 48, 4, 0),
        "truncated": comp[:-16], "comp_len_field": _mut(comp, 32, 8, comp.size + 16),
    }
    return x, cases


@pytest.mark.parametrize("name", sorted(malformed_cases()[1]))
def test_malformed_stream_rejected_like_oracle(name):
    x, cases = malformed_cases()
    c = cases[name]
    rc_o, _ = oracle.decode_rc(c, out_len=x.size)
    assert rc_o != 0
    for path in ("auto", "w2", "w8", "wave", "flow", "wflow"):
        set_path(path)
        try:
            rc, _ = gpu_decode(c, x.size)
        finally:
            set_path("auto")
        assert rc != 0, f"{name}/{path}: accepted"
        assert rc == rc_o, f"{name}/{path}: {ax.STATUS_NAMES.get(rc)} vs oracle {oracle.ERR.get(rc_o)}"


def test_wrong_out_len_and_misaligned_comp():
    x = synth.make("text", 10_000, 1)
    comp = oracle.encode(x)
    rc, _ = gpu_decode(comp, x.size + 1)
    assert rc == ax.ERR_SIZE
    d = torch.zeros(comp.size + 16, dtype=torch.uint8, device="cuda")
    d[1:1 + comp.size] = torch.from_numpy(comp).cuda()
    out = torch.empty(x.size, dtype=torch.uint8, device="cuda")
    assert ax.decode_status(d[1:1 + comp.size], out) == ax.ERR_ARG


def test_async_api_with_caller_workspace():
    x = synth.make("fastq", 2_000_000, 3)
    for kw in (dict(flatten=2), dict(depth_cap=4)):
        comp = oracle.encode(x, **kw)
        info = ax.peek_header(comp[:64])
        ws = torch.zeros(ax.workspace_size(info), dtype=torch.uint8, device="cuda")
        st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        d = to_dev(comp)
        out = torch.empty(x.size, dtype=torch.uint8, device="cuda")
        for _ in range(2):  # the workspace is reused without clearing
            out.fill_(0)
            ax.decode_async(d, out, info, ws, st)
            torch.cuda.synchronize()
            assert int(st.item()) == 0
            assert np.array_equal(out.cpu().numpy(), x)
        small = torch.zeros(16, dtype=torch.uint8, device="cuda")
        with pytest.raises(ax.AceapexError) as e:
            ax.decode_async(d, out, info, small, st)
        assert e.value.code == ax.ERR_NOMEM


def test_batch_decode_and_graph_replay():
    mix = [("text", 300_000), ("fastq", 250_000), ("random", 70_000), ("rle7", 123_457), ("text", 5),
           ("markov", 1_100_000), ("fastq", 0), ("text", 40_000)]
    xs, comps = [], []
    for i, (k, n) in enumerate(mix):
        x = synth.make(k, n, 500 + i)
        xs.append(x)
        comps.append(oracle.encode(x, flatten=2 if i % 3 else 0, block_log2=16 if i % 2 else 20))
    d_comps = [to_dev(c) for c in comps]
    outs = [torch.zeros(x.size, dtype=torch.uint8, device="cuda") for x in xs]
    st = ax.decode_batch(d_comps, outs)
    assert np.all(st == 0), st
    for x, o in zip(xs, outs):
        assert np.array_equal(o.cpu().numpy(), x)
    plan = ax.BatchPlan(d_comps, outs)
    for rep in range(3):
        for o in outs:
            o.fill_(rep + 1)
        plan.launch(graph=True)
        assert np.all(plan.statuses() == 0)
        for x, o in zip(xs, outs):
            assert np.array_equal(o.cpu().numpy(), x)
    plan.close()


def test_batch_reports_per_stream_errors():
    xs = [synth.make("text", 20_000, i) for i in range(3)]
    comps = [oracle.encode(x, flatten=2) for x in xs]
    comps[1] = _mut(comps[1], 0, 4, 0)
    outs = [torch.zeros(x.size, dtype=torch.uint8, device="cuda") for x in xs]
    st = ax.decode_batch([to_dev(c) for c in comps], outs)
    assert st[0] == 0 and st[2] == 0 and st[1] == ax.ERR_FORMAT
    assert np.array_equal(outs[0].cpu().numpy(), xs[0]) and np.array_equal(outs[2].cpu().numpy(), xs[2])


def test_batch_plan_device_statuses_match_host_statuses():
    """The device-status form of a batch: one-pass, wavefront and malformed streams in one plan; the statuses
    gathered on the device equal the host ones and the oracle's codes."""
    xs = [synth.make("text", 30_000 + 7 * i, 50 + i) for i in range(5)]
    comps = [oracle.encode(xs[0], flatten=2), oracle.encode(xs[1]), oracle.encode(xs[2], flatten=2),
             oracle.encode(xs[3]), oracle.encode(xs[4], flatten=2)]
    comps[2] = _mut(comps[2], 0, 4, 0)                       # bad magic: found on the host
    b0 = int.from_bytes(bytes(comps[4][64:72]), "little")
    comps[4] = _mut(comps[4], b0 + 32 + 20 + 4, 1, 77)        # a sync entry: found by the one-pass kernel
    outs = [torch.zeros(x.size, dtype=torch.uint8, device="cuda") for x in xs]
    plan = ax.BatchPlan([to_dev(c) for c in comps], outs)
    try:
        plan.launch()
        d_st = torch.full((5,), 123, dtype=torch.int32, device="cuda")
        plan.statuses_device(d_st)
        host = plan.statuses()
        assert np.array_equal(d_st.cpu().numpy(), host)
        want = [oracle.decode_rc(c, x.size)[0] for c, x in zip(comps, xs)]
        assert list(host) == want and want[2] != 0 and want[4] != 0 and want[0] == want[1] == want[3] == 0
    finally:
        plan.close()


def test_bounded_wait_times_out_and_context_survives():
    """A tile whose flag is withheld makes every later tile's wait run out: the call returns
    ERR_TIMEOUT (no fault, no hang) and the next decode on the same context succeeds."""
    x = synth.make("text", 200_000, 12)
    comp = oracle.encode(x, block_log2=14, tile_log2=10, flatten=2)
    ax.set_wait_limit(20_000_000, withhold_tile=0)
    try:
        rc, _ = gpu_decode(comp, x.size)
    finally:
        ax.set_wait_limit(0)
    assert rc == ax.ERR_TIMEOUT
    check(x, comp, "auto")


@pytest.mark.parametrize("cfg", [(2, 0), (2, 3), (4, 2), (4, 4), (8, 0), (8, 1)])
def test_launch_shapes(cfg):
    x = synth.make("fastq", 1_500_000, 5)
    comp = oracle.encode(x, flatten=2, min_emit=6)
    ax.set_launch_config(*cfg)
    try:
        assert ax.get_launch_config() == cfg
        check(x, comp, "auto")
    finally:
        ax.set_launch_config(4, 0)
