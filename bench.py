"""Benchmark of the GB300 ACEAPEX decoder: one JSON line on rank 0.

A step is one complete decode of one stream (parse, prefix sum, literal scatter, match copies in depth
waves) of the workload, with the compressed stream already in HBM.  Default workload: 1 GiB of synthetic
English-like text encoded with full-depth, unflattened chains (the 1 GiB text configuration).  Other
workloads: --workload fastq-flat | fastq-cap4 (1 GiB FASTQ, chain-flattened / depth cap 4), small (4 MiB).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload text] [--impl ours|reference]

--impl reference times the CPU oracle decoder on the host cores on the same stream (rank 0 only).
Multi-GPU: N independent replicas (one stream per rank, no collective on the data path), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

MiB, GiB = 1 << 20, 1 << 30
WORKLOADS = {
    # name: (generator kind, size, encoder params, description)
    "text": ("text", GiB, dict(min_emit=6),
             "1 GiB synthetic English-like text (Zipf s=1.0, 200k words), full-depth unflattened chains"),
    "fastq-flat": ("fastq", GiB, dict(flatten=2, min_emit=6),
                   "1 GiB synthetic FASTQ (150-base reads, 64 x 1 Mb references, Q30 Gaussian qualities), "
                   "chain-flattened (global)"),
    "fastq-cap4": ("fastq", GiB, dict(depth_cap=4, min_emit=6), "1 GiB synthetic FASTQ, depth cap 4"),
    "small": ("markov", 4 * MiB, dict(min_match=4), "4 MiB Markov text, 4 blocks, min match 4, unflattened"),
}


def stream_stats(comp: np.ndarray):
    """Literal and match byte counts from the block headers (stream format §2.1)."""
    hdr = comp[:64].view(np.uint8)
    N = int(hdr[16:24].view(np.uint64)[0])
    nb = int(hdr[24:32].view(np.uint64)[0])
    n_match = int(hdr[40:48].view(np.uint64)[0])
    max_depth = int(hdr[48:52].view(np.uint32)[0])
    offs = comp[64:64 + 8 * nb].view(np.uint64).astype(np.int64)
    n_lit = int(sum(int(comp[o + 8:o + 12].view(np.uint32)[0]) for o in offs))
    return dict(N=N, C=int(comp.size), n_match=n_match, lit_bytes=n_lit, match_bytes=N - n_lit, max_depth=max_depth,
                n_blocks=nb)


def kernel_bytes(name: str, st: dict) -> float:
    """Algorithmic HBM bytes of one launch of each kernel (stream read once, output written once, each
    match-source byte read once, per-match metadata of the wavefront path at its stored width)."""
    C, N, M, L, nm = st["C"], st["N"], st["match_bytes"], st["lit_bytes"], st["n_match"]
    return {
        "k_flat": C + N + M,                          # stream, output, match sources
        "k_parse": C + L + 24 * nm + N / 16,          # stream, literals, 24 B records, granule index
        "k_depth": 40 * nm,                           # records + writer lookups + depth
        "k_wave": 2 * M + 24 * nm,                    # sources, destinations, queue + records
        "k_scatter": 8 * nm, "k_hist": 4 * nm,
    }.get(name, 0.0)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def make_stream(args, rank: int):
    import paper_2606_04268_gb300 as ax
    kind, n, enc, desc = WORKLOADS[args.workload]
    if args.size:
        n = args.size
    seed = {"text": 2000, "fastq": 3000, "markov": 1000}[kind] + rank
    x = synth.make(kind, n, seed)
    t0 = time.time()
    comp = ax.encode(x, **enc)
    return x, comp, desc, time.time() - t0


def cpu_oracle_baseline(comp: np.ndarray, N: int, min_seconds: float):
    """The oracle decoder as it stands, single-threaded, repeated on the workload's stream."""
    import oracle
    oracle.build()
    reps, t_total = 0, 0.0
    while t_total < min_seconds and reps < 50:
        t0 = time.perf_counter()
        rc, _ = oracle.decode_rc(comp, N)
        t_total += time.perf_counter() - t0
        reps += 1
        assert rc == 0
    return N * reps / t_total / 1e9, reps, t_total


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    x, comp, desc, _ = make_stream(args, 0)
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        rc, _ = oracle.decode_rc(comp, x.size)
        assert rc == 0
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        rc, out = oracle.decode_rc(comp, x.size)
        times.append(time.perf_counter() - t0)
        assert rc == 0
    assert np.array_equal(out, x)
    t = sum(times) / len(times)
    v = x.size / t / 1e9
    line = {"impl": "reference", "metric": "decoded GB/s", "value": round(v, 4), "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": desc, "decoded_bytes": int(x.size), "comp_bytes": int(comp.size)},
            "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"the whole workload stream ({x.size} decoded bytes) per step"},
            "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_2606_04268_gb300 as ax
    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    ax.build()
    x, comp, desc, enc_s = make_stream(args, rank)
    st = stream_stats(comp)
    info = ax.peek_header(comp[:64])
    d_comp = torch.from_numpy(comp).cuda()
    out = torch.empty(x.size, dtype=torch.uint8, device="cuda")
    ws = torch.zeros(ax.workspace_size(info), dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        ax.decode_async(d_comp, out, info, ws, status, stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    hbm_peak, peak_kind = peaks()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        assert int(status.item()) == 0, ax.STATUS_NAMES.get(int(status.item()))
        assert torch.equal(out, torch.from_numpy(x).cuda()), "decoded bytes differ from the input"
        # timed region: K decodes back to back (inputs and outputs exceed L2 several times)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / args.steps
        assert int(status.item()) == 0
        # the same K decodes with CUDA events around every library kernel: per-kernel launch durations
        ax.profile(True)
        for _ in range(args.steps):
            step()
        prof = ax.profile_read()
        ax.profile(False)
        # end to end through the blocking public call with host buffers: H2D of the stream, decode,
        # D2H of the decoded bytes, every step
        h_comp = torch.from_numpy(comp).pin_memory()
        h_out = torch.empty(x.size, dtype=torch.uint8).pin_memory()
        d2 = torch.empty_like(d_comp)
        e2e_steps = max(1, min(args.steps, 10))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            d2.copy_(h_comp, non_blocking=True)
            ax.decode(d2, out, stream)
            h_out.copy_(out, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        assert torch.equal(h_out, torch.from_numpy(x))
    ms_all = torch.tensor([ms], device="cuda")
    if world > 1:
        torch.distributed.all_reduce(ms_all, op=torch.distributed.ReduceOp.MAX)
    ms = float(ms_all.item())
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    total_bytes = st["N"] * world
    value = total_bytes / (ms * 1e-3) / 1e9
    # dominant kernel of a step
    kern = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kern, key=lambda k: kern[k][0])
    dom_ms = kern[dom][0] / kern[dom][1]
    ach = kernel_bytes(dom, st) / (dom_ms * 1e-3) / 1e9
    decode_frac = (st["C"] + 2 * st["N"]) / (ms * 1e-3) / 1e9 / hbm_peak
    line = {
        "metric": "decoded GB/s", "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": desc, "decoded_bytes": st["N"], "comp_bytes": st["C"], "ratio": round(st["C"] / st["N"], 4),
                   "max_depth": st["max_depth"], "n_match": st["n_match"], "path": "one-pass" if st["max_depth"] <= 1 else "wavefront",
                   "parallelism": f"replicas x{world}", "l2": "inputs and outputs larger than L2 (no flush needed)",
                   "encode_s": round(enc_s, 1)},
        "decode_roofline_frac": round(decode_frac, 4),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(ach / hbm_peak, 4), "traffic": None, "peak_kind": peak_kind},
        "kernels_ms": {k: round(v[0] / v[1], 4) for k, v in kern.items()},
        "gpu_launches": int(sum(v[1] for v in kern.values()) // args.steps * args.steps),
        "e2e": {"value": round(st["N"] / e2e_s / 1e9, 3), "unit": "GB/s", "h2d_bytes_per_step": st["C"],
                "d2h_bytes_per_step": st["N"]},
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_cpu:
        v, reps, secs = cpu_oracle_baseline(comp, st["N"], args.cpu_seconds)
        line["cpu_baseline"] = {"value": round(v, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                                "sample": f"the workload's stream decoded {reps} times ({secs:.1f} s)"}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="text", choices=list(WORKLOADS))
    ap.add_argument("--size", type=int, default=0, help="override the workload size (bytes)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
