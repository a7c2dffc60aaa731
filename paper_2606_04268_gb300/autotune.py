"""Launch-shape autotuner for batched decodes.

The tunable knobs of the one-pass path are:
- the kernel variant: one warp per tile reading the compressed sections from global memory, or one warp
  per tile with the sections staged in shared memory by bulk copies, at 32 or 128 sequences per warp step;
- the number of CTAs per SM (occupancy cap of the persistent grid);
- for streams whose tiles exceed 4 KiB, the CTA shape of the CTA-per-tile kernel: threads per CTA and
  sequences per thread per parse chunk.

The tuner times every candidate on the caller's plan (CUDA events, plain launches) and keeps the
fastest. Results are cached in a JSON file keyed by the device and a signature of the batch, so a serving
process tunes once per batch shape.
"""
from __future__ import annotations

import json
import os

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")

# (one-pass kernel variant, threads, ctas per SM, sequences per thread)
CANDIDATES = [(k, t, c, s) for k in (3, 4, 0) for c in (0, 4, 3, 2) for (t, s) in ((256, 4),)] + \
             [(3, t, 0, s) for (t, s) in ((128, 4), (256, 2), (256, 8), (512, 2))]


def apply(cfg) -> None:
    """Make `cfg` the launch configuration of later launches on this context."""
    from . import set_launch_config, set_one_pass_kernel
    kernel, threads, ctas, spt = cfg
    set_one_pass_kernel(kernel)
    set_launch_config(threads, ctas, spt)


def _device_key() -> str:
    import torch
    dev = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{dev.name}|{dev.multi_processor_count}"


def _event_timer(plan, reps: int):
    """ms per launch of `plan` under the current configuration, CUDA events on the current stream."""
    import torch
    stream = torch.cuda.current_stream()

    def timer(cfg) -> float:
        plan.launch(stream=stream)  # warm-up (first use of the shape)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.launch(stream=stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps
    return timer


def tune(plan, signature: str, reps: int = 3, cache_path: str = DEFAULT_CACHE, candidates=None,
         force: bool = False, timer=None, device_key: str | None = None, apply_fn=apply):
    """Pick the fastest launch configuration for `plan`; applies it and returns (cfg, {cfg: ms}).

    timer(cfg) -> ms and device_key replace the CUDA-event timing and the device lookup (tests)."""
    key = f"{device_key or _device_key()}|{signature}"
    cache = {}
    if os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if not force and key in cache:
        cfg = tuple(cache[key]["cfg"])
        apply_fn(cfg)
        return cfg, {tuple(k): v for k, v in cache[key].get("ms", [])}
    timer = timer or _event_timer(plan, reps)
    times = {}
    for cfg in candidates or CANDIDATES:
        apply_fn(cfg)
        times[tuple(cfg)] = float(timer(tuple(cfg)))
    best = min(times, key=times.get)
    apply_fn(best)
    cache[key] = {"cfg": list(best), "ms": [[list(k), v] for k, v in times.items()]}
    try:
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    except OSError:
        pass
    return best, times
