"""Launch-shape autotuner for batched decodes.

The tunable knobs of the one-pass path are the CTA shape of the persistent grid -- warps per CTA (2, 4 or
8; each warp decodes one tile at a time, 32 sequences per step) -- and the number of CTAs per SM (the
occupancy cap).  The chunk width, the tile of the stream format, is fixed by the encoder.

The tuner times every candidate on the caller's plan (CUDA events, plain launches) and keeps the fastest.
Results are cached in a JSON file keyed by the device and a signature of the batch, so a serving process
tunes once per batch shape.  The configuration that was in force before is restored if timing fails.
"""
from __future__ import annotations

import json
import os

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")

# (warps per CTA, CTAs per SM); 0 = as many CTAs as fit
CANDIDATES = [(w, c) for w in (4, 2, 8) for c in (0, 4, 3, 2)]


def apply(cfg) -> None:
    """Make `cfg` the launch configuration of later launches on this context."""
    from . import set_launch_config
    warps, ctas = cfg
    set_launch_config(warps, ctas)


def current():
    from . import get_launch_config
    return tuple(get_launch_config())


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
         force: bool = False, timer=None, device_key: str | None = None, apply_fn=apply, current_fn=current):
    """Pick the fastest launch configuration for `plan`; applies it and returns (cfg, {cfg: ms}).

    timer(cfg) -> ms, device_key, apply_fn and current_fn replace the CUDA-event timing, the device lookup
    and the library calls (tests)."""
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
    before = current_fn() if current_fn else None
    try:
        for cfg in candidates or CANDIDATES:
            apply_fn(cfg)
            times[tuple(cfg)] = float(timer(tuple(cfg)))
    except BaseException:
        if before is not None:
            apply_fn(before)
        raise
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
