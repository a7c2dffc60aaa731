"""The launch-shape autotuner on a real batch plan: it times its candidates on the GPU, and the shape it
picks decodes every stream of the batch byte-exactly (the decode is exact integer work)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_04268_gb300 as ax
import synth
from gpu_util import to_dev
from paper_2606_04268_gb300 import autotune

pytestmark = pytest.mark.gpu


def test_tune_real_plan_and_decode_with_the_choice(tmp_path):
    ax.build()
    mix = [("text", 600_000), ("fastq", 500_000), ("random", 90_000), ("rle7", 300_001), ("markov", 1_000_000)]
    xs = [synth.make(k, n, 700 + i) for i, (k, n) in enumerate(mix)]
    comps = [oracle.encode(x, flatten=2, min_emit=6) for x in xs]
    d_comps = [to_dev(c) for c in comps]
    outs = [torch.zeros(x.size, dtype=torch.uint8, device="cuda") for x in xs]
    plan = ax.BatchPlan(d_comps, outs)
    before = ax.get_launch_config()
    try:
        best, times = autotune.tune(plan, "small-mix", reps=2, cache_path=str(tmp_path / "tune.json"), force=True)
        assert best in times and len(times) == len(autotune.CANDIDATES)
        assert all(t > 0 for t in times.values())
        assert ax.get_launch_config() == best
        for o in outs:
            o.fill_(0xA5)
        plan.launch(graph=False)
        assert np.all(plan.statuses() == 0)
        for x, o in zip(xs, outs):
            assert np.array_equal(o.cpu().numpy(), x)
    finally:
        plan.close()
        ax.set_launch_config(*before)
