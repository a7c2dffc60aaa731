"""The launch-shape autotuner's selection and cache, on CPU with a fake timer (no GPU, no library calls)."""
import pytest

from paper_2606_04268_gb300 import autotune


def test_picks_fastest_applies_it_and_caches(tmp_path):
    cache = str(tmp_path / "tune.json")
    applied = []
    cands = [(4, 0), (2, 0), (8, 2)]
    ms = {cands[0]: 2.0, cands[1]: 3.0, cands[2]: 1.5}
    best, times = autotune.tune(None, "sig-a", cache_path=cache, candidates=cands, timer=lambda c: ms[c],
                                device_key="dev", apply_fn=applied.append, current_fn=lambda: (4, 0))
    assert best == cands[2] and applied[-1] == cands[2]
    assert times == ms
    # second call: from the cache, no timing
    applied.clear()
    best2, _ = autotune.tune(None, "sig-a", cache_path=cache, candidates=cands,
                             timer=lambda c: (_ for _ in ()).throw(AssertionError("timed again")),
                             device_key="dev", apply_fn=applied.append, current_fn=lambda: (4, 0))
    assert best2 == cands[2] and applied == [cands[2]]
    # another signature or device tunes again
    best3, _ = autotune.tune(None, "sig-b", cache_path=cache, candidates=cands[:2], timer=lambda c: ms[c],
                             device_key="dev", apply_fn=applied.append, current_fn=lambda: (4, 0))
    assert best3 == cands[0]


def test_corrupt_cache_is_ignored(tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text("{not json")
    best, _ = autotune.tune(None, "s", cache_path=str(cache), candidates=[(4, 0)], timer=lambda c: 1.0,
                            device_key="dev", apply_fn=lambda c: None, current_fn=lambda: (4, 0))
    assert best == (4, 0)


def test_failed_timing_restores_the_previous_configuration(tmp_path):
    applied = []

    def timer(cfg):
        if cfg == (2, 0):
            raise RuntimeError("launch failed")
        return 1.0

    with pytest.raises(RuntimeError):
        autotune.tune(None, "s", cache_path=str(tmp_path / "t.json"), candidates=[(4, 0), (2, 0), (8, 0)],
                      timer=timer, device_key="dev", apply_fn=applied.append, current_fn=lambda: (8, 3))
    assert applied[-1] == (8, 3)


def test_default_candidates_are_valid_launch_shapes():
    for warps, ctas in autotune.CANDIDATES:
        assert warps in (2, 4, 8) and ctas >= 0
