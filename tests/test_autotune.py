"""The launch-shape autotuner's selection and cache, on CPU with a fake timer (no GPU, no library calls)."""
from paper_2606_04268_gb300 import autotune


def test_picks_fastest_applies_it_and_caches(tmp_path):
    cache = str(tmp_path / "tune.json")
    applied = []
    cands = [(3, 256, 0, 4), (0, 256, 0, 4), (4, 256, 2, 4)]
    ms = {cands[0]: 2.0, cands[1]: 3.0, cands[2]: 1.5}
    best, times = autotune.tune(None, "sig-a", cache_path=cache, candidates=cands, timer=lambda c: ms[c],
                                device_key="dev", apply_fn=applied.append)
    assert best == cands[2] and applied[-1] == cands[2]
    assert times == ms
    # second call: from the cache, no timing
    applied.clear()
    best2, _ = autotune.tune(None, "sig-a", cache_path=cache, candidates=cands,
                             timer=lambda c: (_ for _ in ()).throw(AssertionError("timed again")),
                             device_key="dev", apply_fn=applied.append)
    assert best2 == cands[2] and applied == [cands[2]]
    # another signature or device tunes again
    best3, _ = autotune.tune(None, "sig-b", cache_path=cache, candidates=cands[:2], timer=lambda c: ms[c],
                             device_key="dev", apply_fn=applied.append)
    assert best3 == cands[0]


def test_corrupt_cache_is_ignored(tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text("{not json")
    best, _ = autotune.tune(None, "s", cache_path=str(cache), candidates=[(3, 256, 0, 4)], timer=lambda c: 1.0,
                            device_key="dev", apply_fn=lambda c: None)
    assert best == (3, 256, 0, 4)


def test_default_candidates_are_valid_launch_shapes():
    ok_shapes = {(128, 4), (128, 8), (256, 2), (256, 4), (256, 8), (512, 2), (512, 4)}
    for kernel, threads, ctas, spt in autotune.CANDIDATES:
        assert kernel in (0, 3, 4) and ctas >= 0 and (threads, spt) in ok_shapes
