"""The pre-scan choice between a CPU and a GPU decode (paper §8: size and depth decide), on CPU: the
estimates are the stated model, large shallow streams go to the GPU, small or very deep ones to a fast
CPU, and the copy over the host link counts against the GPU.  No GPU call."""
import pytest

import paper_2606_04268_gb300 as ax


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ax.build()
    ax.lib()


def info(N, depth, tile_log2=12, comp_ratio=0.5):
    i = ax.Info()
    i.decoded_len, i.comp_len, i.max_depth, i.tile_log2, i.block_log2 = N, int(N * comp_ratio), depth, tile_log2, 20
    return i


def test_estimates_follow_the_model():
    which, tc, tg = ax.choose_device(info(1 << 30, 1), cpu_gbps=10.0)
    assert tc == pytest.approx((1 << 30) / 10e9)
    assert tg == pytest.approx(30e-6 + (1 << 30) / 260e9)
    assert which == "gpu"
    _, _, tg2 = ax.choose_device(info(1 << 30, 100), cpu_gbps=10.0)
    assert tg2 == pytest.approx(30e-6 + (1 << 30) / 200e9 + 100 * 16.5e-6)
    _, _, tg3 = ax.choose_device(info(1 << 30, 1, tile_log2=14), cpu_gbps=10.0, gpu_wave_gbps=50.0, gpu_level_us=10.0)
    assert tg3 == pytest.approx(30e-6 + (1 << 30) / 50e9 + 1 * 10e-6)  # tiles over 4 KiB: wavefront path


def test_size_depth_and_link_decide():
    assert ax.choose_device(info(4096, 1), cpu_gbps=10.0)[0] == "cpu"            # fixed GPU overhead dominates
    assert ax.choose_device(info(256 << 20, 1), cpu_gbps=10.0)[0] == "gpu"
    assert ax.choose_device(info(64 << 20, 5000), cpu_gbps=10.0)[0] == "cpu"     # 5000 levels: sequential depth
    assert ax.choose_device(info(64 << 20, 5000), cpu_gbps=0.5)[0] == "gpu"      # ... unless the CPU is slow
    dev, _, tg_dev = ax.choose_device(info(1 << 30, 1), cpu_gbps=10.0)
    host, _, tg_host = ax.choose_device(info(1 << 30, 1), cpu_gbps=10.0, link_gbps=50.0)
    assert tg_host == pytest.approx(tg_dev + (0.5 * (1 << 30) + (1 << 30)) / 50e9)
    assert ax.choose_device(info(1 << 30, 1), cpu_gbps=40.0, link_gbps=20.0)[0] == "cpu"   # the link is the limit


def test_monotone_in_depth_and_size():
    prev = None
    for depth in (2, 10, 100, 1000, 10000):
        _, _, tg = ax.choose_device(info(1 << 30, depth), cpu_gbps=10.0)
        assert prev is None or tg > prev
        prev = tg
    for n in (1 << 20, 1 << 24, 1 << 28):
        which_small = ax.choose_device(info(n, 1), cpu_gbps=10.0)[0]
        if which_small == "gpu":
            assert ax.choose_device(info(n * 4, 1), cpu_gbps=10.0)[0] == "gpu"


def test_bad_arguments():
    with pytest.raises(ax.AceapexError):
        ax.choose_device(info(1 << 20, 1), cpu_gbps=0.0)
