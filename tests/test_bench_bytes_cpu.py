"""The roofline accounting of bench.py: bytes per codeword of one whole
iteration at message width, for the three rates at n = 10^6, against the
figures derived independently in the build's scope table (2 b e_core + b m2
+ n_core (b + 8) + m/8: 21.79 / 41.87 MB at rate 0.1, 14.89 / 28.69 MB at
0.05, 10.91 / 21.21 MB at 0.02, half / float messages), and the check
pass's share of them."""
import pytest

import bench

N = 1_000_000
SPEC = {0.1: (0.20, 20), 0.05: (0.12, 22), 0.02: (0.06, 32)}
EXPECT_MB = {(0.1, "f16"): 21.79, (0.1, "f32"): 41.87, (0.05, "f16"): 14.89, (0.05, "f32"): 28.69,
             (0.02, "f16"): 10.91, (0.02, "f32"): 21.21}


def _stats(rate):
    core_frac, d2 = SPEC[rate]
    n_c = round(core_frac * N)
    n_two = round(0.4 * n_c)
    e_core = 2 * n_two + 3 * (n_c - n_two) + d2 * n_c
    m2 = N - n_c
    m1 = n_c - round(rate * N)
    return {"e_core": e_core, "n_deg1": m2, "n_core": n_c, "n_cn": m1 + m2}


@pytest.mark.parametrize("rate", [0.1, 0.05, 0.02])
@pytest.mark.parametrize("msg", ["f16", "f32"])
def test_iteration_bytes_match_the_scope_table(rate, msg):
    check, iteration = bench.algorithmic_bytes(_stats(rate), msg)
    assert iteration / 1e6 == pytest.approx(EXPECT_MB[(rate, msg)], abs=0.006)
    # the check pass reads the posteriors once and writes none: 4 n_core
    # instead of (b + 8) n_core, the rest identical
    b = 2 if msg == "f16" else 4
    st = _stats(rate)
    assert iteration - check == pytest.approx(st["n_core"] * (b + 8 - 4))


def test_check_pass_bytes_of_the_headline():
    check, _ = bench.algorithmic_bytes(_stats(0.1), "f16")
    assert check / 1e6 == pytest.approx(20.59, abs=0.006)   # 1.318 GB per pass at 64 codewords


def test_layered_iteration_bytes():
    """Layered: per core edge r in and out plus the VN's posterior read and
    written in that edge's layer (2 b + 8 bytes); at rate 0.1, n = 10^6,
    half messages: 4.52e6 x 12 + 2 x 8e5 + 9e5 / 8 = 55.95 MB."""
    st = _stats(0.1)
    assert st["e_core"] == 4_520_000
    check, iteration = bench.algorithmic_bytes(st, "f16", "layered")
    assert check == iteration
    assert iteration / 1e6 == pytest.approx(55.95, abs=0.006)
    _, it32 = bench.algorithmic_bytes(st, "f32", "layered")
    assert it32 - iteration == pytest.approx(4 * st["e_core"] + 2 * st["n_deg1"])
