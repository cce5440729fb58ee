"""Pins for the FP64 oracle: results the paper or the mathematics fix.

Each test checks the oracle against something other than itself: brute-force
bitwise MAP on cycle-free graphs (where BP is exact), closed forms (single
check, repetition chain, phi identities), exhaustive ML, exact symmetries,
the noiseless limit, and the figures printed in the paper's Table 1.
"""
import json
import os

import numpy as np
import pytest

import oracle
from synthetic import (bob_syndrome, make_workload, preset_graph, random_bits,
                       awgn_capacity, sigma_for_beta)
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# phi(x) = -ln tanh(x/2)
# --------------------------------------------------------------------------

def test_phi_closed_forms():
    # tanh(ln(3)/2) = (3-1)/(3+1) = 1/2, so phi(ln 3) = ln 2
    assert oracle.phi(np.log(3.0)) == pytest.approx(np.log(2.0), rel=1e-15)
    # large x: phi(x) = 2 atanh(e^-x) = 2 e^-x (1 + e^-2x/3 + ...)
    for x in (12.0, 20.0, 25.0):
        e = np.exp(-x)
        assert oracle.phi(x) == pytest.approx(2 * e * (1 + e * e / 3), rel=1e-13)
    # small x: tanh(x/2) = (x/2)(1 - x^2/12 + ...), phi = -ln(x/2) + x^2/12 + O(x^4)
    for x in (1e-3, 1e-6, 2.7e-11):
        assert oracle.phi(x) == pytest.approx(-np.log(x / 2) + x * x / 12, rel=1e-12)


def test_phi_is_an_involution_on_clamp_interval():
    lo = oracle.phi(oracle.LMAX)
    xs = np.exp(np.linspace(np.log(lo), np.log(oracle.LMAX), 401))
    back = np.array([oracle.phi(oracle.phi(x)) for x in xs])
    interior = (xs > 1e-9) & (xs < 20)
    assert np.allclose(back[interior], xs[interior], rtol=1e-12, atol=0)
    # phi maps [phi(25), 25] onto itself
    assert oracle.phi(lo) == pytest.approx(oracle.LMAX, rel=1e-12)


# --------------------------------------------------------------------------
# Exactness of BP on cycle-free graphs
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_tree_codes_match_bitwise_map(seed):
    rng = np.random.default_rng(100 + seed)
    g = brute.random_tree_code(rng, int(rng.integers(5, 15)))
    H = brute.parity_matrix(g)
    x = rng.integers(0, 2, g.n_vn).astype(np.uint8)
    s = (H.astype(np.int64) @ x) % 2
    llr = (1 - 2.0 * x) * 0.8 + rng.normal(0, 1.2, g.n_vn)
    out = oracle.decode(g, llr[None], s[None].astype(np.uint8), iters=2 * g.n_vn + 2)
    ref = brute.map_llr(H, s, llr)
    np.testing.assert_allclose(out["post"][0], ref, rtol=1e-9, atol=1e-9)
    assert np.array_equal(out["bits"][0], (ref < 0).astype(np.uint8))


@pytest.mark.parametrize("d,s", [(2, 0), (3, 1), (5, 0), (8, 1)])
def test_single_check_tanh_rule(d, s):
    rng = np.random.default_rng(d * 10 + s)
    g = brute.graph_from_edges(d, 1, [(v, 0) for v in range(d)])
    llr = rng.normal(0.5, 1.5, d)
    out = oracle.decode(g, llr[None], np.array([[s]], np.uint8), iters=1)
    for v in range(d):
        others = np.delete(llr, v)
        expect = llr[v] + brute.tanh_rule(others, s)
        assert out["post"][0, v] == pytest.approx(expect, rel=1e-12, abs=1e-12)


def test_repetition_chain_sums_with_syndrome_signs():
    rng = np.random.default_rng(7)
    n = 10
    g = brute.graph_from_edges(n, n - 1, [(i, i) for i in range(n - 1)] +
                               [(i + 1, i) for i in range(n - 1)])
    s = rng.integers(0, 2, n - 1).astype(np.uint8)
    llr = rng.uniform(-2, 2, n)
    out = oracle.decode(g, llr[None], s[None], iters=n + 1)
    sign = 1 - 2 * s.astype(np.float64)
    for v in range(n):
        tot = 0.0
        for u in range(n):
            lo, hi = min(u, v), max(u, v)
            tot += llr[u] * np.prod(sign[lo:hi])
        assert out["post"][0, v] == pytest.approx(tot, rel=1e-12, abs=1e-12)


# --------------------------------------------------------------------------
# Small loopy codes: exhaustive ML and invariants
# --------------------------------------------------------------------------

def test_ml_never_worse_than_bp_and_converged_words_satisfy_syndrome():
    rng = np.random.default_rng(11)
    n, m = 14, 7
    g = brute.random_code(rng, n, m, col_w=3)
    H = brute.parity_matrix(g)
    frames = 250
    x = rng.integers(0, 2, (frames, n)).astype(np.uint8)
    s = ((x.astype(np.int64) @ H.T) % 2).astype(np.uint8)
    sigma = 0.9
    y = (1 - 2.0 * x) + sigma * rng.standard_normal((frames, n))
    llr = 2 * y / sigma ** 2
    out = oracle.decode(g, llr, s, iters=30, early_term=True)
    bp_err = ml_err = 0
    for f in range(frames):
        ml = brute.ml_decode(H, s[f], llr[f])
        ml_err += int(not np.array_equal(ml, x[f]))
        bp_err += int(not np.array_equal(out["bits"][f], x[f]))
        synd_ok = np.array_equal((H.astype(np.int64) @ out["bits"][f]) % 2, s[f])
        assert bool(out["converged"][f]) == synd_ok
    assert ml_err <= bp_err
    assert bp_err > 0  # the case is hard enough to say something


def test_coset_symmetry_pins_syndrome_sign():
    g = preset_graph(0.1, 4096, 1)
    w = make_workload(0.1, 4096, 3, 1, 1000, beta=0.5, graph=g)
    L = oracle.channel_llr(w.y, w.sigma)
    for z in (w.x, random_bits(3, g.n_vn, 99)):
        Lz = L * (1 - 2.0 * z)
        sz = w.s ^ bob_syndrome(g, z)
        a = oracle.decode(g, L, w.s, iters=12)
        b = oracle.decode(g, Lz, sz, iters=12)
        assert np.array_equal(b["post"], a["post"] * (1 - 2.0 * z))
        nz = a["post"] != 0
        assert np.array_equal(b["bits"][nz], (a["bits"] ^ z)[nz])
    # dropping the syndrome would break the symmetry: decoding with s = 0
    # instead of the true syndrome gives a different answer
    c = oracle.decode(g, L, np.zeros_like(w.s), iters=12)
    assert not np.array_equal(c["post"], a["post"])


def test_noiseless_limit_decodes_in_one_iteration():
    g = preset_graph(0.1, 4096, 1)
    w = make_workload(0.1, 4096, 2, 1, 2000, sigma=0.1, graph=g)
    out = oracle.decode_y(g, w.y, w.sigma, w.s, iters=5, early_term=True)
    assert np.array_equal(out["bits"], w.x)
    assert out["converged"].tolist() == [1, 1]
    assert out["iters_used"].tolist() == [1, 1]


def test_early_termination_equals_fixed_run_to_first_match():
    g = preset_graph(0.1, 4096, 1)
    w = make_workload(0.1, 4096, 4, 1, 3000, beta=0.3, graph=g)
    L = oracle.channel_llr(w.y, w.sigma)
    et = oracle.decode(g, L, w.s, iters=60, early_term=True)
    assert et["converged"].all()
    for b in range(4):
        lb = int(et["iters_used"][b])
        fixed = oracle.decode(g, L[b:b + 1], w.s[b:b + 1], iters=lb)
        assert np.array_equal(fixed["bits"][0], et["bits"][b])
        assert np.array_equal(fixed["post"][0], et["post"][b])
        if lb > 1:
            before = oracle.decode(g, L[b:b + 1], w.s[b:b + 1], iters=lb - 1)
            assert before["converged"][0] == 0


def test_zero_iterations_is_channel_decision():
    g = preset_graph(0.1, 4096, 1)
    w = make_workload(0.1, 4096, 2, 1, 4000, graph=g)
    L = oracle.channel_llr(w.y, w.sigma)
    out = oracle.decode(g, L, w.s, iters=0, early_term=True)
    np.testing.assert_array_equal(out["post"], np.clip(L, -25, 25))
    assert out["iters_used"].tolist() == [0, 0]


# --------------------------------------------------------------------------
# Figures printed in the paper (Table 1)
# --------------------------------------------------------------------------

def _table1():
    with open(os.path.join(GOLDEN, "table1_paper.json")) as f:
        return json.load(f)


def test_table1_accounting_identities():
    t = _table1()
    n = t["block_length"]
    for i, R in enumerate(t["rates"]):
        assert t["updated_cns"][i] == round(n * (1 - R))
        assert t["updated_vns_with_skip"][i] + t["ignored_vns_with_skip"][i] == n
        assert t["edges_passed_with_skip"][i] == t["total_edges"][i] - t["ignored_vns_with_skip"][i]


def test_table1_speed_is_block_length_over_iteration_latency():
    t = _table1()
    n = t["block_length"]
    for key_lat, key_spd in (("latency_ms_per_iteration_skip", "speed_mbit_s_skip"),
                             ("latency_ms_per_iteration_no_skip", "speed_mbit_s_no_skip")):
        for i, it in enumerate(t["iterations"]):
            lat = t[key_lat][i]
            lo = n / (it * (lat + 0.0005) * 1e-3) / 1e6
            hi = n / (it * (lat - 0.0005) * 1e-3) / 1e6
            assert lo - 0.01 <= t[key_spd][i] <= hi + 0.01


def test_table1_beta_follows_gaussian_capacity():
    t = _table1()
    for i, R in enumerate(t["rates"]):
        snr = t["snr"][i]
        lo = R / awgn_capacity(snr + 0.0005) * 100
        hi = R / awgn_capacity(snr - 0.0005) * 100
        assert lo - 0.01 <= t["beta_percent"][i] <= hi + 0.01
        # and the solver inverts it: sigma for that beta gives the SNR back
        sig = sigma_for_beta(R, t["beta_percent"][i] / 100, capacity="awgn")
        assert 1 / sig ** 2 == pytest.approx(snr, abs=0.0006)
