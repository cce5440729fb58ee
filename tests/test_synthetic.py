"""Checks of the seeded input generators (ensemble graph and channel)."""
import numpy as np
import pytest
from scipy import integrate

from synthetic import (biawgn_capacity, awgn_capacity, sigma_for_beta,
                       met_ensemble, preset_graph, make_workload, bob_syndrome,
                       RATE_PRESETS)
from synthetic.ensemble import EDGE_T1, EDGE_T2, EDGE_T2_DEG1


@pytest.mark.parametrize("rate", [0.1, 0.05, 0.02])
def test_ensemble_degree_structure(rate):
    n = 20000
    g = preset_graph(rate, n, 5)
    p = RATE_PRESETS[rate]
    n_c = int(round(p["core_frac"] * n))
    m2 = n - n_c
    m1 = n_c - int(round(rate * n))
    assert (g.n_core, g.m1, g.m2, g.n_cn) == (n_c, m1, m2, m1 + m2)
    assert g.n_cn == n - int(round(rate * n))
    vd = g.vn_degree()
    assert (vd == 1).sum() == m2
    n_two = int(round(0.4 * n_c))
    assert (vd == 2 + p["d2"]).sum() == n_two
    assert (vd == 3 + p["d2"]).sum() == n_c - n_two
    e1 = 2 * n_two + 3 * (n_c - n_two)
    assert (g.edge_type == EDGE_T1).sum() == e1
    assert (g.edge_type == EDGE_T2).sum() == p["d2"] * n_c
    assert (g.edge_type == EDGE_T2_DEG1).sum() == m2
    # no repeated (VN, check) pair
    key = g.edge_vn.astype(np.int64) * g.n_cn + g.edge_cn
    assert np.unique(key).size == key.size
    # every degree-1 VN sits on a check that has exactly one degree-1 VN
    d1_checks = g.edge_cn[g.edge_type == EDGE_T2_DEG1]
    assert np.unique(d1_checks).size == m2
    # check-side sockets dealt evenly per type
    for t, m_t in ((EDGE_T1, m1), (EDGE_T2, m2)):
        cd = np.bincount(g.edge_cn[g.edge_type == t], minlength=g.n_cn)
        cd = cd[cd > 0]
        assert cd.size == m_t and cd.max() - cd.min() <= 1


def test_ensemble_is_deterministic_and_seed_dependent():
    a = preset_graph(0.1, 4096, 1)
    b = preset_graph(0.1, 4096, 1)
    c = preset_graph(0.1, 4096, 2)
    assert np.array_equal(a.edge_vn, b.edge_vn) and np.array_equal(a.edge_cn, b.edge_cn)
    assert not np.array_equal(a.edge_vn, c.edge_vn)


def test_full_size_edge_counts_scale_linearly():
    # edge totals per 10^5 bits (x10 gives the n = 10^6 figures)
    for rate, total, core in ((0.1, 532000, 452000), (0.05, 383200, 295200), (0.02, 301600, 207600)):
        p = RATE_PRESETS[rate]
        g = met_ensemble(100000, rate, p["core_frac"], p["d2"], 3)
        assert g.n_edges == total
        assert int((g.vn_degree()[g.edge_vn] > 1).sum()) == core


def test_biawgn_capacity_against_direct_integration():
    for sigma in (0.5, 1.0, 2.45, 5.65):
        f = lambda y: (np.exp(-(y - 1) ** 2 / (2 * sigma ** 2)) / np.sqrt(2 * np.pi * sigma ** 2)
                       * np.logaddexp(0, -2 * y / sigma ** 2) / np.log(2))
        val, _ = integrate.quad(f, 1 - 40 * sigma, 1 + 40 * sigma, limit=400)
        assert biawgn_capacity(sigma) == pytest.approx(1 - val, abs=1e-9)
        assert biawgn_capacity(sigma) <= awgn_capacity(1 / sigma ** 2) + 1e-12


@pytest.mark.parametrize("rate", [0.1, 0.05, 0.02])
def test_sigma_for_beta_inverts_capacity(rate):
    s = sigma_for_beta(rate, 0.9)
    assert rate / biawgn_capacity(s) == pytest.approx(0.9, rel=1e-9)


def test_syndrome_and_observation_shapes_and_seeding():
    g = preset_graph(0.1, 4096, 1)
    w = make_workload(0.1, 4096, 3, 1, 1000, graph=g)
    H = np.zeros((g.n_cn, g.n_vn), np.int64)
    H[g.edge_cn, g.edge_vn] = 1
    assert np.array_equal(w.s, ((w.x.astype(np.int64) @ H.T) % 2).astype(np.uint8))
    assert np.array_equal(bob_syndrome(g, w.x[1:2])[0], w.s[1])
    w2 = make_workload(0.1, 4096, 2, 1, 1000, graph=g)
    assert np.array_equal(w2.x, w.x[:2]) and np.array_equal(w2.y, w.y[:2])
    assert w.y.dtype == np.float32 and abs(np.std(w.y + (2.0 * w.x - 1)) - w.sigma[0]) < 0.05


@pytest.mark.parametrize("rate", [0.1, 0.05, 0.02])
def test_layer_structured_ensemble(rate):
    """Same degree structure as the plain ensemble; its check groups are
    VN-disjoint layers, d2 + 3 of them."""
    from synthetic import preset_graph_layered
    n = 20000
    g = preset_graph_layered(rate, n, 5)
    ref = preset_graph(rate, n, 5)
    assert (g.n_vn, g.n_cn, g.n_edges, g.m1, g.m2) == (ref.n_vn, ref.n_cn, ref.n_edges, ref.m1, ref.m2)
    np.testing.assert_array_equal(np.bincount(g.vn_degree()), np.bincount(ref.vn_degree()))
    for t in (EDGE_T1, EDGE_T2, EDGE_T2_DEG1):
        assert (g.edge_type == t).sum() == (ref.edge_type == t).sum()
    key = g.edge_vn.astype(np.int64) * g.n_cn + g.edge_cn
    assert np.unique(key).size == key.size
    lay = g.meta["layer_of_check"]
    assert lay.shape == (g.n_cn,) and g.meta["n_layers"] == RATE_PRESETS[rate]["d2"] + 3
    assert np.array_equal(np.unique(lay), np.arange(g.meta["n_layers"]))
    core = g.vn_degree()[g.edge_vn] > 1
    pair = lay[g.edge_cn[core]].astype(np.int64) * g.n_vn + g.edge_vn[core]
    assert np.unique(pair).size == pair.size       # no core VN twice in a layer
    # check degrees within one type differ by at most one
    for t in (EDGE_T1, EDGE_T2):
        cd = np.bincount(g.edge_cn[g.edge_type == t], minlength=g.n_cn)
        cd = cd[cd > 0]
        assert cd.max() - cd.min() <= 1
