"""Parity of the CUDA decoder (through the C ABI) against the FP64 oracle.

Tolerances (derived from the arithmetic):
* phi: float evaluation of the two polynomial pieces on top of MUFU lg2/ex2
  (relative error about 2^-22 each) -- relative error below 2e-6 on
  [phi(25), 25].
* One iteration, float messages: each check output carries a few float
  roundings through phi and the prefix/suffix sums; a posterior sums up to
  d_v of them.  Bound used: |dL| <= 1e-4 + 1e-5 |L|.
* One iteration, half messages: each stored message is rounded to half
  (relative error <= 2^-11, |r| <= 25), so |dL| <= 2^-11 * sum_e |r_e| +
  1e-4 <= 2^-11 * 25 * d_v + 1e-4.
* After N iterations: hard decisions agree on >= 99.99 % of bits, converged
  flags and iteration counts identical, and every converged word satisfies
  H x = s exactly.
"""
import numpy as np
import pytest

import oracle
from synthetic import make_workload, preset_graph
from tests import brute

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mld():
    import paper_1711_01783_gb300 as m
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _np(t):
    return t.cpu().numpy() if t is not None else None


def _llr32(w):
    return (2.0 * w.y.astype(np.float64) / (w.sigma.astype(np.float64)[:, None] ** 2)).astype(np.float32)


def _syndrome_holds(g, bits, s):
    H_ev, H_ec = g.edge_vn.astype(np.int64), g.edge_cn.astype(np.int64)
    ok = []
    for b in range(bits.shape[0]):
        par = np.bincount(H_ec, weights=bits[b, H_ev].astype(np.float64), minlength=g.n_cn).astype(np.int64) & 1
        ok.append(np.array_equal(par.astype(np.uint8), s[b]))
    return np.array(ok)


def test_library_reports_version(mld):
    assert "sm_103a" in mld.version()


def test_phi_matches_closed_form(mld):
    lo = oracle.phi(25.0)
    x = np.exp(np.linspace(np.log(lo), np.log(25.0), 20001)).astype(np.float32)
    got = _np(mld.phi(_dev(x))).astype(np.float64)
    xd = x.astype(np.float64)
    ref = np.log1p(2.0 / np.expm1(xd))
    rel = np.abs(got - ref) / ref
    assert rel.max() < 2e-6, rel.max()


@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_one_iteration_llr_error(mld, msg):
    w = make_workload(0.1, 4096, 4, 1, 1000)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 4, msg_dtype=msg)
    L = _llr32(w)
    out = dec.decode(_dev(L), _dev(w.s), iters=1, want_post=True)
    ref = oracle.decode(w.graph, L, w.s, iters=1)
    d = np.abs(_np(out["post"]).astype(np.float64) - ref["post"])
    if msg == "f32":
        bound = 1e-4 + 1e-5 * np.abs(ref["post"])
    else:
        dv = w.graph.vn_degree()[None, :]
        bound = 2.0 ** -11 * 25.0 * dv + 1e-4
    assert np.all(d <= bound), (d.max(), (d - bound).max())
    print(f"{msg}: one-iteration |dL| max {d.max():.3g} mean {d.mean():.3g}")


@pytest.mark.parametrize("msg,beta,iters,et", [
    ("f32", 0.9, 50, False),     # the workload's own operating point: BP does not converge
    ("f32", 0.3, 50, True),      # converging regime with early termination
    ("f16", 0.9, 50, False),
    ("f16", 0.3, 50, True),
])
def test_decode_matches_oracle(mld, msg, beta, iters, et):
    w = make_workload(0.1, 4096, 4, 1, 1000, beta=beta)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 4, msg_dtype=msg)
    out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=iters, early_term=et, want_post=True)
    ref = oracle.decode_y(w.graph, w.y, w.sigma, w.s, iters=iters, early_term=et)
    bits = _np(out["bits"])
    agree = (bits == ref["bits"]).mean()
    assert agree >= 0.9999, agree
    assert np.array_equal(_np(out["converged"]), ref["converged"])
    assert np.array_equal(_np(out["iters_used"]), ref["iters_used"])
    conv = _np(out["converged"]).astype(bool)
    assert np.array_equal(_syndrome_holds(w.graph, bits, w.s), conv)


@pytest.mark.parametrize("B,W,msg", [(5, 32, "f32"), (37, 16, "f32"), (3, 8, "f16"), (70, 64, "f16")])
def test_ragged_batches_and_slab_widths(mld, B, W, msg):
    g0 = preset_graph(0.05, 3000, 4)
    w = make_workload(0.05, 3000, B, 4, 500, beta=0.35, graph=g0)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, B + 3, msg_dtype=msg, slab_width=W)
    out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=25, early_term=True, want_post=True)
    ref = oracle.decode_y(w.graph, w.y, w.sigma, w.s, iters=25, early_term=True)
    assert (_np(out["bits"]) == ref["bits"]).mean() >= 0.9999
    assert np.array_equal(_np(out["converged"]), ref["converged"])
    assert np.array_equal(_np(out["iters_used"]), ref["iters_used"])


def test_host_and_device_pointers_agree(mld):
    w = make_workload(0.1, 4096, 6, 1, 600, beta=0.4)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 8, msg_dtype="f16")
    a = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=20, want_post=True)
    b = dec.decode_y(w.y, w.sigma, w.s, iters=20, want_post=True)
    assert np.array_equal(_np(a["bits"]), b["bits"])
    assert np.array_equal(_np(a["post"]), b["post"])
    assert np.array_equal(_np(a["iters_used"]), b["iters_used"])


def test_llr_and_y_entry_points_agree(mld):
    w = make_workload(0.1, 4096, 4, 1, 700, beta=0.4)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 4)
    a = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=15, want_post=True)
    b = dec.decode(_dev(_llr32(w)), _dev(w.s), iters=15, want_post=True)
    assert (_np(a["bits"]) == _np(b["bits"])).mean() >= 0.9999
    assert np.abs(_np(a["post"]) - _np(b["post"])).max() < 1e-2


def test_zero_iterations_and_empty_batch(mld):
    w = make_workload(0.1, 4096, 3, 1, 800)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 4)
    L = _llr32(w)
    out = dec.decode(_dev(L), _dev(w.s), iters=0, early_term=True, want_post=True)
    ref = oracle.decode(w.graph, L, w.s, iters=0, early_term=True)
    assert np.array_equal(_np(out["bits"]), ref["bits"])
    np.testing.assert_array_equal(_np(out["post"]), np.clip(L, -25, 25))
    assert np.array_equal(_np(out["converged"]), ref["converged"])
    assert _np(out["iters_used"]).tolist() == [0, 0, 0]
    empty = dec.decode(_dev(L[:0]), _dev(w.s[:0]), iters=5)
    assert empty["bits"].shape == (0, g.n_vn)


@pytest.mark.parametrize("seed", range(6))
def test_tree_codes_against_oracle(mld, seed):
    rng = np.random.default_rng(300 + seed)
    t = brute.random_tree_code(rng, int(rng.integers(6, 15)))
    H = brute.parity_matrix(t)
    B = 8
    x = rng.integers(0, 2, (B, t.n_vn)).astype(np.uint8)
    s = ((x.astype(np.int64) @ H.T) % 2).astype(np.uint8)
    L = ((1 - 2.0 * x) * 0.8 + rng.normal(0, 1.2, x.shape)).astype(np.float32)
    g = mld.Graph(t.edge_vn, t.edge_cn, t.n_vn, t.n_cn)
    dec = mld.Decoder(g, B, slab_width=8)
    out = dec.decode(_dev(L), _dev(s), iters=2 * t.n_vn, want_post=True)
    for b in range(B):
        np.testing.assert_allclose(_np(out["post"])[b], brute.map_llr(H, s[b], L[b]), rtol=1e-4, atol=1e-4)


def test_irregular_graph_edge_cases(mld):
    """High-degree checks (register-spill path), degree-0 VNs, empty checks,
    checks with several degree-1 VNs."""
    rng = np.random.default_rng(9)
    n, m = 400, 60
    edges = set()
    for v in range(300):                       # core VNs, degree 3 into 40 checks -> check degree ~22
        for c in rng.choice(40, 3, replace=False):
            edges.add((v, int(c)))
    for v in range(300, 390):                  # degree-1 VNs, several per check on checks 40..54
        edges.add((v, 40 + (v % 15)))
    # VNs 390..399 have degree 0; checks 55..59 have no edges
    e = np.array(sorted(edges), dtype=np.int64)
    from types import SimpleNamespace
    gg = SimpleNamespace(n_vn=n, n_cn=m, edge_vn=e[:, 0].astype(np.int32), edge_cn=e[:, 1].astype(np.int32))
    H = brute.parity_matrix(gg)
    B = 9
    x = rng.integers(0, 2, (B, n)).astype(np.uint8)
    s = ((x.astype(np.int64) @ H.T) % 2).astype(np.uint8)
    L = ((1 - 2.0 * x) * 1.5 + rng.normal(0, 1.0, x.shape)).astype(np.float32)
    g = mld.Graph(gg.edge_vn, gg.edge_cn, n, m)
    assert g.stats["max_check_deg"] > 8 and g.stats["n_deg1"] == 90
    for msg in ("f32", "f16"):
        dec = mld.Decoder(g, B, msg_dtype=msg, slab_width=16)
        for it, et in ((1, False), (12, True)):
            out = dec.decode(_dev(L), _dev(s), iters=it, early_term=et, want_post=True)
            ref = oracle.decode(gg, L, s, iters=it, early_term=et)
            if msg == "f32" and it == 1:
                np.testing.assert_allclose(_np(out["post"]), ref["post"], rtol=1e-4, atol=1e-3)
            assert (_np(out["bits"]) == ref["bits"]).mean() >= 0.999
            assert np.array_equal(_np(out["converged"]), ref["converged"])


def test_invalid_arguments_raise(mld):
    w = make_workload(0.1, 4096, 2, 1, 900)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 2)
    with pytest.raises(mld.MldError):
        dec.decode(_dev(_llr32(w)), _dev(w.s), iters=-1)
    big = np.zeros((3, g.n_vn), np.float32)
    with pytest.raises(mld.MldError):
        dec.decode(_dev(big), _dev(np.zeros((3, g.n_cn), np.uint8)), iters=1)
    with pytest.raises(mld.MldError):
        mld.Decoder(g, 0)
    with pytest.raises(mld.MldError):
        mld.Decoder(g, 4, slab_width=24)
