"""Parity of the CUDA decoder (through the C ABI) against the FP64 oracle.

Tolerances (derived from the arithmetic):
* phi: float evaluation of the two polynomial pieces on top of MUFU lg2/ex2
  (relative error about 2^-22 each) -- relative error below 2e-6 on
  [phi(25), 25] for the fit used with float messages, below 2.5e-4 for the
  shorter fit used with half messages (fit error 2.0e-4, under half's 2^-11
  rounding of each stored message).
* One iteration, float messages: each check output carries a few float
  roundings through phi and the prefix/suffix sums; a posterior sums up to
  d_v of them.  Bound used: |dL| <= 1e-4 + 1e-5 |L|.
* One iteration, half messages: each stored message is rounded to half
  (relative error <= 2^-11, |r| <= 25 nats) and carries the half fit's error:
  2.3e-4 relative from the output phi, plus the inputs' 2.3e-4 relative error
  in the leave-one-out sum y, which moves psi(y) by at most
  max |y psi'(y)| * 2.3e-4 <= 1.45 * 2.3e-4 bits (2.3e-4 nats).  So
  |dL| <= d_v * ((2^-11 + 2.3e-4) * 25 + 2.3e-4) + 1e-4.
* After N iterations, float messages: hard decisions agree on >= 99.99 % of
  bits, converged flags and iteration counts identical, and every converged
  word satisfies H x = s exactly.
* After N iterations, half messages, and float messages on many frames near
  the decoding threshold: on frames that BP fails to decode there, the
  trajectory drifts from the FP64 one (float rounding is enough), so the
  comparison is per frame: frames both sides decode are bit-identical
  with identical iteration counts, every converged word satisfies H x = s,
  and the frame error rate lies in the 95 % Clopper-Pearson interval of the
  oracle's.
"""
import numpy as np
import pytest

import oracle
from synthetic import make_workload, preset_graph
from tests import brute
from tests.parity import _check_frames, _cp_interval, _llr32, _np, _syndrome_holds

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mld():
    import paper_1711_01783_gb300 as m
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_library_reports_version(mld):
    assert "sm_103a" in mld.version()


@pytest.mark.parametrize("msg,tol", [("f32", 2e-6), ("f16", 2.5e-4)])
def test_phi_matches_closed_form(mld, msg, tol):
    lo = oracle.phi(25.0)
    x = np.exp(np.linspace(np.log(lo), np.log(25.0), 20001)).astype(np.float32)
    got = _np(mld.phi(_dev(x), msg_dtype=msg)).astype(np.float64)
    xd = x.astype(np.float64)
    ref = np.log1p(2.0 / np.expm1(xd))
    rel = np.abs(got - ref) / ref
    assert rel.max() < tol, rel.max()


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
        bound = dv * ((2.0 ** -11 + 2.3e-4) * 25.0 + 2.3e-4) + 1e-4
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
    _check_frames(out, ref, w.graph, w.s, msg)
    if beta == 0.9:  # the stuck fixed point is stable: bits agree in both precisions
        assert (_np(out["bits"]) == ref["bits"]).mean() >= 0.9999


@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_early_termination_decisions_only(mld, msg):
    # without soft output, a degree-1 decision compares o with phi(|L_ch|)
    # instead of taking the sign of L_ch + phi(o): the two differ only where
    # |L_ch| and |r| agree to within the phi fit's error, so a frame's
    # trajectory may drift (as between float and half), and the criteria are
    # those of near-threshold frames, plus agreement with the soft-output run
    w = make_workload(0.1, 4096, 32, 1, 1300, beta=0.36)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 32, msg_dtype=msg)
    soft = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=40, early_term=True, want_post=True)
    hard = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=40, early_term=True)
    ref = oracle.decode_y(w.graph, w.y, w.sigma, w.s, iters=40, early_term=True)
    _check_frames(hard, ref, w.graph, w.s, msg, near_threshold=True)
    both = _np(soft["converged"]).astype(bool) & _np(hard["converged"]).astype(bool)
    assert (_np(soft["converged"]) == _np(hard["converged"])).mean() >= 0.9
    assert np.array_equal(_np(soft["bits"])[both], _np(hard["bits"])[both])


@pytest.mark.parametrize("B,W,msg", [(5, 32, "f32"), (37, 16, "f32"), (3, 8, "f16"), (70, 64, "f16")])
def test_ragged_batches_and_slab_widths(mld, B, W, msg):
    g0 = preset_graph(0.05, 3000, 4)
    w = make_workload(0.05, 3000, B, 4, 500, beta=0.35, graph=g0)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, B + 3, msg_dtype=msg, slab_width=W)
    out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=25, early_term=True, want_post=True)
    ref = oracle.decode_y(w.graph, w.y, w.sigma, w.s, iters=25, early_term=True)
    _check_frames(out, ref, w.graph, w.s, msg)


def test_frame_error_rate_half_and_float_against_oracle(mld):
    """The FP16-message and FP32 forms reach the oracle's FER on many frames
    near the threshold of the ensemble (n = 4096, beta = 0.42)."""
    B = 192
    g0 = preset_graph(0.1, 4096, 1)
    w = make_workload(0.1, 4096, B, 1, 7000, beta=0.42, graph=g0)
    ref = oracle.decode_y(w.graph, w.y, w.sigma, w.s, iters=60, early_term=True)
    k = int(B - ref["converged"].sum())
    assert 0 < k < B, k  # a regime where frames both succeed and fail
    lo, hi = _cp_interval(k, B)
    g = mld.Graph.from_edges(w.graph)
    for msg in ("f32", "f16"):
        dec = mld.Decoder(g, B, msg_dtype=msg)
        out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=60, early_term=True)
        _check_frames(out, ref, w.graph, w.s, msg, near_threshold=True)
        fer = 1.0 - _np(out["converged"]).mean()
        print(f"{msg}: FER {fer:.3f}, oracle {k / B:.3f} [{lo:.3f}, {hi:.3f}]")
        assert lo <= fer <= hi


def test_host_and_device_pointers_agree(mld):
    w = make_workload(0.1, 4096, 6, 1, 600, beta=0.4)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 8, msg_dtype="f16")
    a = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=20, want_post=True)
    b = dec.decode_y(w.y, w.sigma, w.s, iters=20, want_post=True)
    assert np.array_equal(_np(a["bits"]), b["bits"])
    assert np.array_equal(_np(a["post"]), b["post"])
    assert np.array_equal(_np(a["iters_used"]), b["iters_used"])


def test_pinned_host_buffers_are_used_in_place(mld):
    # page-locked host buffers are read and written by the kernels directly
    w = make_workload(0.1, 4096, 8, 1, 650, beta=0.4)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 8, msg_dtype="f16")
    a = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=20, want_post=True, early_term=True)
    pin = lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
    out = dict(bits=torch.zeros((8, g.n_vn), dtype=torch.uint8).pin_memory(),
               post=torch.zeros((8, g.n_vn), dtype=torch.float32).pin_memory(),
               converged=torch.zeros(8, dtype=torch.uint8).pin_memory(),
               iters_used=torch.zeros(8, dtype=torch.int32).pin_memory())
    b = dec.decode_y(pin(w.y), pin(w.sigma), pin(w.s), iters=20, want_post=True, early_term=True, out=out)
    for k in ("bits", "post", "converged", "iters_used"):
        assert np.array_equal(_np(a[k]), b[k].numpy()), k


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
    # internal units are bits (LLR * log2 e): the round trip costs two roundings
    np.testing.assert_allclose(_np(out["post"]), np.clip(L, -25, 25), rtol=3e-7, atol=0)
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
        for it, et, post in ((1, False, True), (12, True, True), (12, True, False)):
            # early termination without soft output on a graph with irregular
            # and empty checks: degree-1 decisions only, separate syndrome checks
            out = dec.decode(_dev(L), _dev(s), iters=it, early_term=et, want_post=post)
            ref = oracle.decode(gg, L, s, iters=it, early_term=et)
            if msg == "f32" and it == 1:
                np.testing.assert_allclose(_np(out["post"]), ref["post"], rtol=1e-4, atol=1e-3)
            assert (_np(out["bits"]) == ref["bits"]).mean() >= 0.999
            assert np.array_equal(_np(out["converged"]), ref["converged"])
            assert np.array_equal(_syndrome_holds(gg, _np(out["bits"]), s), _np(out["converged"]).astype(bool))


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


@pytest.fixture(scope="module")
def full_size():
    """The benchmarked workload: rate 0.1, n = 10^6, 64 codewords, 100
    iterations, beta = 0.90; the oracle decodes two sampled codewords."""
    w = make_workload(0.1, 1_000_000, 64, 2, 1000)
    sample = [0, 37]
    ref = oracle.decode_y(w.graph, w.y[sample], w.sigma[sample], w.s[sample], iters=100)
    return w, sample, ref


@pytest.mark.parametrize("msg,vn", [("f16", "gather"), ("f32", "gather"), ("f16", "accumulate"),
                                    ("f32", "accumulate")])
def test_full_size_sampled_codewords(mld, full_size, msg, vn):
    w, sample, ref = full_size
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 64, msg_dtype=msg, vn_update=vn)
    out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=100, want_post=True)
    bits = _np(out["bits"])
    conv = _np(out["converged"]).astype(bool)
    assert _np(out["iters_used"]).tolist() == [100] * 64
    # properties at full size: converged words satisfy H x = s, and the rest do not
    assert np.array_equal(_syndrome_holds(w.graph, bits, w.s), conv)
    # sampled codewords against the oracle
    agree = (bits[sample] == ref["bits"]).mean()
    print(f"{msg}: sampled bit agreement {agree:.6f}, converged {conv.sum()}/64")
    assert agree >= 0.9999
    assert np.array_equal(conv[sample], ref["converged"].astype(bool))
    d = np.abs(_np(out["post"])[sample].astype(np.float64) - ref["post"])
    print(f"{msg}: sampled posterior |dL| median {np.median(d):.3g} p99.9 {np.quantile(d, 0.999):.3g}")


def test_sampled_timing_counts_and_changes_no_result(mld):
    w = make_workload(0.1, 4096, 8, 1, 900, beta=0.4)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 8, msg_dtype="f16")
    L = _dev(_llr32(w))
    s = _dev(w.s)
    plain = dec.decode(L, s, iters=10, want_post=True)
    dec.timing(3)
    dec.read_timing()
    timed = dec.decode(L, s, iters=10, want_post=True)
    kt = dec.read_timing()
    dec.timing(0)
    assert np.array_equal(_np(plain["bits"]), _np(timed["bits"]))
    assert np.array_equal(_np(plain["post"]), _np(timed["post"]))
    # iterations 1, 4, 7 and 10 are timed; every launch is counted
    assert kt["check_timed"] == 4 and kt["var_timed"] == 4
    assert kt["var_launches"] == 10
    assert kt["check_launches"] > 0 and kt["check_launches"] % 10 == 0
    assert kt["check_ms"] > 0 and kt["var_ms"] > 0
    assert kt["layout_timed"] == kt["layout_launches"] >= 2
    assert kt["syndrome_launches"] == 2        # the final check and its lane update
    assert dec.read_timing()["check_launches"] == 0
    with pytest.raises(Exception):
        dec.timing(-1)


# ---------------------------------------------------------------------------
# Posterior accumulation (vn_update="accumulate"): the check update adds each
# new message, as stored, into the next posteriors with atomic adds.  Eq. 4
# is the same sum; only the order of its float additions changes, and with
# it the last bits of a posterior: |dL| <= d_v * 2^-24 * (|L_ch| + sum |r|)
# between two runs or against the gather (at most ~1e-4 nats here).
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_accumulate_one_iteration_and_order_independence(mld, msg):
    w = make_workload(0.1, 4096, 64, 1, 1010)
    g = mld.Graph.from_edges(w.graph)
    L = _dev(_llr32(w))
    s = _dev(w.s)
    acc = mld.Decoder(g, 64, msg_dtype=msg, vn_update="accumulate")
    gat = mld.Decoder(g, 64, msg_dtype=msg)
    a1 = acc.decode(L, s, iters=1, want_post=True)
    g1 = gat.decode(L, s, iters=1, want_post=True)
    ref = oracle.decode(w.graph, _llr32(w), w.s, iters=1)
    d = np.abs(_np(a1["post"]).astype(np.float64) - ref["post"])
    if msg == "f32":
        bound = 1e-4 + 1e-5 * np.abs(ref["post"])
    else:
        dv = w.graph.vn_degree()[None, :]
        bound = dv * ((2.0 ** -11 + 2.3e-4) * 25.0 + 2.3e-4) + 1e-4
    assert np.all(d <= bound), (d.max(), (d - bound).max())
    # the same messages summed in another order
    np.testing.assert_allclose(_np(a1["post"]), _np(g1["post"]), rtol=1e-5, atol=1e-4)
    # several iterations, twice: results agree up to the order of additions
    a = acc.decode(L, s, iters=30, want_post=True)
    b = acc.decode(L, s, iters=30, want_post=True)
    gg = gat.decode(L, s, iters=30, want_post=True)
    for x in (b, gg):
        assert (_np(a["bits"]) == _np(x["bits"])).mean() >= 0.9999
        assert np.array_equal(_np(a["converged"]), _np(x["converged"]))
    ref30 = oracle.decode(w.graph, _llr32(w), w.s, iters=30)
    assert (_np(a["bits"]) == ref30["bits"]).mean() >= 0.9999
    assert np.array_equal(_np(a["converged"]), ref30["converged"])


def test_accumulate_falls_back_to_gather_under_early_termination(mld):
    w = make_workload(0.1, 4096, 32, 1, 1020, beta=0.36)
    g = mld.Graph.from_edges(w.graph)
    acc = mld.Decoder(g, 32, msg_dtype="f32", vn_update="accumulate")
    gat = mld.Decoder(g, 32, msg_dtype="f32")
    a = acc.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=40, early_term=True, want_post=True)
    b = gat.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=40, early_term=True, want_post=True)
    for k in ("bits", "post", "converged", "iters_used"):
        assert torch.equal(a[k], b[k]), k


def test_accumulate_rejects_unsupported_decoders(mld):
    w = make_workload(0.1, 4096, 2, 1, 1030)
    g = mld.Graph.from_edges(w.graph)
    with pytest.raises(mld.MldError):
        mld.Decoder(g, 8, msg_dtype="f16", slab_width=16, vn_update="accumulate")
    # a check of degree above 8 (irregular class)
    ev = np.arange(12, dtype=np.int32)
    ec = np.zeros(12, dtype=np.int32)
    gi = mld.Graph(np.concatenate([ev, ev]), np.concatenate([ec, ec + 1]), 12, 2)
    with pytest.raises(mld.MldError):
        mld.Decoder(gi, 4, msg_dtype="f32", vn_update="accumulate")
