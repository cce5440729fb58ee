"""The layered (serial-schedule) decoder against the FP64 layered oracle.

Both sides take the same layering (synthetic.check_layers), so the GPU's
layer-by-layer updates and the oracle's check-by-check order are the same
schedule.  Criteria: one iteration from identical inputs stays within the
per-iteration error bounds of the flooding decoder (tests/test_gpu_parity.py)
with a factor 2 for the errors that later layers of the same iteration
inherit through the posteriors; after N iterations the flooding criteria
(>= 99.99 % of bits, identical converged flags and iteration counts with
float messages in stable regimes; per-frame criteria otherwise); cycle-free
codes reach bitwise MAP; converged words satisfy H x = s.
"""
import numpy as np
import pytest

import oracle
from synthetic import check_layers, layer_order, make_workload, preset_graph
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


def _layered(mld, g0, B, msg):
    lay, _ = check_layers(g0)
    g = mld.Graph.from_edges(g0)
    g.set_layers(lay)
    got, n = g.layers()
    assert np.array_equal(got, lay) and n == lay.max() + 1
    return g, mld.Decoder(g, B, msg_dtype=msg, schedule="layered"), layer_order(lay)


@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_one_iteration_against_the_layered_oracle(mld, msg):
    w = make_workload(0.1, 4096, 8, 1, 6000)
    g, dec, od = _layered(mld, w.graph, 8, msg)
    L = _llr32(w)
    out = dec.decode(_dev(L), _dev(w.s), iters=1, want_post=True)
    ref = oracle.decode_layered(w.graph, L, w.s, iters=1, order=od)
    d = np.abs(_np(out["post"]).astype(np.float64) - ref["post"])
    if msg == "f32":
        bound = 2 * (1e-4 + 1e-5 * np.abs(ref["post"]))
    else:
        dv = w.graph.vn_degree()[None, :]
        bound = 2 * (dv * ((2.0 ** -11 + 2.3e-4) * 25.0 + 2.3e-4) + 1e-4)
    assert np.all(d <= bound), (d.max(), (d - bound).max())
    print(f"{msg}: layered one-iteration |dL| max {d.max():.3g} mean {d.mean():.3g}")


@pytest.mark.parametrize("msg,beta,iters,et", [
    ("f32", 0.9, 30, False),
    ("f32", 0.3, 40, True),
    ("f16", 0.9, 30, False),
    ("f16", 0.3, 40, True),
])
def test_decode_matches_layered_oracle(mld, msg, beta, iters, et):
    w = make_workload(0.1, 4096, 8, 1, 6100, beta=beta)
    g, dec, od = _layered(mld, w.graph, 8, msg)
    out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=iters, early_term=et, want_post=True)
    ref = oracle.decode_layered(w.graph, oracle.channel_llr(w.y, w.sigma), w.s, iters=iters, order=od,
                                early_term=et)
    if beta == 0.9:   # the stuck state is stable: bits agree in both precisions
        _check_frames(out, ref, w.graph, w.s, msg)
        assert (_np(out["bits"]) == ref["bits"]).mean() >= 0.9999
        return
    # converging regime: a frame that fails (on either side) drifts from the
    # FP64 trajectory, so frames are compared one by one; with float messages
    # the outcome and the iteration count of every frame must also agree
    _check_frames(out, ref, w.graph, w.s, msg, near_threshold=True)
    if msg == "f32":
        conv = _np(out["converged"]).astype(bool)
        assert np.array_equal(conv, ref["converged"].astype(bool))
        assert np.array_equal(_np(out["iters_used"])[conv], ref["iters_used"][conv])


@pytest.mark.parametrize("seed", range(4))
def test_tree_codes_reach_map(mld, seed):
    rng = np.random.default_rng(700 + seed)
    t = brute.random_tree_code(rng, int(rng.integers(6, 15)))
    H = brute.parity_matrix(t)
    B = 8
    x = rng.integers(0, 2, (B, t.n_vn)).astype(np.uint8)
    s = ((x.astype(np.int64) @ H.T) % 2).astype(np.uint8)
    L = ((1 - 2.0 * x) * 0.8 + rng.normal(0, 1.2, x.shape)).astype(np.float32)
    g = mld.Graph(t.edge_vn, t.edge_cn, t.n_vn, t.n_cn)   # default layering
    dec = mld.Decoder(g, B, schedule="layered")
    out = dec.decode(_dev(L), _dev(s), iters=t.n_vn + 2, want_post=True)
    for b in range(B):
        np.testing.assert_allclose(_np(out["post"])[b], brute.map_llr(H, s[b], L[b]), rtol=1e-4, atol=1e-4)


def test_frame_error_rate_and_fewer_iterations_than_flooding(mld):
    """Near the ensemble's threshold (n = 4096, beta = 0.42): the layered
    decoder's FER lies in the layered oracle's 95 % interval, and frames
    converge in fewer iterations than with flooding."""
    B = 128
    g0 = preset_graph(0.1, 4096, 1)
    w = make_workload(0.1, 4096, B, 1, 6200, beta=0.42, graph=g0)
    g, dec, od = _layered(mld, g0, B, "f32")
    ref = oracle.decode_layered(g0, oracle.channel_llr(w.y, w.sigma), w.s, iters=60, order=od, early_term=True)
    out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=60, early_term=True)
    _check_frames(out, ref, g0, w.s, "f32", near_threshold=True)
    flo = mld.Decoder(g, B, msg_dtype="f32").decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=60,
                                                      early_term=True)
    both = _np(out["converged"]).astype(bool) & _np(flo["converged"]).astype(bool)
    it_l, it_f = _np(out["iters_used"])[both].mean(), _np(flo["iters_used"])[both].mean()
    k = int(B - ref["converged"].sum())
    lo, hi = _cp_interval(k, B)
    print(f"layered FER {1 - _np(out['converged']).mean():.3f} (oracle {k / B:.3f} [{lo:.3f}, {hi:.3f}]), "
          f"flooding FER {1 - _np(flo['converged']).mean():.3f}; mean iterations on frames both decode: "
          f"layered {it_l:.2f}, flooding {it_f:.2f}")
    assert it_l < 0.75 * it_f


def test_full_size_converging_regime(mld):
    """n = 10^6, 64 codewords, beta = 0.40, early termination (the launch the
    benchmark's schedule comparison times); the oracle decodes three frames."""
    w = make_workload(0.1, 1_000_000, 64, 2, 7000, beta=0.40)
    lay, _ = check_layers(w.graph)
    od = layer_order(lay)
    sample = [0, 37, 63]
    ref = oracle.decode_layered(w.graph, oracle.channel_llr(w.y[sample], w.sigma[sample]), w.s[sample], iters=100,
                                order=od, early_term=True)
    g = mld.Graph.from_edges(w.graph)
    g.set_layers(lay)
    for msg in ("f32", "f16"):
        dec = mld.Decoder(g, 64, msg_dtype=msg, schedule="layered")
        out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=100, early_term=True, want_post=True)
        conv = _np(out["converged"]).astype(bool)
        assert np.array_equal(_syndrome_holds(w.graph, _np(out["bits"]), w.s), conv)
        sub = {k: (v[sample] if v is not None else None) for k, v in out.items()}
        _check_frames(sub, ref, w.graph, w.s[sample], msg)
        print(f"{msg}: layered at n=1e6 converged {conv.sum()}/64, mean iterations "
              f"{_np(out['iters_used']).mean():.2f} (oracle sample {ref['iters_used'].tolist()})")


def test_invalid_layerings_are_refused(mld):
    g0 = preset_graph(0.1, 4096, 1)
    g = mld.Graph.from_edges(g0)
    with pytest.raises(mld.MldError) as e:
        g.set_layers(np.zeros(g.n_cn, np.int32))        # every check in one layer: shared VNs
    assert e.value.status == mld.MLD_EGRAPH
    with pytest.raises(ValueError):
        g.set_layers(np.zeros(3, np.int32))
    with pytest.raises(mld.MldError):
        mld.Decoder(g, 8, msg_dtype="f16", slab_width=16, schedule="layered")
    with pytest.raises(mld.MldError):
        mld.Decoder(g, 8, msg_dtype="f32", vn_update="accumulate", schedule="layered")
    # plans run the flooding schedule
    w = make_workload(0.1, 4096, 2, 1, 6300, graph=g0)
    dec = mld.Decoder(g, 2, schedule="layered")
    with pytest.raises(mld.MldError):
        mld.Plan([dict(decoder=dec, y=_dev(w.y), sigma=_dev(w.sigma), syndrome=_dev(w.s), max_iters=5)])


def test_irregular_graph_against_the_layered_oracle(mld):
    """Checks of degree ~22 and checks with several degree-1 VNs run the
    runtime-degree layered kernel; degree-0 VNs and empty checks as well."""
    from types import SimpleNamespace
    rng = np.random.default_rng(19)
    n, m = 400, 60
    edges = set()
    for v in range(300):
        for c in rng.choice(40, 3, replace=False):
            edges.add((v, int(c)))
    for v in range(300, 390):
        edges.add((v, 40 + (v % 15)))
    e = np.array(sorted(edges), dtype=np.int64)
    gg = SimpleNamespace(n_vn=n, n_cn=m, edge_vn=e[:, 0].astype(np.int32), edge_cn=e[:, 1].astype(np.int32))
    H = brute.parity_matrix(gg)
    B = 9
    x = rng.integers(0, 2, (B, n)).astype(np.uint8)
    s = ((x.astype(np.int64) @ H.T) % 2).astype(np.uint8)
    L = ((1 - 2.0 * x) * 1.5 + rng.normal(0, 1.0, x.shape)).astype(np.float32)
    lay, _ = check_layers(gg)
    g = mld.Graph(gg.edge_vn, gg.edge_cn, n, m)
    g.set_layers(lay)
    dec = mld.Decoder(g, B, msg_dtype="f32", schedule="layered")
    for it, et in ((1, False), (10, True)):
        out = dec.decode(_dev(L), _dev(s), iters=it, early_term=et, want_post=True)
        ref = oracle.decode_layered(gg, L, s, iters=it, order=layer_order(lay), early_term=et)
        if it == 1:
            np.testing.assert_allclose(_np(out["post"]), ref["post"], rtol=1e-4, atol=1e-3)
        assert (_np(out["bits"]) == ref["bits"]).mean() >= 0.999
        assert np.array_equal(_np(out["converged"]), ref["converged"])
        assert np.array_equal(_syndrome_holds(gg, _np(out["bits"]), s), _np(out["converged"]).astype(bool))


@pytest.mark.parametrize("n,B,beta,iters,sample", [
    (4096, 16, 0.30, 60, None),
    (1_000_000, 64, 0.40, 100, [0, 37, 63]),
])
def test_layer_structured_ensemble(mld, n, B, beta, iters, sample):
    """The layer-structured ensemble decoded with its own check groups as
    layers (d2 + 3 = 23 at rate 0.1): against the layered oracle in the same
    order, float and half messages, early termination.  The short code runs
    at beta = 0.30: at 0.40 it sits at its finite-length threshold (about
    half the frames fail), where half-precision rounding moves the iteration
    at which single frames converge by tens of iterations."""
    from synthetic import preset_graph_layered
    g0 = preset_graph_layered(0.1, n, 4)
    lay = g0.meta["layer_of_check"]
    w = make_workload(0.1, n, B, 4, 7300, beta=beta, graph=g0)
    g = mld.Graph.from_edges(g0)
    g.set_layers(lay)
    assert g.layers()[1] == g0.meta["n_layers"] == 23
    sel = list(range(B)) if sample is None else sample
    ref = oracle.decode_layered(g0, oracle.channel_llr(w.y[sel], w.sigma[sel]), w.s[sel], iters=iters,
                                order=layer_order(lay), early_term=True)
    for msg in ("f32", "f16"):
        dec = mld.Decoder(g, B, msg_dtype=msg, schedule="layered")
        out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=iters, early_term=True, want_post=True)
        conv = _np(out["converged"]).astype(bool)
        assert np.array_equal(_syndrome_holds(g0, _np(out["bits"]), w.s), conv)
        sub = {k: (v[sel] if v is not None else None) for k, v in out.items()}
        _check_frames(sub, ref, g0, w.s[sel], msg, near_threshold=msg == "f16")
        print(f"n={n} {msg}: structured layered converged {conv.sum()}/{B}, mean iterations "
              f"{_np(out['iters_used']).mean():.2f} (oracle {ref['iters_used'].mean():.2f})")
        dec.close()


@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_early_termination_decisions_only(mld, msg):
    """Layered decode without soft output: a degree-1 VN's decision compares
    the leave-one-out sum with phi(|L_ch|) instead of taking the sign of
    L_ch + phi(o) (no posterior stored).  Against the layered oracle with
    the near-threshold criteria, and against the soft-output run: frames
    both decode agree bit for bit, converged flags on >= 90 %."""
    w = make_workload(0.1, 4096, 32, 1, 1310, beta=0.36)
    g, dec, od = _layered(mld, w.graph, 32, msg)
    args = (_dev(w.y), _dev(w.sigma), _dev(w.s))
    soft = dec.decode_y(*args, iters=40, early_term=True, want_post=True)
    hard = dec.decode_y(*args, iters=40, early_term=True)
    assert hard.get("post") is None
    ref = oracle.decode_layered(w.graph, oracle.channel_llr(w.y, w.sigma), w.s, iters=40, order=od,
                                early_term=True)
    _check_frames(hard, ref, w.graph, w.s, msg, near_threshold=True)
    both = _np(soft["converged"]).astype(bool) & _np(hard["converged"]).astype(bool)
    assert (_np(soft["converged"]) == _np(hard["converged"])).mean() >= 0.9
    assert np.array_equal(_np(soft["bits"])[both], _np(hard["bits"])[both])
    print(f"{msg}: decisions-only converged {int(_np(hard['converged']).sum())}/32, soft-output "
          f"{int(_np(soft['converged']).sum())}/32, oracle {int(ref['converged'].sum())}/32")


@pytest.mark.parametrize("rate", [0.05, 0.02])
@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_other_rates_against_the_layered_oracle(mld, rate, msg):
    """The check shapes of the rate-0.05 and rate-0.02 ensembles (4 to 6
    terms) in the layered kernels: one iteration within the bounds of the
    one-iteration test, then 30 iterations with early termination against
    the layered oracle (per-frame criteria)."""
    w = make_workload(rate, 20000, 8, 3, 6400, beta=0.30)
    g, dec, od = _layered(mld, w.graph, 8, msg)
    L = _llr32(w)
    out = dec.decode(_dev(L), _dev(w.s), iters=1, want_post=True)
    ref = oracle.decode_layered(w.graph, L, w.s, iters=1, order=od)
    d = np.abs(_np(out["post"]).astype(np.float64) - ref["post"])
    if msg == "f32":
        bound = 2 * (1e-4 + 1e-5 * np.abs(ref["post"]))
    else:
        dv = w.graph.vn_degree()[None, :]
        bound = 2 * (dv * ((2.0 ** -11 + 2.3e-4) * 25.0 + 2.3e-4) + 1e-4)
    assert np.all(d <= bound), (d.max(), (d - bound).max())
    out = dec.decode(_dev(L), _dev(w.s), iters=30, early_term=True, want_post=True)
    ref = oracle.decode_layered(w.graph, L, w.s, iters=30, order=od, early_term=True)
    _check_frames(out, ref, w.graph, w.s, msg, near_threshold=True)
    print(f"rate {rate} {msg}: layers {g.layers()[1]}, one-iteration |dL| max {d.max():.3g}; converged "
          f"{int(_np(out['converged']).sum())}/8 (oracle {int(ref['converged'].sum())}/8)")
