"""Offset min-sum on the GPU against the FP64 min-sum oracle.

Min-sum's check update is exact arithmetic (minimum, subtraction, sign
product); the GPU carries LLRs in bits (x log2 e), which moves each value by
a float rounding or two.  Criteria: one iteration from identical inputs
within |dL| <= 1e-4 + 1e-5 |L| (float messages) or the half-storage bound of
the sum-product tests; after N iterations the flooding criteria (>= 99.99 %
of bits, identical converged flags and iteration counts with float messages
in a converging regime; per-frame criteria otherwise); the frame error rate
inside the oracle's 95 % interval near min-sum's threshold.
"""
import numpy as np
import pytest

import oracle
from synthetic import make_workload, preset_graph
from tests.parity import _check_frames, _cp_interval, _llr32, _np, _syndrome_holds

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OFF = 0.7


@pytest.fixture(scope="module")
def mld():
    import paper_1711_01783_gb300 as m
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_one_iteration(mld, msg):
    w = make_workload(0.1, 4096, 8, 1, 8300)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 8, msg_dtype=msg, check_rule="min_sum", ms_offset=OFF)
    L = _llr32(w)
    out = dec.decode(_dev(L), _dev(w.s), iters=1, want_post=True)
    ref = oracle.decode_ms(w.graph, L, w.s, iters=1, offset=OFF)
    d = np.abs(_np(out["post"]).astype(np.float64) - ref["post"])
    if msg == "f32":
        bound = 1e-4 + 1e-5 * np.abs(ref["post"])
    else:
        bound = w.graph.vn_degree()[None, :] * (2.0 ** -11 * 25.0) + 1e-4
    assert np.all(d <= bound), (d.max(), (d - bound).max())
    print(f"{msg}: min-sum one-iteration |dL| max {d.max():.3g}")


@pytest.mark.parametrize("msg,beta,et", [("f32", 0.25, True), ("f16", 0.25, True), ("f32", 0.9, False)])
def test_decode_matches_minsum_oracle(mld, msg, beta, et):
    w = make_workload(0.1, 4096, 8, 1, 8400, beta=beta)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 8, msg_dtype=msg, check_rule="min_sum", ms_offset=OFF)
    out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=40, early_term=et, want_post=True)
    ref = oracle.decode_ms(w.graph, oracle.channel_llr(w.y, w.sigma), w.s, iters=40, offset=OFF, early_term=et)
    if beta == 0.9:
        _check_frames(out, ref, w.graph, w.s, msg)
        return
    _check_frames(out, ref, w.graph, w.s, msg, near_threshold=True)
    if msg == "f32":
        conv = _np(out["converged"]).astype(bool)
        assert np.array_equal(conv, ref["converged"].astype(bool))
        assert np.array_equal(_np(out["iters_used"])[conv], ref["iters_used"][conv])


def test_frame_error_rate_near_threshold(mld):
    B = 128
    g0 = preset_graph(0.1, 4096, 1)
    w = make_workload(0.1, 4096, B, 1, 8500, beta=0.31, graph=g0)
    ref = oracle.decode_ms(g0, oracle.channel_llr(w.y, w.sigma), w.s, iters=60, offset=OFF, early_term=True)
    g = mld.Graph.from_edges(g0)
    dec = mld.Decoder(g, B, msg_dtype="f32", check_rule="min_sum", ms_offset=OFF)
    out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=60, early_term=True)
    _check_frames(out, ref, g0, w.s, "f32", near_threshold=True)
    k = int(B - ref["converged"].sum())
    lo, hi = _cp_interval(k, B)
    print(f"min-sum FER {1 - _np(out['converged']).mean():.3f}, oracle {k / B:.3f} [{lo:.3f}, {hi:.3f}]")


def test_full_size_against_sum_product(mld):
    """n = 10^6, 64 frames at beta = 0.30 (both rules decode every frame
    there at n = 4096): sampled frames against the min-sum oracle, and the
    iteration counts of both rules."""
    w = make_workload(0.1, 1_000_000, 64, 2, 8600, beta=0.30)
    sample = [0, 63]
    ref = oracle.decode_ms(w.graph, oracle.channel_llr(w.y[sample], w.sigma[sample]), w.s[sample], iters=100,
                           offset=OFF, early_term=True)
    g = mld.Graph.from_edges(w.graph)
    ms = mld.Decoder(g, 64, msg_dtype="f16", check_rule="min_sum", ms_offset=OFF)
    out = ms.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=100, early_term=True, want_post=True)
    conv = _np(out["converged"]).astype(bool)
    assert np.array_equal(_syndrome_holds(w.graph, _np(out["bits"]), w.s), conv)
    sub = {k: (v[sample] if v is not None else None) for k, v in out.items()}
    _check_frames(sub, ref, w.graph, w.s[sample], "f16")
    sp = mld.Decoder(g, 64, msg_dtype="f16").decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=100,
                                                      early_term=True)
    print(f"n=1e6 beta 0.30: min-sum converged {conv.sum()}/64 in {_np(out['iters_used']).mean():.2f} iterations; "
          f"sum-product {int(sp['converged'].sum())}/64 in {sp['iters_used'].float().mean():.2f}")


def test_minsum_rejects_unsupported_decoders(mld):
    w = make_workload(0.1, 4096, 2, 1, 8700)
    g = mld.Graph.from_edges(w.graph)
    with pytest.raises(mld.MldError):
        mld.Decoder(g, 8, msg_dtype="f16", slab_width=16, check_rule="min_sum")
    with pytest.raises(mld.MldError):
        mld.Decoder(g, 8, check_rule="min_sum", schedule="layered")
    with pytest.raises(mld.MldError):
        mld.Decoder(g, 8, check_rule="min_sum", ms_offset=-1.0)


@pytest.mark.parametrize("rate", [0.05, 0.02])
@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_other_rates_against_the_minsum_oracle(mld, rate, msg):
    """The check shapes of the rate-0.05 and rate-0.02 ensembles in the
    min-sum kernels (several checks per thread at n = 2e4): one iteration
    within the one-iteration bounds, then 30 iterations with early
    termination against the min-sum oracle."""
    w = make_workload(rate, 20000, 8, 3, 8800, beta=0.25)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 8, msg_dtype=msg, check_rule="min_sum", ms_offset=OFF)
    L = _llr32(w)
    out = dec.decode(_dev(L), _dev(w.s), iters=1, want_post=True)
    ref = oracle.decode_ms(w.graph, L, w.s, iters=1, offset=OFF)
    d = np.abs(_np(out["post"]).astype(np.float64) - ref["post"])
    if msg == "f32":
        bound = 1e-4 + 1e-5 * np.abs(ref["post"])
    else:
        bound = w.graph.vn_degree()[None, :] * (2.0 ** -11 * 25.0) + 1e-4
    assert np.all(d <= bound), (d.max(), (d - bound).max())
    out = dec.decode(_dev(L), _dev(w.s), iters=30, early_term=True, want_post=True)
    ref = oracle.decode_ms(w.graph, L, w.s, iters=30, offset=OFF, early_term=True)
    _check_frames(out, ref, w.graph, w.s, msg, near_threshold=True)
    print(f"rate {rate} {msg}: min-sum one-iteration |dL| max {d.max():.3g}; converged "
          f"{int(_np(out['converged']).sum())}/8 (oracle {int(ref['converged'].sum())}/8)")
