"""Parity at the benchmarked sizes (n = 10^6, 64 codewords) for every rate,
for the uneven plan at its real lengths, and in a converging regime.

At these sizes the oracle (FP64, one codeword per host thread) decodes a
sample of the batch; the GPU decodes the whole batch in the launch
configuration the benchmark times.  Criteria (tests/test_gpu_parity.py
derives them): sampled codewords agree with the oracle on >= 99.99 % of
bits with identical converged flags (half messages at rate 0.02, where the
stuck state holds many posteriors within half's rounding of 0: every bit
whose FP64 posterior is more than 1e-2 nats from 0, >= 99.98 % overall); every codeword of the batch satisfies
"converged <=> H x = s"; in the converging regime the frame error rate lies
in the 95 % Clopper-Pearson interval of the oracle's on the same frames,
frames both sides decode are bit-identical, and with float messages the
iteration counts are identical.

The classes of the rate-0.05 and rate-0.02 ensembles (checks of 4 to 6
terms) run the looped check kernels on a grid capped at two waves, so a
thread walks several checks: only full-size graphs reach that loop with
more than one check per thread.
"""
import numpy as np
import pytest

import oracle
from synthetic import make_workload, preset_graph
from tests.parity import _check_frames, _cp_interval, _np, _syndrome_holds

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 1_000_000
ITERS = {0.1: 100, 0.05: 150, 0.02: 200}
SAMPLE = [0, 37, 63]   # first lanes of slab 0, a middle lane, the last lane


@pytest.fixture(scope="module")
def mld():
    import paper_1711_01783_gb300 as m
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", params=[0.05, 0.02])
def rate_case(request):
    """The rate-0.05 / rate-0.02 workloads of the benchmark (beta = 0.90,
    150 / 200 fixed iterations); the oracle decodes three sampled codewords."""
    rate = request.param
    w = make_workload(rate, N, 64, 2, 1000)
    ref = oracle.decode_y(w.graph, w.y[SAMPLE], w.sigma[SAMPLE], w.s[SAMPLE], iters=ITERS[rate])
    return rate, w, ref


@pytest.mark.parametrize("msg", ["f16", "f32"])
def test_full_size_other_rates(mld, rate_case, msg):
    rate, w, ref = rate_case
    it = ITERS[rate]
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 64, msg_dtype=msg)
    out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=it, want_post=True)
    bits = _np(out["bits"])
    conv = _np(out["converged"]).astype(bool)
    assert _np(out["iters_used"]).tolist() == [it] * 64
    assert np.array_equal(_syndrome_holds(w.graph, bits, w.s), conv)
    agree = (bits[SAMPLE] == ref["bits"]).mean()
    d = np.abs(_np(out["post"])[SAMPLE].astype(np.float64) - ref["post"])
    dis = bits[SAMPLE] != ref["bits"]
    la = np.abs(ref["post"][dis])
    print(f"rate {rate} {msg}: sampled bit agreement {agree:.6f}, converged {conv.sum()}/64, "
          f"|dL| median {np.median(d):.3g} p99.9 {np.quantile(d, 0.999):.3g} max {d.max():.3g}; "
          f"{int(dis.sum())} disagreeing bits, FP64 |L| there: max {la.max() if la.size else 0:.3g} "
          f"p50 {np.median(la) if la.size else 0:.3g}; FP64 |L| < 1e-2 on "
          f"{(np.abs(ref['post']) < 1e-2).mean():.5f} of bits, < 1e-3 on {(np.abs(ref['post']) < 1e-3).mean():.5f}")
    assert np.array_equal(conv[SAMPLE], ref["converged"].astype(bool))
    if msg == "f32" or rate != 0.02:
        assert agree >= 0.9999
    else:
        # Half storage at rate 0.02: every frame fails at beta = 0.90, and
        # about 0.17 % of the bits of the stuck state have |L| < 1e-3 nats.
        # Each iteration moves a posterior by up to d_v (2^-11 + 2.3e-4) |r|
        # (rounding of every stored message plus the half fit), about 2.5e-3
        # nats at d_v = 35 and |r| ~ 0.1; in a state that does not converge
        # these perturbations persist, so bits that close to 0 may decide
        # either way.  Every bit farther than 1e-2 nats from 0 must agree.
        assert agree >= 0.9998
        assert la.size == 0 or la.max() < 1e-2, la.max()


@pytest.fixture(scope="module")
def converging():
    """Rate 0.1, n = 10^6, 64 frames at beta = 0.40 (well inside the
    ensemble's decoding region), early termination, cap 100; the oracle
    decodes every frame."""
    w = make_workload(0.1, N, 64, 2, 7000, beta=0.40)
    ref = oracle.decode_y(w.graph, w.y, w.sigma, w.s, iters=100, early_term=True)
    return w, ref


@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_full_size_converging_regime(mld, converging, msg):
    w, ref = converging
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, 64, msg_dtype=msg)
    out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=100, early_term=True)
    k = int(64 - ref["converged"].sum())
    lo, hi = _cp_interval(k, 64)
    fer = 1.0 - _np(out["converged"]).mean()
    print(f"{msg}: FER {fer:.3f}, oracle {k / 64:.3f} [{lo:.3f}, {hi:.3f}], mean iterations "
          f"{_np(out['iters_used']).mean():.2f} (oracle {ref['iters_used'].mean():.2f})")
    # float messages follow the FP64 trajectory in a converging regime; half
    # messages are held to the per-frame criteria
    _check_frames(out, ref, w.graph, w.s, msg)
    assert lo - 1e-12 <= fer <= hi + 1e-12


def test_uneven_plan_at_real_lengths(mld):
    """One plan over an n = 10^6 job (rate 0.05, half messages, slab 16)
    and an n = 2^18 job (rate 0.02, float messages, slab 8), each with its
    own cap, early termination, beta = 0.40: every codeword as single-graph
    decoding, and sampled codewords against the oracle."""
    specs = [(0.05, N, 5, 150, "f16", 16, 21), (0.02, 2 ** 18, 6, 200, "f32", 8, 22)]
    jobs = []
    for k, (rate, n, B, it, msg, W, gs) in enumerate(specs):
        g0 = preset_graph(rate, n, gs)
        w = make_workload(rate, n, B, gs, 7100 + 10 * k, beta=0.40, graph=g0)
        g = mld.Graph.from_edges(g0)
        dec = mld.Decoder(g, B, msg_dtype=msg, slab_width=W)
        jobs.append(dict(w=w, g=g, decoder=dec, y=_dev(w.y), sigma=_dev(w.sigma), syndrome=_dev(w.s),
                         max_iters=it, msg=msg, W=W))
    plan = mld.Plan(jobs, early_term=True, want_post=True)
    outs = plan.launch()
    torch.cuda.synchronize()
    for jb, o in zip(jobs, outs):
        w = jb["w"]
        single = mld.Decoder(jb["g"], w.y.shape[0], msg_dtype=jb["msg"], slab_width=jb["W"])
        ref1 = single.decode_y(jb["y"], jb["sigma"], jb["syndrome"], jb["max_iters"], early_term=True,
                               want_post=True)
        torch.cuda.synchronize()
        for key in ("bits", "post", "converged", "iters_used"):
            assert torch.equal(o[key], ref1[key]), (key, w.graph.n_vn)
        sample = [0, w.y.shape[0] - 1]
        ref = oracle.decode_y(w.graph, w.y[sample], w.sigma[sample], w.s[sample], iters=jb["max_iters"],
                              early_term=True)
        sub = {k: (v[sample] if v is not None else None) for k, v in o.items()}
        _check_frames(sub, ref, w.graph, w.s[sample], jb["msg"])
        print(f"rate {w.rate} n {w.graph.n_vn}: converged {int(o['converged'].sum())}/{w.y.shape[0]}, "
              f"iterations {o['iters_used'].cpu().tolist()} (oracle sample {ref['iters_used'].tolist()})")


def test_many_slabs_at_full_length(mld):
    """512 codewords at n = 10^6 (8 slabs of 64, half messages): message
    offsets of the last slabs pass 2^31 elements (7 x 4.52e6 edges x 64), so
    every slab-relative offset must be 64-bit.  Sampled codewords of the
    first, a middle and the last slab against the oracle."""
    B = 512
    w = make_workload(0.1, N, B, 2, 9400)
    sample = [0, 300, 511]
    it = 20
    ref = oracle.decode_y(w.graph, w.y[sample], w.sigma[sample], w.s[sample], iters=it)
    g = mld.Graph.from_edges(w.graph)
    dec = mld.Decoder(g, B, msg_dtype="f16")
    out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=it, want_post=True)
    bits = _np(out["bits"])
    agree = (bits[sample] == ref["bits"]).mean(axis=1)
    d = np.abs(_np(out["post"])[sample].astype(np.float64) - ref["post"])
    print(f"512 codewords: sampled bit agreement {agree}, |dL| p99.9 {np.quantile(d, 0.999):.3g}")
    assert np.all(agree >= 0.9999)
    assert np.array_equal(_np(out["converged"])[sample].astype(bool), ref["converged"].astype(bool))
