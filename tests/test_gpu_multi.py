"""Plans over several graphs (uneven batches) against single-graph decoding
and the FP64 oracle.  A plan runs the same device functions as mld_decode,
so each job must reproduce its single-graph result exactly."""
import numpy as np
import pytest

import oracle
from synthetic import make_workload, preset_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def mld():
    import paper_1711_01783_gb300 as m
    return m


def _jobs(mld, specs, beta):
    """specs: (rate, n, batch, max_iters, msg, slab_width, graph_seed)."""
    out = []
    for k, (rate, n, B, it, msg, W, gs) in enumerate(specs):
        g0 = preset_graph(rate, n, gs)
        w = make_workload(rate, n, B, gs, 900 + 10 * k, beta=beta, graph=g0)
        g = mld.Graph.from_edges(g0)
        dec = mld.Decoder(g, B + 2, msg_dtype=msg, slab_width=W)
        out.append(dict(w=w, g=g, decoder=dec, y=_dev(w.y), sigma=_dev(w.sigma), syndrome=_dev(w.s),
                        max_iters=it, msg=msg, W=W))
    return out


SPECS = [(0.1, 4096, 5, 30, "f16", 16, 1), (0.05, 3000, 9, 45, "f32", 8, 4),
         (0.02, 5000, 3, 60, "f16", 64, 6), (0.1, 2048, 70, 20, "f32", 32, 8)]


@pytest.mark.parametrize("early_term,beta", [(True, 0.35), (False, 0.9), (True, 0.9)])
def test_plan_reproduces_single_graph_decoding(mld, early_term, beta):
    jobs = _jobs(mld, SPECS, beta)
    plan = mld.Plan(jobs, early_term=early_term, want_post=True)
    for rep in range(2):  # a plan can be replayed; every launch starts afresh
        outs = plan.launch()
        torch.cuda.synchronize()
        for jb, o in zip(jobs, outs):
            ref_dec = mld.Decoder(jb["g"], jb["y"].shape[0], msg_dtype=jb["msg"], slab_width=jb["W"])
            ref = ref_dec.decode_y(jb["y"], jb["sigma"], jb["syndrome"], jb["max_iters"],
                                   early_term=early_term, want_post=True)
            torch.cuda.synchronize()
            for key in ("bits", "post", "converged", "iters_used"):
                assert torch.equal(o[key], ref[key]), (key, jb["w"].graph.n_vn, rep)


def test_plan_against_oracle(mld):
    jobs = _jobs(mld, SPECS[:3], 0.35)
    plan = mld.Plan(jobs, early_term=True)
    outs = plan.launch()
    torch.cuda.synchronize()
    for jb, o in zip(jobs, outs):
        w = jb["w"]
        ref = oracle.decode_y(w.graph, w.y, w.sigma, w.s, iters=jb["max_iters"], early_term=True)
        conv = o["converged"].cpu().numpy()
        bits = o["bits"].cpu().numpy()
        both = conv.astype(bool) & ref["converged"].astype(bool)
        assert np.array_equal(bits[both], ref["bits"][both])
        if jb["msg"] == "f32":
            assert np.array_equal(conv, ref["converged"])
            assert np.array_equal(o["iters_used"].cpu().numpy(), ref["iters_used"])


def test_plan_with_a_zero_iteration_job(mld):
    jobs = _jobs(mld, [(0.1, 4096, 4, 0, "f32", 32, 1), (0.05, 3000, 3, 10, "f16", 64, 4)], 0.4)
    outs = mld.Plan(jobs, early_term=True, want_post=True).launch()
    torch.cuda.synchronize()
    w = jobs[0]["w"]
    L = (2.0 * w.y.astype(np.float64) / (w.sigma.astype(np.float64)[:, None] ** 2))
    assert np.array_equal(outs[0]["bits"].cpu().numpy(), (np.clip(L, -25, 25) < 0).astype(np.uint8))
    assert outs[0]["iters_used"].cpu().numpy().tolist() == [0] * 4
    assert outs[1]["iters_used"].cpu().numpy().max() <= 10


def test_plan_rejects_bad_jobs(mld):
    jobs = _jobs(mld, SPECS[:2], 0.5)
    with pytest.raises(mld.MldError):
        mld.Plan([jobs[0], dict(jobs[1], decoder=jobs[0]["decoder"])])
    with pytest.raises(mld.MldError):
        big = dict(jobs[0], y=torch.zeros((50, jobs[0]["g"].n_vn), device="cuda"),
                   syndrome=torch.zeros((50, jobs[0]["g"].n_cn), dtype=torch.uint8, device="cuda"),
                   sigma=torch.ones(50, device="cuda"))
        mld.Plan([big])


def test_decoder_tuner_picks_a_valid_fastest_option(mld, tmp_path):
    from paper_1711_01783_gb300.tune import DecoderTuner
    g0 = preset_graph(0.1, 4096, 1)
    g = mld.Graph.from_edges(g0)
    tuner = DecoderTuner(str(tmp_path / "tune.json"), iters=3, reps=2)
    for msg in ("f16", "f32"):
        opts = tuner.choose_options(g, 64, msg)
        times = tuner.trials[tuner._key(g, 64, msg)]
        assert opts == min(times, key=lambda t: t[0])[1]
        # 4 widths with the gather + accumulation (+ two staged forms, half)
        assert len(times) == (7 if msg == "f16" else 5)
        dec = mld.Decoder(g, 64, msg_dtype=msg, **opts)   # the choice builds a working decoder
        w = make_workload(0.1, 4096, 64, 1, 9300, beta=0.35, graph=g0)
        out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), 20)
        assert out["bits"].shape == (64, 4096)
    # cached: a new tuner reads the same choice without timing
    again = DecoderTuner(str(tmp_path / "tune.json"))
    assert again.choose_options(g, 64, "f16") == tuner.choose_options(g, 64, "f16")
    assert not again.trials
