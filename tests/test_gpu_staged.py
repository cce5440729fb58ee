"""The staged check update (operands brought into shared memory by bulk
copies one group of checks ahead, mld_opts.staging = MLD_STAGE_BULK)
against the direct one and the oracle.

The arithmetic of both is the same function (check_terms), so decodes must
agree bit for bit: bits, posteriors, converged flags and iteration counts.
Sizes: n = 4096 (one stage per block), n = 10^5 (about a dozen stages per
block, so both buffers are reused with both phase parities), a ragged
batch (the last slab partly padding), classes of every rate, early
termination with soft output (staged) and without (the decisions-only
pass, which stays direct)."""
import numpy as np
import pytest

import oracle
from synthetic import make_workload, preset_graph
from tests.parity import _check_frames, _np, _syndrome_holds

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mld():
    import paper_1711_01783_gb300 as m
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


MODES = ["bulk", "bulk_lsu"]


def _pair(mld, g0, B, mode):
    g = mld.Graph.from_edges(g0)
    return (g, mld.Decoder(g, B, msg_dtype="f16"), mld.Decoder(g, B, msg_dtype="f16", staging=mode))


def _same(o1, o2):
    for key in ("bits", "converged", "iters_used"):
        assert torch.equal(o1[key], o2[key]), key
    if o1.get("post") is not None:
        assert torch.equal(o1["post"], o2["post"])


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("rate,n,B", [
    (0.1, 4096, 64), (0.1, 100_000, 100), (0.05, 100_000, 64), (0.02, 100_000, 64), (0.02, 4096, 7),
])
def test_staged_equals_direct_fixed_iterations(mld, rate, n, B, mode):
    w = make_workload(rate, n, B, 3, 8100)
    g, direct, staged = _pair(mld, w.graph, B, mode)
    args = (_dev(w.y), _dev(w.sigma), _dev(w.s))
    for it in (1, 17):
        o1 = direct.decode_y(*args, iters=it, want_post=True)
        o2 = staged.decode_y(*args, iters=it, want_post=True)
        torch.cuda.synchronize()
        _same(o1, o2)
    assert staged.status() == 0


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("post", [True, False])
def test_staged_equals_direct_early_termination(mld, post, mode):
    w = make_workload(0.1, 100_000, 64, 3, 8200, beta=0.40)
    g, direct, staged = _pair(mld, w.graph, 64, mode)
    args = (_dev(w.y), _dev(w.sigma), _dev(w.s))
    o1 = direct.decode_y(*args, iters=60, early_term=True, want_post=post)
    o2 = staged.decode_y(*args, iters=60, early_term=True, want_post=post)
    torch.cuda.synchronize()
    _same(o1, o2)
    assert int(o2["converged"].sum()) > 0
    assert staged.status() == 0


@pytest.mark.parametrize("mode", MODES)
def test_staged_against_the_oracle(mld, mode):
    """Independent of the direct kernel: one converging and one stuck batch
    at n = 4096 against the FP64 oracle with the flooding criteria."""
    for beta, it, et in ((0.30, 50, True), (0.90, 30, False)):
        w = make_workload(0.1, 4096, 16, 1, 8300, beta=beta)
        g = mld.Graph.from_edges(w.graph)
        dec = mld.Decoder(g, 16, msg_dtype="f16", staging=mode)
        out = dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=it, early_term=et, want_post=True)
        ref = oracle.decode_y(w.graph, w.y, w.sigma, w.s, iters=it, early_term=et)
        _check_frames(out, ref, w.graph, w.s, "f16")
        if beta == 0.90:
            assert (_np(out["bits"]) == ref["bits"]).mean() >= 0.9999


def test_staging_where_it_does_not_apply(mld):
    """Float messages, other slab widths, min-sum and accumulation ignore the
    option (their results equal the direct decoder's); unknown values are
    refused."""
    w = make_workload(0.1, 4096, 16, 1, 8400)
    g = mld.Graph.from_edges(w.graph)
    args = (_dev(w.y), _dev(w.sigma), _dev(w.s))
    for kw in (dict(msg_dtype="f32"), dict(msg_dtype="f16", slab_width=16),
               dict(msg_dtype="f16", check_rule="min_sum"), dict(msg_dtype="f16", vn_update="accumulate")):
        o1 = mld.Decoder(g, 16, **kw).decode_y(*args, iters=9, want_post=True)
        o2 = mld.Decoder(g, 16, staging="bulk", **kw).decode_y(*args, iters=9, want_post=True)
        torch.cuda.synchronize()
        if kw.get("vn_update") == "accumulate":   # sums in arrival order
            assert (o1["bits"] == o2["bits"]).float().mean() >= 0.9999
        else:
            _same(o1, o2)
    with pytest.raises(KeyError):
        mld.Decoder(g, 16, staging="tma")


@pytest.mark.parametrize("mode", MODES)
def test_full_size_headline_shape(mld, mode):
    """n = 10^6, 64 codewords, 100 fixed iterations (the headline workload):
    staged equals direct, and every converged flag matches H x = s."""
    w = make_workload(0.1, 1_000_000, 64, 2, 1000)
    g, direct, staged = _pair(mld, w.graph, 64, mode)
    args = (_dev(w.y), _dev(w.sigma), _dev(w.s))
    o1 = direct.decode_y(*args, iters=100, want_post=True)
    o2 = staged.decode_y(*args, iters=100, want_post=True)
    torch.cuda.synchronize()
    _same(o1, o2)
    assert np.array_equal(_syndrome_holds(w.graph, _np(o2["bits"]), w.s), _np(o2["converged"]).astype(bool))
    assert staged.status() == 0


@pytest.mark.parametrize("mode", MODES)
def test_timeout_path(mld, mode):
    """A stage whose mbarrier expects 16 bytes more than its copies bring
    (mld_decoder_test_stall): block (0, 0) of each staged launch waits 2 s,
    records MLD_ETIMEOUT and leaves without storing; no fault, and the
    context keeps decoding correctly with a fresh decoder."""
    import time
    w = make_workload(0.1, 4096, 64, 1, 8500)
    g = mld.Graph.from_edges(w.graph)
    args = (_dev(w.y), _dev(w.sigma), _dev(w.s))
    dec = mld.Decoder(g, 64, msg_dtype="f16", staging=mode)
    dec.decode_y(*args, iters=1)
    torch.cuda.synchronize()
    assert dec.status() == 0
    dec.test_stall(16)
    t0 = time.time()
    dec.decode_y(*args, iters=1)
    torch.cuda.synchronize()
    dt = time.time() - t0
    assert dec.status() == mld.MLD_ETIMEOUT
    assert 1.9 < dt < 60, dt
    # the status is sticky for that decoder; a new one is clean and exact
    assert dec.status() == mld.MLD_ETIMEOUT
    _, direct, staged = _pair(mld, w.graph, 64, mode)
    o1 = direct.decode_y(*args, iters=5, want_post=True)
    o2 = staged.decode_y(*args, iters=5, want_post=True)
    torch.cuda.synchronize()
    _same(o1, o2)
    assert staged.status() == 0
    with pytest.raises(mld.MldError):
        dec.test_stall(-1)
