"""Differentiable weighted BP on the GPU against the FP64 oracle's forward
and reverse-mode gradient (which finite differences pin, see
test_oracle_wbp.py).  Gradient tolerance: relative 1e-3 in the norm; the
float forward differs from FP64 by ~1e-6 per message, which moves a few
clamp and sign decisions at most."""
import numpy as np
import pytest

import oracle
from synthetic import make_workload, preset_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mld():
    import paper_1711_01783_gb300 as m
    return m


def _setup(mld, n, B, beta, seed, W=16):
    g0 = preset_graph(0.1, n, seed)
    w = make_workload(0.1, n, B, seed, 60 + seed, beta=beta, graph=g0)
    L = (2.0 * w.y.astype(np.float64) / (w.sigma.astype(np.float64)[:, None] ** 2)).astype(np.float32)
    g = mld.Graph.from_edges(g0)
    dec = mld.Decoder(g, B, msg_dtype="f32", slab_width=W)
    return g0, w, L, dec


def _loss_and_grads(mld, dec, L, s, x, W, k):
    llr = torch.from_numpy(L).cuda().requires_grad_(True)
    wt = torch.from_numpy(W.astype(np.float32)).cuda().requires_grad_(True)
    soft = mld.weighted_bp(dec, llr, torch.from_numpy(s).cuda(), wt, ckpt_k=k)
    y = 1.0 - 2.0 * torch.from_numpy(x.astype(np.float32)).cuda()
    loss = torch.nn.functional.softplus(-y * soft).mean()
    loss.backward()
    return float(loss.detach()), soft.detach().cpu().numpy(), wt.grad.cpu().numpy(), llr.grad.cpu().numpy()


def _relnorm(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_unit_weights_equal_plain_bp(mld):
    g0, w, L, dec = _setup(mld, 4096, 8, 0.5, 1)
    T = 12
    soft, _ = dec.wbp_forward(torch.from_numpy(L).cuda(), torch.from_numpy(w.s).cuda(),
                              torch.ones((T, 3), device="cuda"), keep_tape=False)
    ref = dec.decode(torch.from_numpy(L).cuda(), torch.from_numpy(w.s).cuda(), T, want_post=True)
    np.testing.assert_allclose(soft.cpu().numpy(), ref["post"].cpu().numpy(), rtol=1e-5, atol=1e-5)
    ora = oracle.decode(g0, L, w.s, iters=T)
    np.testing.assert_allclose(soft.cpu().numpy(), ora["post"], rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("k", [1, 2, 5, 6])
def test_gradients_match_oracle(mld, k):
    g0, w, L, dec = _setup(mld, 4096, 4, 0.5, 2)
    T = 6
    rng = np.random.default_rng(3)
    W = 1.0 + 0.25 * rng.uniform(-1, 1, (T, 3))
    loss, soft, dw, dllr = _loss_and_grads(mld, dec, L, w.s, w.x, W, k)
    ref = oracle.wbp(g0, L, w.s, w.x, W)
    assert loss == pytest.approx(ref["loss"], rel=1e-5)
    np.testing.assert_allclose(soft, ref["post"], rtol=1e-4, atol=1e-4)
    assert _relnorm(dw, ref["dw"]) < 1e-3
    assert _relnorm(dllr, ref["dllr"]) < 1e-3


def test_gradients_at_the_training_size(mld):
    """n = 10^5, 16 codewords, T = 20, checkpoint every 5 iterations."""
    g0, w, L, dec = _setup(mld, 100_000, 16, 0.45, 4)
    T = 20
    W = np.full((T, 3), 0.95)
    loss, soft, dw, dllr = _loss_and_grads(mld, dec, L, w.s, w.x, W, 5)
    ref = oracle.wbp(g0, L, w.s, w.x, W)
    print(f"loss {loss:.6f} / {ref['loss']:.6f}; dw rel {_relnorm(dw, ref['dw']):.2e}; "
          f"dllr rel {_relnorm(dllr, ref['dllr']):.2e}")
    assert loss == pytest.approx(ref["loss"], rel=1e-4)
    assert _relnorm(dw, ref["dw"]) < 1e-3
    assert _relnorm(dllr, ref["dllr"]) < 1e-3


def test_weight_gradient_against_gpu_central_differences(mld):
    g0, w, L, dec = _setup(mld, 4096, 8, 0.5, 5)
    T = 5
    W = np.full((T, 3), 1.1)
    _, _, dw, _ = _loss_and_grads(mld, dec, L, w.s, w.x, W, 5)
    s = torch.from_numpy(w.s).cuda()
    llr = torch.from_numpy(L).cuda()
    y = 1.0 - 2.0 * torch.from_numpy(w.x.astype(np.float32)).cuda()

    def loss_at(Wv):
        soft, _ = dec.wbp_forward(llr, s, torch.from_numpy(Wv.astype(np.float32)).cuda(), keep_tape=False)
        return float(torch.nn.functional.softplus(-y.double() * soft.double()).mean())

    h = 1e-2
    for (t, k) in ((0, 0), (2, 1), (4, 2)):
        Wp, Wm = W.copy(), W.copy()
        Wp[t, k] += h
        Wm[t, k] -= h
        fd = (loss_at(Wp) - loss_at(Wm)) / (2 * h)
        assert dw[t, k] == pytest.approx(fd, rel=2e-2, abs=1e-6)


def test_training_lowers_the_loss(mld):
    g0, w, L, dec = _setup(mld, 20_000, 16, 0.45, 6)
    T = 10
    wt = torch.ones((T, 3), device="cuda", requires_grad=True)
    opt = torch.optim.Adam([wt], lr=0.02)
    llr = torch.from_numpy(L).cuda()
    s = torch.from_numpy(w.s).cuda()
    y = 1.0 - 2.0 * torch.from_numpy(w.x.astype(np.float32)).cuda()
    losses = []
    for _ in range(15):
        opt.zero_grad()
        soft = mld.weighted_bp(dec, llr, s, wt, ckpt_k=5)
        loss = torch.nn.functional.softplus(-y * soft).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < losses[0]


def test_reused_tape_buffers_give_the_same_gradients(mld):
    """A destroyed tape's buffers serve the decoder's next forward of the
    same shape: repeated forward + backward calls (and a change of T and of
    ckpt_k in between, which takes fresh buffers) give the gradients of a
    decoder used once."""
    rng = np.random.default_rng(5)
    g0, w, L, dec = _setup(mld, 4096, 8, 0.45, 3)
    results = {}
    for T, k in ((8, 3), (8, 3), (6, 2), (8, 3), (8, 3)):
        Wt = 1.0 + 0.05 * rng.standard_normal((T, 3))
        key = (T, k, float(Wt.sum()))
        got = _loss_and_grads(mld, dec, L, w.s, w.x, Wt, k)
        fresh = _setup(mld, 4096, 8, 0.45, 3)[3]
        ref = _loss_and_grads(mld, fresh, L, w.s, w.x, Wt, k)
        fresh.close()
        assert got[0] == ref[0], key
        for a, b in zip(got[1:], ref[1:]):
            np.testing.assert_array_equal(a, b)
        results[key] = got[0]
    assert len(results) == 5
