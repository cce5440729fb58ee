"""Pins for the oracle's weighted BP and its reverse-mode gradient."""
import numpy as np
import pytest

import oracle
from synthetic import make_workload, preset_graph


def _case(n=600, B=3, beta=0.5, seed=11):
    g = preset_graph(0.1, n, seed)
    w = make_workload(0.1, n, B, seed, 77, beta=beta, graph=g)
    return g, w, oracle.channel_llr(w.y, w.sigma)


def test_unit_weights_reproduce_plain_bp():
    g, w, L = _case()
    T = 7
    out = oracle.wbp(g, L, w.s, w.x, np.ones((T, 3)))
    ref = oracle.decode(g, L, w.s, iters=T)
    assert np.array_equal(out["post"], ref["post"])
    y = 1 - 2.0 * w.x
    loss = np.mean(np.logaddexp(0, -y * ref["post"]))
    assert out["loss"] == pytest.approx(loss, rel=1e-12)


def test_weight_gradient_matches_central_differences():
    g, w, L = _case()
    T = 6
    rng = np.random.default_rng(5)
    W = 1.0 + 0.3 * rng.uniform(-1, 1, (T, 3))
    out = oracle.wbp(g, L, w.s, w.x, W)
    h = 1e-3
    fd = np.zeros_like(W)
    for t in range(T):
        for k in range(3):
            Wp, Wm = W.copy(), W.copy()
            Wp[t, k] += h
            Wm[t, k] -= h
            fd[t, k] = (oracle.wbp(g, L, w.s, w.x, Wp)["loss"] - oracle.wbp(g, L, w.s, w.x, Wm)["loss"]) / (2 * h)
    scale = np.abs(out["dw"]).max()
    assert scale > 0
    np.testing.assert_allclose(out["dw"], fd, rtol=1e-4, atol=1e-5 * scale)


def test_llr_gradient_matches_central_differences():
    g, w, L = _case(B=2)
    T = 5
    W = np.full((T, 3), 0.9)
    out = oracle.wbp(g, L, w.s, w.x, W)
    rng = np.random.default_rng(8)
    h = 1e-3
    for _ in range(12):
        b, v = int(rng.integers(0, L.shape[0])), int(rng.integers(0, L.shape[1]))
        Lp, Lm = L.copy(), L.copy()
        Lp[b, v] += h
        Lm[b, v] -= h
        fd = (oracle.wbp(g, Lp, w.s, w.x, W)["loss"] - oracle.wbp(g, Lm, w.s, w.x, W)["loss"]) / (2 * h)
        assert out["dllr"][b, v] == pytest.approx(fd, rel=1e-4, abs=1e-9)


def test_gradient_is_zero_through_a_saturated_channel_value():
    g, w, L = _case(B=1)
    L = L.copy()
    L[0, 5] = 40.0  # clamped at 25: no gradient flows back to this input
    out = oracle.wbp(g, L, w.s, w.x, np.ones((3, 3)))
    assert out["dllr"][0, 5] == 0.0


def test_weight_gradient_with_saturated_messages():
    """Strong channel values and weights above 1 push many variable-to-check
    messages into the +-25 clamp: their weight derivative must vanish."""
    g = preset_graph(0.1, 600, 11)
    w = make_workload(0.1, 600, 2, 11, 78, sigma=1.0, graph=g)
    L = oracle.channel_llr(w.y, w.sigma)
    T = 3
    W = np.full((T, 3), 1.6)     # ~45 % of the posteriors end beyond +-25
    out = oracle.wbp(g, L, w.s, w.x, W)
    h = 1e-4
    fd = np.zeros_like(W)
    for t in range(T):
        for k in range(3):
            Wp, Wm = W.copy(), W.copy()
            Wp[t, k] += h
            Wm[t, k] -= h
            fd[t, k] = (oracle.wbp(g, L, w.s, w.x, Wp)["loss"] - oracle.wbp(g, L, w.s, w.x, Wm)["loss"]) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    np.testing.assert_allclose(out["dw"], fd, rtol=1e-3, atol=1e-4 * scale)
