"""Pins for the layered (serial-schedule) oracle, oracle.decode_layered.

The layered schedule updates the checks one at a time in a given order, each
check forming its incoming messages from the latest outgoing messages (the
paper's Steps 3-4, Eqs. 2-4, taken check by check instead of all checks at
once).  Each test checks it against something other than itself: bitwise
MAP on cycle-free graphs, the closed form of one sweep along a repetition
chain, the invariance of the result under reordering checks that share no
VN, the coset symmetry, exhaustive ML, the noiseless limit and, where every
check is isolated from the others, the flooding schedule.  A last test plants
mistakes in a copy of the oracle and checks that a pin catches each.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from synthetic import (bob_syndrome, check_layers, layer_order, make_workload, preset_graph,
                       random_bits)
from tests import brute


def _chain(n):
    """Repetition chain: check i joins VN i and VN i+1."""
    return brute.graph_from_edges(n, n - 1, [(i, i) for i in range(n - 1)] + [(i + 1, i) for i in range(n - 1)])


def _signed_sum(llr, sign, u, v):
    lo, hi = min(u, v), max(u, v)
    return llr[u] * np.prod(sign[lo:hi])


@pytest.mark.parametrize("seed", range(10))
def test_tree_codes_match_bitwise_map(seed):
    rng = np.random.default_rng(500 + seed)
    g = brute.random_tree_code(rng, int(rng.integers(5, 15)))
    H = brute.parity_matrix(g)
    x = rng.integers(0, 2, g.n_vn).astype(np.uint8)
    s = (H.astype(np.int64) @ x) % 2
    llr = (1 - 2.0 * x) * 0.8 + rng.normal(0, 1.2, g.n_vn)
    order = rng.permutation(g.n_cn)
    out = oracle.decode_layered(g, llr[None], s[None].astype(np.uint8), iters=g.n_vn + 2, order=order)
    ref = brute.map_llr(H, s, llr)
    np.testing.assert_allclose(out["post"][0], ref, rtol=1e-9, atol=1e-9)


def test_one_sweep_along_a_chain_carries_the_whole_prefix():
    """In chain order, one iteration carries every channel value forward: the
    last VN's posterior is the syndrome-signed sum of all channel LLRs (the
    flooding schedule would have moved each value one check only)."""
    rng = np.random.default_rng(17)
    n = 10
    g = _chain(n)
    s = rng.integers(0, 2, n - 1).astype(np.uint8)
    llr = rng.uniform(-2, 2, n)
    sign = 1 - 2 * s.astype(np.float64)
    fwd = oracle.decode_layered(g, llr[None], s[None], iters=1, order=np.arange(n - 1))
    full = sum(_signed_sum(llr, sign, u, n - 1) for u in range(n))
    assert fwd["post"][0, n - 1] == pytest.approx(full, rel=1e-12, abs=1e-12)
    # in reverse order the first VN collects everything instead
    rev = oracle.decode_layered(g, llr[None], s[None], iters=1, order=np.arange(n - 1)[::-1])
    full0 = sum(_signed_sum(llr, sign, u, 0) for u in range(n))
    assert rev["post"][0, 0] == pytest.approx(full0, rel=1e-12, abs=1e-12)
    # flooding: one hop only
    flo = oracle.decode(g, llr[None], s[None], iters=1)
    assert flo["post"][0, n - 1] == pytest.approx(llr[n - 1] + sign[n - 2] * llr[n - 2], rel=1e-12)
    # after enough iterations both schedules reach the exact chain posterior
    lay = oracle.decode_layered(g, llr[None], s[None], iters=n, order=np.arange(n - 1))
    for v in range(n):
        tot = sum(_signed_sum(llr, sign, u, v) for u in range(n))
        assert lay["post"][0, v] == pytest.approx(tot, rel=1e-12, abs=1e-12)


def test_layers_are_vn_disjoint_and_reordering_inside_a_layer_changes_nothing():
    g = preset_graph(0.1, 4096, 1)
    lay, n_layers = check_layers(g)
    vdeg = np.bincount(g.edge_vn, minlength=g.n_vn)
    core = vdeg[g.edge_vn] >= 2
    for L in range(n_layers):
        sel = core & (lay[g.edge_cn] == L)
        assert np.unique(g.edge_vn[sel]).size == sel.sum()   # no core VN twice in a layer
    w = make_workload(0.1, 4096, 3, 1, 5100, beta=0.4, graph=g)
    L0 = oracle.channel_llr(w.y, w.sigma)
    a = oracle.decode_layered(g, L0, w.s, iters=8, order=layer_order(lay))
    rng = np.random.default_rng(3)
    # the same layers, their checks shuffled inside each layer
    key = lay.astype(np.int64) * g.n_cn + rng.permutation(g.n_cn)
    b = oracle.decode_layered(g, L0, w.s, iters=8, order=np.argsort(key).astype(np.int32))
    assert np.array_equal(a["post"], b["post"])
    # a different serial order (checks sharing VNs swapped) is a different schedule
    c = oracle.decode_layered(g, L0, w.s, iters=8, order=np.arange(g.n_cn))
    assert not np.array_equal(a["post"], c["post"])


def test_isolated_checks_make_layered_equal_flooding():
    """Checks that share no VN: every order is the flooding schedule."""
    rng = np.random.default_rng(23)
    edges = []
    v = 0
    for c in range(6):
        for _ in range(int(rng.integers(2, 6))):
            edges.append((v, c))
            v += 1
    g = brute.graph_from_edges(v, 6, edges)
    llr = rng.normal(0.3, 1.5, (4, v))
    s = rng.integers(0, 2, (4, 6)).astype(np.uint8)
    a = oracle.decode_layered(g, llr, s, iters=3, order=rng.permutation(6))
    b = oracle.decode(g, llr, s, iters=3)
    np.testing.assert_allclose(a["post"], b["post"], rtol=1e-14, atol=1e-14)


def test_coset_symmetry():
    g = preset_graph(0.1, 4096, 1)
    lay, _ = check_layers(g)
    od = layer_order(lay)
    w = make_workload(0.1, 4096, 3, 1, 5200, beta=0.5, graph=g)
    L = oracle.channel_llr(w.y, w.sigma)
    a = oracle.decode_layered(g, L, w.s, iters=10, order=od)
    for z in (w.x, random_bits(3, g.n_vn, 77)):
        b = oracle.decode_layered(g, L * (1 - 2.0 * z), w.s ^ bob_syndrome(g, z), iters=10, order=od)
        assert np.array_equal(b["post"], a["post"] * (1 - 2.0 * z))
    c = oracle.decode_layered(g, L, np.zeros_like(w.s), iters=10, order=od)
    assert not np.array_equal(c["post"], a["post"])


def test_ml_never_worse_and_converged_words_satisfy_syndrome():
    rng = np.random.default_rng(29)
    n, m = 14, 7
    g = brute.random_code(rng, n, m, col_w=3)
    H = brute.parity_matrix(g)
    frames = 200
    x = rng.integers(0, 2, (frames, n)).astype(np.uint8)
    s = ((x.astype(np.int64) @ H.T) % 2).astype(np.uint8)
    sigma = 0.9
    llr = 2 * ((1 - 2.0 * x) + sigma * rng.standard_normal((frames, n))) / sigma ** 2
    out = oracle.decode_layered(g, llr, s, iters=30, order=rng.permutation(m), early_term=True)
    bp_err = ml_err = 0
    for f in range(frames):
        ml = brute.ml_decode(H, s[f], llr[f])
        ml_err += int(not np.array_equal(ml, x[f]))
        bp_err += int(not np.array_equal(out["bits"][f], x[f]))
        assert bool(out["converged"][f]) == np.array_equal((H.astype(np.int64) @ out["bits"][f]) % 2, s[f])
    assert ml_err <= bp_err and bp_err > 0


def test_noiseless_limit_and_early_termination():
    g = preset_graph(0.1, 4096, 1)
    od = layer_order(check_layers(g)[0])
    w = make_workload(0.1, 4096, 2, 1, 5300, sigma=0.1, graph=g)
    out = oracle.decode_layered(g, oracle.channel_llr(w.y, w.sigma), w.s, iters=5, order=od, early_term=True)
    assert np.array_equal(out["bits"], w.x) and out["iters_used"].tolist() == [1, 1]
    # early termination stops at the first iteration whose decision matches
    w = make_workload(0.1, 4096, 3, 1, 5400, beta=0.35, graph=g)
    L = oracle.channel_llr(w.y, w.sigma)
    et = oracle.decode_layered(g, L, w.s, iters=40, order=od, early_term=True)
    assert et["converged"].all()
    for b in range(3):
        lb = int(et["iters_used"][b])
        fixed = oracle.decode_layered(g, L[b:b + 1], w.s[b:b + 1], iters=lb, order=od)
        assert np.array_equal(fixed["post"][0], et["post"][b])
        if lb > 1:
            before = oracle.decode_layered(g, L[b:b + 1], w.s[b:b + 1], iters=lb - 1, order=od)
            assert before["converged"][0] == 0


def test_layered_needs_fewer_iterations_than_flooding():
    """The property the schedule is used for: at the same channel, frames
    converge in fewer iterations (measured on 16 frames at n = 4096)."""
    g = preset_graph(0.1, 4096, 1)
    od = layer_order(check_layers(g)[0])
    w = make_workload(0.1, 4096, 16, 1, 5500, beta=0.35, graph=g)
    L = oracle.channel_llr(w.y, w.sigma)
    fl = oracle.decode(g, L, w.s, iters=80, early_term=True)
    la = oracle.decode_layered(g, L, w.s, iters=80, order=od, early_term=True)
    both = fl["converged"].astype(bool) & la["converged"].astype(bool)
    assert both.sum() >= 12
    assert la["iters_used"][both].mean() < 0.75 * fl["iters_used"][both].mean()


def test_order_is_validated():
    g = _chain(4)
    with pytest.raises(RuntimeError):
        oracle.decode_layered(g, np.zeros((1, 4)), np.zeros((1, 3), np.uint8), 1, order=[0, 0, 1])


# --------------------------------------------------------------------------
# Planted mistakes: each edit of the layered function makes a pin fail
# --------------------------------------------------------------------------

MUTATIONS = {
    "checks in index order instead of the given order": ("const int32_t c = J->order[k];", "const int32_t c = k;"),
    "syndrome sign dropped": ("double sgn = (s[c] & 1) ? -1.0 : 1.0;\n                double sum", "double sgn = 1.0;\n                double sum"),
    "own message kept in the leave-one-out sum": ("if (k2 == k1) continue;", ";"),
    "own message kept in q": ("if (a->vedge[k2] != e) acc += r[a->vedge[k2]];", "acc += r[a->vedge[k2]];"),
}


def _mutant(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    head, sep, tail = src.partition("static int decode_one_layered")
    assert sep and old in tail, name
    path = tmp_path / f"m{abs(hash(name))}.c"
    path.write_text(head + sep + tail.replace(old, new, 1))
    so = str(path) + ".so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", so, str(path), "-lm",
                    "-lpthread"], check=True)
    lib = ctypes.CDLL(so)
    i32, i64, dbl, ptr = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    lib.oracle_decode_layered.restype = ctypes.c_int
    lib.oracle_decode_layered.argtypes = [i32, i32, i64, ptr, ptr, ptr, i32, ptr, ptr, i32, i32, dbl, ptr, ptr,
                                          ptr, ptr, i32]

    def run(g, llr, s, iters, order):
        p = lambda a: ctypes.c_void_p(a.ctypes.data)
        ev = np.ascontiguousarray(g.edge_vn, np.int32)
        ec = np.ascontiguousarray(g.edge_cn, np.int32)
        L = np.ascontiguousarray(np.atleast_2d(llr), np.float64)
        S = np.ascontiguousarray(np.atleast_2d(s), np.uint8)
        od = np.ascontiguousarray(order, np.int32)
        B = L.shape[0]
        post = np.zeros_like(L)
        bits = np.zeros(L.shape, np.uint8)
        conv = np.zeros(B, np.uint8)
        used = np.zeros(B, np.int32)
        st = lib.oracle_decode_layered(g.n_vn, g.n_cn, ev.shape[0], p(ev), p(ec), p(od), B, p(L), p(S), iters, 0,
                                       25.0, p(post), p(bits), p(conv), p(used), 1)
        assert st == 0
        return post
    return run


def _pins_hold(run):
    """The chain, tree and coset pins on one small case each."""
    rng = np.random.default_rng(41)
    n = 8
    g = _chain(n)
    s = rng.integers(0, 2, n - 1).astype(np.uint8)
    s[0] = 1
    llr = rng.uniform(-2, 2, n)
    sign = 1 - 2 * s.astype(np.float64)
    post = run(g, llr, s, 1, np.arange(n - 1)[::-1])
    if abs(post[0, 0] - sum(_signed_sum(llr, sign, u, 0) for u in range(n))) > 1e-9:
        return False
    t = brute.random_tree_code(np.random.default_rng(5), 10)
    H = brute.parity_matrix(t)
    x = rng.integers(0, 2, t.n_vn).astype(np.uint8)
    st = ((H.astype(np.int64) @ x) % 2).astype(np.uint8)
    lt = (1 - 2.0 * x) * 0.8 + rng.normal(0, 1.2, t.n_vn)
    pt = run(t, lt, st, t.n_vn + 2, np.arange(t.n_cn))
    return bool(np.allclose(pt[0], brute.map_llr(H, st, lt), rtol=1e-9, atol=1e-9))


def test_planted_mistakes_fail_a_pin(tmp_path):
    for name, (old, new) in MUTATIONS.items():
        run = _mutant(tmp_path, name, old, new)
        assert not _pins_hold(run), name
    # and the unmodified function passes them
    assert _pins_hold(_mutant(tmp_path, "none", "const int32_t c = J->order[k];", "const int32_t c = J->order[k];"))
