"""Pins for the offset min-sum oracle, oracle.decode_ms.

Offset min-sum keeps the sign rule of the check update (Eqs. 2-3 with the
syndrome sign) and replaces its magnitude phi(sum phi(|q|)) by
max(min |q| - offset, 0) over the other edges.  Pins: on degree-2 checks
the minimum of one value is that value, so with offset 0 a repetition chain
is decoded exactly (the sum-product closed form); on one check of any degree
phi(sum phi(x_i)) <= min x_i, so min-sum's messages are at least as large as
sum-product's with the same signs, and the offset's effect is its closed
form; the coset symmetry; exhaustive ML; the noiseless limit; and planted
mistakes in a copy of the oracle fail a pin.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from synthetic import bob_syndrome, make_workload, preset_graph, random_bits
from tests import brute


def _chain(n):
    return brute.graph_from_edges(n, n - 1, [(i, i) for i in range(n - 1)] + [(i + 1, i) for i in range(n - 1)])


def test_degree_two_chain_is_exact_with_zero_offset():
    rng = np.random.default_rng(31)
    n = 10
    g = _chain(n)
    s = rng.integers(0, 2, n - 1).astype(np.uint8)
    llr = rng.uniform(-2, 2, n)
    sign = 1 - 2 * s.astype(np.float64)
    out = oracle.decode_ms(g, llr[None], s[None], iters=n + 1, offset=0.0)
    ref = oracle.decode(g, llr[None], s[None], iters=n + 1)
    for v in range(n):
        tot = sum(llr[u] * np.prod(sign[min(u, v):max(u, v)]) for u in range(n))
        assert out["post"][0, v] == pytest.approx(tot, rel=1e-12, abs=1e-12)
    np.testing.assert_allclose(out["post"], ref["post"], rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("d,s", [(3, 0), (4, 1), (6, 0), (9, 1)])
def test_single_check_bounds_sum_product_and_offset_closed_form(d, s):
    rng = np.random.default_rng(100 + d)
    g = brute.graph_from_edges(d, 1, [(v, 0) for v in range(d)])
    llr = rng.normal(0.3, 1.5, (20, d))
    syn = np.full((20, 1), s, np.uint8)
    ms = oracle.decode_ms(g, llr, syn, iters=1, offset=0.0)
    sp = oracle.decode(g, llr, syn, iters=1)
    r_ms = ms["post"] - llr
    r_sp = sp["post"] - llr
    nz = np.abs(r_sp) > 1e-12
    assert np.all(np.sign(r_ms[nz]) == np.sign(r_sp[nz]))
    assert np.all(np.abs(r_ms) >= np.abs(r_sp) - 1e-12)
    # the offset: |r| = max(min of the other |L| - offset, 0), signs unchanged
    for off in (0.2, 0.7):
        mo = oracle.decode_ms(g, llr, syn, iters=1, offset=off)["post"] - llr
        for f in range(20):
            for v in range(d):
                others = np.delete(llr[f], v)
                expect = (1 - 2 * s) * np.prod(np.sign(others)) * max(np.abs(others).min() - off, 0.0)
                assert mo[f, v] == pytest.approx(expect, abs=1e-12)


def test_coset_symmetry_and_noiseless_limit():
    g = preset_graph(0.1, 4096, 1)
    w = make_workload(0.1, 4096, 3, 1, 8100, beta=0.5, graph=g)
    L = oracle.channel_llr(w.y, w.sigma)
    a = oracle.decode_ms(g, L, w.s, iters=10, offset=0.1)
    for z in (w.x, random_bits(3, g.n_vn, 55)):
        b = oracle.decode_ms(g, L * (1 - 2.0 * z), w.s ^ bob_syndrome(g, z), iters=10, offset=0.1)
        assert np.array_equal(b["post"], a["post"] * (1 - 2.0 * z))
    c = oracle.decode_ms(g, L, np.zeros_like(w.s), iters=10, offset=0.1)
    assert not np.array_equal(c["post"], a["post"])
    w = make_workload(0.1, 4096, 2, 1, 8200, sigma=0.1, graph=g)
    out = oracle.decode_ms(g, oracle.channel_llr(w.y, w.sigma), w.s, iters=5, offset=0.1, early_term=True)
    assert np.array_equal(out["bits"], w.x) and out["iters_used"].tolist() == [1, 1]


def test_ml_never_worse_and_converged_words_satisfy_syndrome():
    rng = np.random.default_rng(37)
    n, m = 14, 7
    g = brute.random_code(rng, n, m, col_w=3)
    H = brute.parity_matrix(g)
    frames = 200
    x = rng.integers(0, 2, (frames, n)).astype(np.uint8)
    s = ((x.astype(np.int64) @ H.T) % 2).astype(np.uint8)
    sigma = 0.9
    llr = 2 * ((1 - 2.0 * x) + sigma * rng.standard_normal((frames, n))) / sigma ** 2
    out = oracle.decode_ms(g, llr, s, iters=30, offset=0.2, early_term=True)
    bp_err = ml_err = 0
    for f in range(frames):
        ml = brute.ml_decode(H, s[f], llr[f])
        ml_err += int(not np.array_equal(ml, x[f]))
        bp_err += int(not np.array_equal(out["bits"][f], x[f]))
        assert bool(out["converged"][f]) == np.array_equal((H.astype(np.int64) @ out["bits"][f]) % 2, s[f])
    assert ml_err <= bp_err and bp_err > 0


# --------------------------------------------------------------------------
# Planted mistakes in the min-sum function
# --------------------------------------------------------------------------

MUTATIONS = {
    "own message in the minimum": ("if (k2 == k) continue;\n                    const double qe", ";\n                    const double qe"),
    "offset dropped": ("const double mag = mn - J->ms_offset > 0.0 ? mn - J->ms_offset : 0.0;", "const double mag = mn;"),
    "syndrome sign dropped": ("double sgn = (s[c] & 1) ? -1.0 : 1.0;\n                double mn", "double sgn = 1.0;\n                double mn"),
    "sign product dropped": ("if (qe < 0.0) sgn = -sgn;", ";"),
}


def _mutant(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    head, sep, tail = src.partition("static int decode_one_ms")
    assert sep and old in tail, name
    path = tmp_path / f"ms{abs(hash(name))}.c"
    path.write_text(head + sep + tail.replace(old, new, 1))
    so = str(path) + ".so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", so, str(path), "-lm",
                    "-lpthread"], check=True)
    lib = ctypes.CDLL(so)
    i32, i64, dbl, ptr = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    lib.oracle_decode_ms.restype = ctypes.c_int
    lib.oracle_decode_ms.argtypes = [i32, i32, i64, ptr, ptr, dbl, i32, ptr, ptr, i32, i32, dbl, ptr, ptr, ptr,
                                     ptr, i32]

    def run(g, llr, s, iters, offset):
        p = lambda a: ctypes.c_void_p(a.ctypes.data)
        ev = np.ascontiguousarray(g.edge_vn, np.int32)
        ec = np.ascontiguousarray(g.edge_cn, np.int32)
        L = np.ascontiguousarray(np.atleast_2d(llr), np.float64)
        S = np.ascontiguousarray(np.atleast_2d(s), np.uint8)
        B = L.shape[0]
        post = np.zeros_like(L)
        bits = np.zeros(L.shape, np.uint8)
        conv = np.zeros(B, np.uint8)
        used = np.zeros(B, np.int32)
        assert lib.oracle_decode_ms(g.n_vn, g.n_cn, ev.shape[0], p(ev), p(ec), offset, B, p(L), p(S), iters, 0,
                                    25.0, p(post), p(bits), p(conv), p(used), 1) == 0
        return post
    return run


def _pins_hold(run):
    rng = np.random.default_rng(43)
    d, s = 5, 1
    g = brute.graph_from_edges(d, 1, [(v, 0) for v in range(d)])
    llr = rng.normal(0.3, 1.5, (6, d))
    syn = np.full((6, 1), s, np.uint8)
    mo = run(g, llr, syn, 1, 0.3) - llr
    for f in range(6):
        for v in range(d):
            others = np.delete(llr[f], v)
            expect = (1 - 2 * s) * np.prod(np.sign(others)) * max(np.abs(others).min() - 0.3, 0.0)
            if abs(mo[f, v] - expect) > 1e-12:
                return False
    return True


def test_planted_mistakes_fail_a_pin(tmp_path):
    for name, (old, new) in MUTATIONS.items():
        assert not _pins_hold(_mutant(tmp_path, name, old, new)), name
    assert _pins_hold(_mutant(tmp_path, "none", "double mn = lmax;", "double mn = lmax;"))
