"""PEG-built codes through the decoder against the FP64 oracle.

The graph comes from the library's construction (mld_peg_edges, checked edge
for edge against oracle/peg.py on the CPU); decoding it follows the flooding
criteria of tests/test_gpu_parity.py.
"""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from oracle import peg
from synthetic import biawgn_observe, bob_syndrome, random_bits, sigma_for_beta
from tests.parity import _check_frames, _cp_interval, _np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mld():
    import paper_1711_01783_gb300 as m
    return m


@pytest.fixture(scope="module")
def peg_graph(mld):
    n = 4096
    deg, mask = peg.met_spec(n, 0.1, 0.2, 20)
    ev, ec, et = mld.peg_edges(deg, mask, np.random.default_rng(1).permutation(mask.shape[0]))
    return SimpleNamespace(n_vn=n, n_cn=mask.shape[0], edge_vn=ev, edge_cn=ec, edge_type=et)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _frames(g, B, beta, seed):
    sig = sigma_for_beta(0.1, beta)
    x = random_bits(B, g.n_vn, seed)
    return x, bob_syndrome(g, x), biawgn_observe(x, sig, seed), np.full(B, sig, np.float32)


@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_peg_code_decodes_like_the_oracle(mld, peg_graph, msg):
    g = peg_graph
    x, s, y, sig = _frames(g, 16, 0.30, 901)
    dec = mld.Decoder(mld.Graph.from_edges(g), 16, msg_dtype=msg)
    out = dec.decode_y(_dev(y), _dev(sig), _dev(s), iters=50, early_term=True, want_post=True)
    ref = oracle.decode_y(g, y, sig, s, iters=50, early_term=True)
    _check_frames(out, ref, g, s, msg, near_threshold=(msg == "f16"))


def test_peg_frame_error_rate_near_threshold(mld, peg_graph):
    g = peg_graph
    B = 128
    x, s, y, sig = _frames(g, B, 0.42, 77)
    ref = oracle.decode_y(g, y, sig, s, iters=80, early_term=True)
    out = mld.Decoder(mld.Graph.from_edges(g), B, msg_dtype="f32").decode_y(_dev(y), _dev(sig), _dev(s), iters=80,
                                                                            early_term=True)
    _check_frames(out, ref, g, s, "f32", near_threshold=True)
    k = int(B - ref["converged"].sum())
    lo, hi = _cp_interval(k, B)
    print(f"PEG code, beta 0.42: FER {1 - _np(out['converged']).mean():.3f}, oracle {k / B:.3f} [{lo:.3f}, {hi:.3f}]")
