"""The multidimensional-reconciliation kernels against the FP64 oracle
(oracle/md.py), and the front end feeding the decoder.

Both sides compute in their own arithmetic from the same samples: alpha and
|y| to float rounding (relative 1e-5), Alice's LLRs to 1e-5 relative of
their block's scale; then Bob's syndrome of his bits and Alice's LLRs from
the front end decode to Bob's bits in a regime where the decoder converges.
"""
import numpy as np
import pytest

from oracle import md
from synthetic import bob_syndrome, preset_graph, sigma_for_beta

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mld():
    import paper_1711_01783_gb300 as m
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_bob_and_alice_match_the_oracle(mld):
    rng = np.random.default_rng(11)
    rows, n = 5, 8 * 3001
    sx, sz = 1.0, 0.8
    x = rng.normal(0, sx, (rows, n)).astype(np.float32)
    y = (x + rng.normal(0, sz, (rows, n))).astype(np.float32)
    bits = rng.integers(0, 2, (rows, n)).astype(np.uint8)
    alpha, ynorm = mld.md_bob(_dev(y), _dev(bits))
    a_ref, n_ref = md.bob(y.astype(np.float64), bits)
    np.testing.assert_allclose(ynorm.cpu().numpy(), n_ref, rtol=1e-5)
    np.testing.assert_allclose(alpha.cpu().numpy(), a_ref, rtol=0, atol=2e-6)   # |alpha_i| <= 1
    nv = np.full(rows, sz ** 2, np.float32)
    llr = mld.md_alice(_dev(x), alpha, ynorm, _dev(nv)).cpu().numpy().astype(np.float64)
    # the oracle from the same (float32) messages Bob sent
    ref = md.alice(x.astype(np.float64), alpha.cpu().numpy().astype(np.float64),
                   ynorm.cpu().numpy().astype(np.float64), sz ** 2)
    scale = np.repeat(2 * ynorm.cpu().numpy().astype(np.float64) * np.abs(x).reshape(rows, -1, 8).max(axis=2)
                      / (np.sqrt(8) * sz ** 2), 8, axis=1) * np.sqrt(8)
    assert np.all(np.abs(llr - ref) <= 1e-5 * scale + 1e-6), np.abs(llr - ref).max()
    # noiseless: Alice's decisions are Bob's bits
    a0, n0 = mld.md_bob(_dev(x), _dev(bits))
    l0 = mld.md_alice(_dev(x), a0, n0, _dev(nv)).cpu().numpy()
    assert np.array_equal((l0 < 0).astype(np.uint8), bits)


def test_front_end_feeds_the_decoder(mld):
    """Gaussian raw keys at the SNR of the rate-0.1 code at beta = 0.30:
    Bob's syndrome and Alice's front-end LLRs decode to Bob's bits."""
    rng = np.random.default_rng(12)
    g0 = preset_graph(0.1, 4096, 1)
    B, n = 16, g0.n_vn
    # the virtual channel's signal-to-noise is the physical one, sigma_x^2 / sigma_z^2
    sig = sigma_for_beta(0.1, 0.30)
    sx, sz = 1.0, sig
    x = rng.normal(0, sx, (B, n)).astype(np.float32)
    y = (x + rng.normal(0, sz, (B, n))).astype(np.float32)
    bits = rng.integers(0, 2, (B, n)).astype(np.uint8)
    s = bob_syndrome(g0, bits)
    alpha, ynorm = mld.md_bob(_dev(y), _dev(bits))
    llr = mld.md_alice(_dev(x), alpha, ynorm, _dev(np.full(B, sz ** 2, np.float32)))
    g = mld.Graph.from_edges(g0)
    out = mld.Decoder(g, B, msg_dtype="f32").decode(llr, _dev(s), iters=60, early_term=True)
    conv = out["converged"].cpu().numpy().astype(bool)
    got = out["bits"].cpu().numpy()
    print(f"front end + decoder: {conv.sum()}/{B} frames decoded")
    assert conv.sum() >= B - 2
    assert np.array_equal(got[conv], bits[conv])


def test_bad_arguments(mld):
    y = torch.zeros(12, device="cuda")
    with pytest.raises(ValueError):
        mld.md_bob(y, torch.zeros(12, dtype=torch.uint8, device="cuda"))
    with pytest.raises(TypeError):
        mld.md_bob(torch.zeros(16), torch.zeros(16, dtype=torch.uint8))
