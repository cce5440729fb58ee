"""Parity criteria shared by the GPU test files (the CUDA decoder against the
FP64 oracle); the criteria and their derivation are stated in the docstring
of tests/test_gpu_parity.py."""
import numpy as np


def _np(t):
    return t.cpu().numpy() if t is not None else None


def _llr32(w):
    return (2.0 * w.y.astype(np.float64) / (w.sigma.astype(np.float64)[:, None] ** 2)).astype(np.float32)


def _cp_interval(k, n, alpha=0.05):
    from scipy.stats import beta
    lo = 0.0 if k == 0 else beta.ppf(alpha / 2, k, n - k + 1)
    hi = 1.0 if k == n else beta.ppf(1 - alpha / 2, k + 1, n - k)
    return lo, hi


def _check_frames(out, ref, g, s, msg, near_threshold=False):
    """Parity of one decode against the oracle (criteria in the module doc)."""
    bits = _np(out["bits"])
    conv = _np(out["converged"]).astype(bool)
    it = _np(out["iters_used"])
    assert np.array_equal(_syndrome_holds(g, bits, s), conv)
    if msg == "f32" and not near_threshold:
        assert (bits == ref["bits"]).mean() >= 0.9999
        assert np.array_equal(conv, ref["converged"].astype(bool))
        assert np.array_equal(it, ref["iters_used"])
        return
    both = conv & ref["converged"].astype(bool)
    assert np.array_equal(bits[both], ref["bits"][both])
    # the iteration at which a frame first satisfies the syndrome may move by
    # a few iterations when the trajectory is perturbed; the mean must hold
    if both.any():
        d_it = it[both].astype(np.float64) - ref["iters_used"][both]
        assert abs(d_it.mean()) <= 0.05 * ref["iters_used"][both].mean() + 0.5, d_it
    B = bits.shape[0]
    lo, hi = _cp_interval(int(B - ref["converged"].sum()), B)
    fer = 1.0 - conv.mean()
    assert lo - 1e-12 <= fer <= hi + 1e-12, (fer, lo, hi)


def _syndrome_holds(g, bits, s):
    H_ev, H_ec = g.edge_vn.astype(np.int64), g.edge_cn.astype(np.int64)
    ok = []
    for b in range(bits.shape[0]):
        par = np.bincount(H_ec, weights=bits[b, H_ev].astype(np.float64), minlength=g.n_cn).astype(np.int64) & 1
        ok.append(np.array_equal(par.astype(np.uint8), s[b]))
    return np.array(ok)
