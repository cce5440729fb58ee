"""The allocation-free entry point (mld_decode_noalloc) against mld_decode.

mld_decode_noalloc is for callers that cannot call cudaMalloc (device memory
owned by their own allocator or capped at start-up, or code paths where an
allocation or its implicit device synchronisation is not allowed).  It keeps
its working memory in one static device array shared by every call, so this
file checks that two calls in a row, with different inputs and sizes, each
reproduce what the allocating decoder returns, and that a working set larger
than the array is refused.  It is collected last so that a failure here does
not stop the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

from synthetic import make_workload, preset_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _llr32(w):
    return (2.0 * w.y.astype(np.float64) / (w.sigma.astype(np.float64)[:, None] ** 2)).astype(np.float32)


def _outputs(B, n):
    return (torch.empty((B, n), dtype=torch.uint8, device="cuda"),
            torch.empty((B, n), dtype=torch.float32, device="cuda"),
            torch.empty(B, dtype=torch.uint8, device="cuda"),
            torch.empty(B, dtype=torch.int32, device="cuda"))


def _noalloc(mld, g, msg, llr, s, iters, early_term, outs=None):
    """One call through the C ABI with caller-owned device buffers."""
    B, n = llr.shape[0], g.n_vn
    bits, post, conv, used = outs if outs is not None else _outputs(B, n)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    flags = mld.MLD_DEVICE_PTRS | (mld.MLD_EARLY_TERM if early_term else 0)
    dt = mld.MLD_MSG_F16 if msg == "f16" else mld.MLD_MSG_F32
    st = mld.lib().mld_decode_noalloc(g.handle, dt, p(llr), p(s), B, iters, flags, p(bits), p(post), p(conv),
                                      p(used), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, mld.lib().mld_last_error().decode()
    torch.cuda.synchronize()
    return dict(bits=bits.cpu().numpy(), post=post.cpu().numpy(), converged=conv.cpu().numpy(),
                iters_used=used.cpu().numpy())


def test_noalloc_matches_decoder_on_two_calls_in_a_row():
    import paper_1711_01783_gb300 as mld
    g0 = preset_graph(0.1, 4096, 1)
    g = mld.Graph.from_edges(g0)
    cases = [  # (msg dtype, batch, beta, iterations, early termination)
        ("f16", 70, 0.40, 30, True),
        ("f32", 9, 0.90, 12, False),
    ]
    for k, (msg, B, beta, iters, et) in enumerate(cases):
        w = make_workload(0.1, 4096, B, 1, 4200 + k, beta=beta, graph=g0)
        llr, s = _dev(_llr32(w)), _dev(w.s)
        got = _noalloc(mld, g, msg, llr, s, iters, et)
        dec = mld.Decoder(g, B, msg_dtype=msg)
        ref = dec.decode(llr, s, iters, early_term=et, want_post=True)
        torch.cuda.synchronize()
        # same kernels on the same inputs: the results must coincide
        assert np.array_equal(got["bits"], ref["bits"].cpu().numpy())
        assert np.array_equal(got["converged"], ref["converged"].cpu().numpy())
        assert np.array_equal(got["iters_used"], ref["iters_used"].cpu().numpy())
        np.testing.assert_allclose(got["post"], ref["post"].cpu().numpy(), rtol=0, atol=1e-6)


def test_a_warm_call_takes_no_device_memory():
    """After the first call on the device (which may load the library's
    module and with it the static array), a call must leave the device's
    free memory unchanged: the outputs are allocated beforehand by the
    caller, and the library itself allocates nothing."""
    import paper_1711_01783_gb300 as mld
    g0 = preset_graph(0.1, 4096, 1)
    g = mld.Graph.from_edges(g0)
    w = make_workload(0.1, 4096, 40, 1, 4300, beta=0.40, graph=g0)
    llr, s = _dev(_llr32(w)), _dev(w.s)
    outs = _outputs(40, g.n_vn)
    _noalloc(mld, g, "f16", llr, s, 10, True, outs)  # warm-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    got = _noalloc(mld, g, "f16", llr, s, 10, True, outs)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert got["iters_used"].max() <= 10


def test_noalloc_refuses_a_working_set_larger_than_its_array():
    import paper_1711_01783_gb300 as mld
    g0 = preset_graph(0.1, 200000, 3)
    g = mld.Graph.from_edges(g0)
    B = 64
    llr = torch.zeros((B, g.n_vn), dtype=torch.float32, device="cuda")
    s = torch.zeros((B, g.n_cn), dtype=torch.uint8, device="cuda")
    with pytest.raises(mld.MldError) as e:
        mld.decode_noalloc(g, llr, s, 5, msg_dtype="f16")
    assert e.value.status == mld.MLD_EINVAL and "bytes of scratch" in str(e.value)
