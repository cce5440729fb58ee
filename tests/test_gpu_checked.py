"""Decoders created with `checked` validate the graph store on the device
before decoding and report a corruption through the call's status and
mld_decode_status, without launching any decoding kernel.  The corruption is
a stray write from an unrelated kernel: the library's front-end kernel is
given the store's column array as its output (32 bytes of floats)."""
import numpy as np
import pytest

from synthetic import make_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mld():
    import paper_1711_01783_gb300 as m
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_checked_decoder_decodes_like_the_plain_one(mld):
    w = make_workload(0.1, 4096, 8, 1, 9100, beta=0.35)
    g = mld.Graph.from_edges(w.graph)
    a = mld.Decoder(g, 8, msg_dtype="f16", checked=True)
    b = mld.Decoder(g, 8, msg_dtype="f16")
    for et in (False, True):
        oa = a.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=20, early_term=et, want_post=True)
        ob = b.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=20, early_term=et, want_post=True)
        for k in ("bits", "post", "converged", "iters_used"):
            assert torch.equal(oa[k], ob[k]), k
    assert a.status() == mld.MLD_OK


def test_a_stray_write_into_the_store_is_reported(mld):
    w = make_workload(0.1, 4096, 8, 1, 9200)
    g = mld.Graph.from_edges(w.graph)
    arrays = g.index_arrays()
    assert arrays["n_col"] == g.stats["e_core"] and arrays["n_unit"] == g.n_vn
    dec = mld.Decoder(g, 8, msg_dtype="f32", checked=True)
    dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=3)     # intact store
    assert dec.status() == mld.MLD_OK
    # an unrelated kernel writes 8 floats over col[0..7]
    x = torch.full((1, 8), 3.0, device="cuda")
    alpha = torch.zeros((1, 8), device="cuda")
    alpha[0, 0] = 1.0
    import ctypes
    ynorm = torch.ones(1, device="cuda")
    nvar = torch.ones(1, device="cuda")
    st = mld.lib().mld_md_alice(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(alpha.data_ptr()),
                                ctypes.c_void_p(ynorm.data_ptr()), ctypes.c_void_p(nvar.data_ptr()), 1, 8,
                                ctypes.c_void_p(arrays["col"]),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    with pytest.raises(mld.MldError) as e:
        dec.decode_y(_dev(w.y), _dev(w.sigma), _dev(w.s), iters=3)
    assert e.value.status == mld.MLD_EGRAPH and "col[" in str(e.value)
    assert dec.status() == mld.MLD_EGRAPH
    # (no unchecked decoder may run on this graph: its kernels would read out of bounds)
