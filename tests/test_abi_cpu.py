"""CPU-side checks of the C ABI: the library loads, exports every declared
symbol, and rejects malformed graphs on the host before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "metldpc.h")


@pytest.fixture(scope="module")
def mld():
    from paper_1711_01783_gb300 import build
    build.build()
    import paper_1711_01783_gb300 as m
    return m


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mld_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_are_all_exported(mld):
    names = _declared()
    assert len(names) >= 10
    lib = ctypes.CDLL(mld.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(mld.EXPORTS)


def test_version_string(mld):
    assert mld.version().startswith("metldpc") and "sm_103a" in mld.version()


def _create(mld, ev, ec, n_vn, n_cn, et=None):
    lib = mld.lib()
    h = ctypes.c_void_p()
    ev = np.ascontiguousarray(ev, np.int32)
    ec = np.ascontiguousarray(ec, np.int32)
    p = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)
    st = lib.mld_graph_create(p(ev), p(ec), p(et), ev.shape[0], n_vn, n_cn, ctypes.byref(h))
    return st, lib.mld_last_error().decode()


def test_graph_validation_happens_on_host(mld):
    st, msg = _create(mld, [0, 1, 5], [0, 0, 1], 4, 2)
    assert st == mld.MLD_EGRAPH and "out of range" in msg
    st, msg = _create(mld, [0, 1, 1], [0, 1, 1], 4, 2)
    assert st == mld.MLD_EGRAPH and "repeated" in msg
    st, msg = _create(mld, [0], [-1], 4, 2)
    assert st == mld.MLD_EGRAPH
    st, msg = _create(mld, [0, 1], [0, 0], 4, 2, et=np.array([0, 9], np.uint8))
    assert st == mld.MLD_EGRAPH and "type" in msg
    st, _ = _create(mld, [], [], -1, 2)
    assert st == mld.MLD_EINVAL


def test_null_handles_are_rejected(mld):
    lib = mld.lib()
    assert lib.mld_decode(None, None, None, 1, 1, 0, None, None, None, None, None) == mld.MLD_EINVAL
    assert lib.mld_graph_destroy(None) == 0 and lib.mld_decoder_destroy(None) == 0
    o = mld.Opts()
    assert lib.mld_decoder_create(None, ctypes.byref(o), ctypes.byref(ctypes.c_void_p())) == mld.MLD_EINVAL


class _FakeCuda:
    """Stands in for a CUDA tensor in host-only checks (nothing is launched)."""

    def __init__(self, shape, dtype, device="cuda:0", is_cuda=True):
        self.shape, self.dtype, self.device, self.is_cuda = tuple(shape), dtype, device, is_cuda

    def dim(self):
        return len(self.shape)


def test_noalloc_binding_rejects_bad_arguments_before_the_library(mld):
    """decode_noalloc passes device pointers only: host tensors, a wrong
    dtype or a wrong shape must raise in the binding, before any call."""
    import torch
    from types import SimpleNamespace
    g = SimpleNamespace(n_vn=10, n_cn=4, handle=None)
    good_l = _FakeCuda((3, 10), torch.float32)
    good_s = _FakeCuda((3, 4), torch.uint8)
    with pytest.raises(TypeError):
        mld.decode_noalloc(g, torch.zeros((3, 10)), torch.zeros((3, 4), dtype=torch.uint8), 5)
    with pytest.raises(TypeError):
        mld.decode_noalloc(g, np.zeros((3, 10), np.float32), good_s, 5)
    with pytest.raises(TypeError):
        mld.decode_noalloc(g, _FakeCuda((3, 10), torch.float64), good_s, 5)
    with pytest.raises(ValueError):
        mld.decode_noalloc(g, _FakeCuda((3, 9), torch.float32), good_s, 5)
    with pytest.raises(ValueError):
        mld.decode_noalloc(g, good_l, _FakeCuda((3, 5), torch.uint8), 5)
    with pytest.raises(ValueError):
        mld.decode_noalloc(g, good_l, _FakeCuda((2, 4), torch.uint8), 5)
    with pytest.raises(ValueError):
        mld.decode_noalloc(g, good_l, _FakeCuda((3, 4), torch.uint8, device="cuda:1"), 5)
    with pytest.raises(ValueError):
        mld.decode_noalloc(g, good_l, good_s, 5, msg_dtype="bf16")


def test_staging_and_stall_hook_are_declared(mld):
    """The staging constants and the timeout test hook are in the header and
    the binding (no GPU call)."""
    m = mld
    hdr = open(HEADER).read()
    for name, val in (("MLD_STAGE_DIRECT", 0), ("MLD_STAGE_BULK", 1), ("MLD_STAGE_BULK_LSU", 2)):
        assert re.search(rf"#define {name}\s+{val}\b", hdr)
        assert getattr(m, name) == val
    assert "int mld_decoder_test_stall(mld_decoder *d, int32_t bytes);" in hdr
    assert [f for f, _ in m.Opts._fields_][-3:] == ["checked", "staging", "reserved"]
