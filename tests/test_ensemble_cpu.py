"""The library's seeded MET ensemble (mld_ensemble_size / mld_ensemble_edges),
on the host: sizes, structure, determinism and errors.

The construction is that of the input module ``synthetic/`` with another
random number generator, so every count and every degree histogram must be
identical to the Python ensemble's, while the edges themselves differ.
"""
import collections

import numpy as np
import pytest

from synthetic import ensemble as pyens


@pytest.fixture(scope="module")
def mld():
    from paper_1711_01783_gb300 import build
    build.build()
    import paper_1711_01783_gb300 as m
    return m


# (rate, d2): core VNs, type-1 checks, type-2 checks, type-1 edges, type-2
# core edges, degree-1 edges at n = 10^6, from the ensemble definition
SIZES_1E6 = {
    (0.1, 20): (200_000, 100_000, 800_000, 520_000, 4_000_000, 800_000),
    (0.05, 22): (120_000, 70_000, 880_000, 312_000, 2_640_000, 880_000),
    (0.02, 32): (60_000, 40_000, 940_000, 156_000, 1_920_000, 940_000),
}


@pytest.mark.parametrize("rate,d2", list(SIZES_1E6))
def test_sizes_at_one_million(mld, rate, d2):
    import ctypes
    n_c, m1, m2, e1, e2, e3 = SIZES_1E6[(rate, d2)]
    e, m = ctypes.c_int64(), ctypes.c_int32()
    st = mld.lib().mld_ensemble_size(rate, 10**6, d2, mld.ENSEMBLE_CORE_FRAC[rate], ctypes.byref(e), ctypes.byref(m))
    assert st == 0
    assert e.value == e1 + e2 + e3
    assert m.value == m1 + m2 == 10**6 - round(rate * 10**6)


def _split(ev, ec, et, n, m):
    vdeg = np.bincount(ev, minlength=n)
    per_type = {t: (ev[et == t], ec[et == t]) for t in (0, 1, 2)}
    return vdeg, per_type


@pytest.mark.parametrize("rate,d2", list(SIZES_1E6))
def test_structure(mld, rate, d2):
    n = 20_000
    ev, ec, et, m = mld.ensemble_edges(rate, n, d2, seed=7)
    cf = mld.ENSEMBLE_CORE_FRAC[rate]
    n_c = round(cf * n)
    m2 = n - n_c
    m1 = n_c - round(rate * n)
    assert m == m1 + m2
    assert ev.min() >= 0 and ev.max() < n and ec.min() >= 0 and ec.max() < m
    # sorted by (check, VN), no repeated pair
    key = ec.astype(np.int64) * n + ev
    assert np.all(np.diff(key) > 0)
    vdeg, per = _split(ev, ec, et, n, m)
    v1, c1 = per[0]
    v2, c2 = per[1]
    v3, c3 = per[2]
    # degree-1 VNs: exactly the m2 VNs of degree 1, each on its own type-2 check
    assert np.array_equal(np.sort(v3), np.sort(np.nonzero(vdeg == 1)[0]))
    assert v3.shape[0] == m2 and np.unique(c3).shape[0] == m2
    t2_checks = set(c3.tolist())
    assert set(c2.tolist()) <= t2_checks
    assert not (set(c1.tolist()) & t2_checks)
    assert len(set(c1.tolist())) == m1
    # core VNs: 2 or 3 type-1 edges (round(0.4 n_c) of them with 2), d2 type-2
    d1 = np.bincount(v1, minlength=n)
    d2v = np.bincount(v2, minlength=n)
    core = np.nonzero(vdeg > 1)[0]
    assert core.shape[0] == n_c
    assert set(np.unique(d1[core]).tolist()) == {2, 3}
    assert int((d1[core] == 2).sum()) == round(0.4 * n_c)
    assert np.all(d2v[core] == d2)
    # check sockets of each type dealt evenly: floor or ceil of the mean
    for vv, cc, mt in ((v1, c1, m1), (v2, c2, m2)):
        cnt = np.bincount(cc, minlength=m)
        cnt = cnt[np.unique(c1 if mt == m1 else c3)]
        assert cnt.max() - cnt.min() <= 1
        assert cnt.sum() == vv.shape[0]


@pytest.mark.parametrize("rate", [0.1, 0.05, 0.02])
def test_histograms_equal_the_python_ensemble(mld, rate):
    n = 8192
    d2 = pyens.RATE_PRESETS[rate]["d2"]
    ev, ec, et, m = mld.ensemble_edges(rate, n, d2, seed=3)
    g = pyens.preset_graph(rate, n, 3)
    assert m == g.n_cn and ev.shape[0] == g.n_edges
    for t in (0, 1, 2):
        a = collections.Counter(np.bincount(ev[et == t], minlength=n).tolist())
        b = collections.Counter(np.bincount(g.edge_vn[g.edge_type == t], minlength=n).tolist())
        assert a == b, t
        a = collections.Counter(np.bincount(ec[et == t], minlength=m).tolist())
        b = collections.Counter(np.bincount(g.edge_cn[g.edge_type == t], minlength=m).tolist())
        assert a == b, t
    # same shape, different random numbers: the edges themselves differ
    assert not np.array_equal(ev, g.edge_vn)


def test_deterministic_in_the_seed(mld):
    a = mld.ensemble_edges(0.05, 5000, 22, seed=11)
    b = mld.ensemble_edges(0.05, 5000, 22, seed=11)
    c = mld.ensemble_edges(0.05, 5000, 22, seed=12)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    assert not np.array_equal(a[0], c[0]) or not np.array_equal(a[1], c[1])
    d = mld.ensemble_edges(0.1, 5000, 20, seed=11, core_frac=0.3)
    assert d[3] == 5000 - 500 and int((np.bincount(d[0], minlength=5000) > 1).sum()) == 1500


def test_errors(mld):
    import ctypes
    lib = mld.lib()
    e, m = ctypes.c_int64(), ctypes.c_int32()
    assert lib.mld_ensemble_size(0.0, 1000, 20, 0.2, ctypes.byref(e), ctypes.byref(m)) == mld.MLD_EINVAL
    assert lib.mld_ensemble_size(0.1, 1000, 0, 0.2, ctypes.byref(e), ctypes.byref(m)) == mld.MLD_EINVAL
    # more information bits than core VNs: no type-1 checks
    assert lib.mld_ensemble_size(0.5, 1000, 20, 0.2, ctypes.byref(e), ctypes.byref(m)) == mld.MLD_EINVAL
    assert "degenerate" in lib.mld_last_error().decode()
    assert lib.mld_ensemble_size(0.1, 1000, 20, 0.2, ctypes.byref(e), ctypes.byref(m)) == 0
    buf = np.empty(e.value - 1, np.int32)
    p = ctypes.c_void_p(buf.ctypes.data)
    assert lib.mld_ensemble_edges(0.1, 1000, 20, 0.2, 1, p, p, None, e.value - 1) == mld.MLD_EINVAL
    # mld_graph_generate rejects a rate outside its table before any device work
    h = ctypes.c_void_p()
    assert lib.mld_graph_generate(0.3, 1000, 20, 1, ctypes.byref(h)) == mld.MLD_EINVAL
    assert not h.value
