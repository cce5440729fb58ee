"""Progressive edge growth: the oracle (oracle/peg.py) pinned against the
definition with independent graph code, and the library's construction
(mld_peg_edges, host only) against the oracle, edge for edge."""
import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import shortest_path

from oracle import peg


def _regular_spec(n, dv, m):
    return np.full((1, n), dv, np.int64), np.ones(m, np.int64)


def _check_structure(deg, mask, ev, ec, et):
    T, n = deg.shape
    for t in range(T):
        np.testing.assert_array_equal(np.bincount(ev[et == t], minlength=n), deg[t])
    assert np.all((mask[ec] >> et.astype(np.int64)) & 1)
    pairs = ev.astype(np.int64) * mask.shape[0] + ec
    assert np.unique(pairs).size == pairs.size


def test_met_structure_and_degree1_bijection():
    deg, mask = peg.met_spec(400, 0.1, 0.2, 8)
    ev, ec, et = peg.peg(deg, mask)
    _check_structure(deg, mask, ev, ec, et)
    # degree-1 VNs come first and take distinct checks of their type
    d1 = et == 2
    assert np.unique(ec[d1]).size == d1.sum()


def test_every_placement_is_farthest_then_lightest():
    """Replay: before each edge, distances from its VN in the graph built so
    far (scipy shortest paths on the bipartite graph) must make the chosen
    check the farthest allowed one, then the lowest in (degree, prio)."""
    rng = np.random.default_rng(3)
    deg, mask = peg.met_spec(160, 0.1, 0.2, 5)
    n, m = deg.shape[1], mask.shape[0]
    prio = rng.permutation(m)
    ev, ec, et = peg.peg(deg, mask, prio)
    for k in range(ev.shape[0]):
        v, c, t = int(ev[k]), int(ec[k]), int(et[k])
        if k:
            a = coo_matrix((np.ones(k), (ev[:k], n + ec[:k])), shape=(n + m, n + m))
            dist = shortest_path(a, directed=False, unweighted=True, indices=v)[n:]
        else:
            dist = np.full(m, np.inf)
        cdeg = np.bincount(ec[:k], minlength=m)
        allowed = [x for x in range(m) if (mask[x] >> t) & 1 and not np.any((ev[:k] == v) & (ec[:k] == x))]
        far = max(dist[x] for x in allowed)
        best = min((x for x in allowed if dist[x] == far), key=lambda x: (cdeg[x], prio[x]))
        assert c == best, k


def test_no_four_cycles_where_the_socket_graph_has_them():
    deg, mask = _regular_spec(200, 3, 100)
    ev, ec, et = peg.peg(deg, mask)
    _check_structure(deg, mask, ev, ec, et)
    H = np.zeros((100, 200), np.int64)
    H[ec, ev] = 1
    overlap = H.T @ H
    np.fill_diagonal(overlap, 0)
    assert overlap.max() <= 1          # no two VNs share two checks: girth >= 6
    rng = np.random.default_rng(0)
    sockets = rng.permutation(np.repeat(np.arange(100), 6))
    Hs = np.zeros((100, 200), np.int64)
    np.add.at(Hs, (sockets, np.repeat(np.arange(200), 3)), 1)
    ov = Hs.T @ Hs
    np.fill_diagonal(ov, 0)
    assert ov.max() >= 2               # a random socket pairing has 4-cycles


@pytest.fixture(scope="module")
def mld():
    from paper_1711_01783_gb300 import build
    build.build()
    import paper_1711_01783_gb300 as m
    return m


@pytest.mark.parametrize("case", ["met", "regular"])
def test_library_construction_equals_the_oracle(mld, case):
    rng = np.random.default_rng(9)
    if case == "met":
        deg, mask = peg.met_spec(512, 0.1, 0.2, 6)
    else:
        deg, mask = _regular_spec(300, 3, 150)
    prio = rng.permutation(mask.shape[0])
    ref = peg.peg(deg, mask, prio)
    got = mld.peg_edges(deg, mask, prio)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def test_library_refuses_impossible_degrees(mld):
    deg, mask = _regular_spec(4, 3, 2)           # a VN of degree 3 with 2 checks
    with pytest.raises(mld.MldError):
        mld.peg_edges(deg, mask)
