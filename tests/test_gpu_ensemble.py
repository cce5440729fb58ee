"""mld_graph_generate on the GPU: the generated graph is the one its host edge
list describes, and decoding on it matches the FP64 oracle on those edges."""
import numpy as np
import pytest

import oracle
from synthetic import make_workload
from synthetic.ensemble import MetGraph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mld():
    import paper_1711_01783_gb300 as m
    return m


def _metgraph(mld, rate, n, d2, seed):
    ev, ec, et, m = mld.ensemble_edges(rate, n, d2, seed)
    return MetGraph(n_vn=n, n_cn=m, edge_vn=ev, edge_cn=ec, edge_type=et, rate=rate, d2=d2, seed=seed)


@pytest.mark.parametrize("rate,d2", [(0.1, 20), (0.05, 22), (0.02, 32)])
def test_generated_graph_decodes_like_its_edge_list(mld, rate, d2):
    n, seed = 4096, 5
    gen = mld.Graph.generate(rate, n, d2, seed)
    mg = _metgraph(mld, rate, n, d2, seed)
    ref_graph = mld.Graph.from_edges(mg)
    assert gen.stats == ref_graph.stats
    w = make_workload(rate, n, 16, 0, 77, beta=0.3, graph=mg)
    L = (2.0 * w.y.astype(np.float64) / (w.sigma.astype(np.float64)[:, None] ** 2)).astype(np.float32)
    outs = []
    for g in (gen, ref_graph):
        dec = mld.Decoder(g, 16, msg_dtype="f32")
        outs.append(dec.decode(torch.from_numpy(L).cuda(), torch.from_numpy(w.s).cuda(), iters=30,
                               early_term=True, want_post=True))
    for k in ("bits", "post", "converged", "iters_used"):
        assert np.array_equal(outs[0][k].cpu().numpy(), outs[1][k].cpu().numpy()), k
    ref = oracle.decode(mg, L, w.s, iters=30, early_term=True)
    conv = outs[0]["converged"].cpu().numpy().astype(bool)
    assert np.array_equal(conv, ref["converged"].astype(bool))
    assert np.array_equal(outs[0]["iters_used"].cpu().numpy(), ref["iters_used"])
    assert np.array_equal(outs[0]["bits"].cpu().numpy()[conv], ref["bits"][conv])
    assert conv.mean() > 0.5
