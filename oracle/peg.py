"""Progressive-edge-growth (PEG) construction of a multi-edge-type Tanner
graph, written plainly (test infrastructure; the library never imports it).

The paper's codes are built by PEG from multi-edge-type degree distributions
(Results, "GPU-based error correction speed"; Table 1).  This is the
construction as the PEG method defines it, for edges of several types:

* VN v has deg[t][v] edges of type t; check c accepts the edge types whose
  bits are set in mask[c]; prio[c] breaks ties.
* VNs are connected in order of increasing total degree (ties by index);
  a VN's edges are placed type by type (t = 0, 1, ...), one at a time.
* An edge of type t from v goes to a check that accepts t and is not yet a
  neighbour of v, chosen among those farthest from v in the graph built so
  far: if some such check cannot be reached from v, among the unreachable
  ones; otherwise among those at the largest distance.  Among these, the
  lowest current degree wins, then the lowest prio.

Distances are counted in check levels of a breadth-first search from v:
v's neighbours are level 1, the checks of their other VNs level 2, and so on.
The function returns the edges in the order they were placed.

Parity status: pinned by exact degrees, no repeated pairs, a replay of every
placement against an independent shortest-path computation, and the absence
of 4-cycles where the degrees allow it (tests/test_peg.py).
"""
from __future__ import annotations

import numpy as np


def peg(deg: np.ndarray, mask: np.ndarray, prio: np.ndarray | None = None):
    """deg: int [T, n_vn]; mask: int [n_cn] (bit t: check takes type t);
    prio: int [n_cn] or None (index order).  Returns (edge_vn, edge_cn,
    edge_type) as int arrays in placement order."""
    deg = np.asarray(deg, dtype=np.int64)
    T, n_vn = deg.shape
    mask = np.asarray(mask, dtype=np.int64)
    n_cn = mask.shape[0]
    prio = np.arange(n_cn) if prio is None else np.asarray(prio, dtype=np.int64)
    vn_adj = [[] for _ in range(n_vn)]
    cn_adj = [[] for _ in range(n_cn)]
    cdeg = [0] * n_cn
    order = sorted(range(n_vn), key=lambda v: (int(deg[:, v].sum()), v))
    ev, ec, et = [], [], []
    for v in order:
        for t in range(T):
            for _ in range(int(deg[t, v])):
                level = _levels(v, vn_adj, cn_adj, n_cn)
                allowed = [c for c in range(n_cn) if (mask[c] >> t) & 1 and c not in vn_adj[v]]
                if not allowed:
                    raise ValueError(f"no check left for an edge of type {t} of VN {v}")
                unreached = [c for c in allowed if level[c] == 0]
                if unreached:
                    cand = unreached
                else:
                    far = max(level[c] for c in allowed)
                    cand = [c for c in allowed if level[c] == far]
                c = min(cand, key=lambda k: (cdeg[k], int(prio[k])))
                vn_adj[v].append(c)
                cn_adj[c].append(v)
                cdeg[c] += 1
                ev.append(v)
                ec.append(c)
                et.append(t)
    return np.array(ev, np.int32), np.array(ec, np.int32), np.array(et, np.uint8)


def _levels(v, vn_adj, cn_adj, n_cn):
    """BFS levels of the checks from VN v (0 = not reached)."""
    level = [0] * n_cn
    seen_v = {v}
    frontier = [v]
    lv = 0
    while frontier:
        lv += 1
        new_c = []
        for u in frontier:
            for c in vn_adj[u]:
                if level[c] == 0:
                    level[c] = lv
                    new_c.append(c)
        frontier = []
        for c in new_c:
            for w in cn_adj[c]:
                if w not in seen_v:
                    seen_v.add(w)
                    frontier.append(w)
    return level


def met_spec(n: int, rate: float, core_frac: float, d2: int, frac_two: float = 0.4):
    """Degrees and check masks of the benchmark's multi-edge-type family:
    n_c core VNs with 2 (first 40 %) or 3 type-0 edges and d2 type-1 edges,
    n - n_c degree-1 VNs with one type-2 edge; m1 = n_c - rate n checks take
    type 0, m2 = n - n_c checks take types 1 and 2."""
    n_c = int(round(core_frac * n))
    m2 = n - n_c
    m1 = n_c - int(round(rate * n))
    deg = np.zeros((3, n), np.int64)
    n_two = int(round(frac_two * n_c))
    deg[0, :n_c] = 3
    deg[0, :n_two] = 2
    deg[1, :n_c] = d2
    deg[2, n_c:] = 1
    mask = np.concatenate([np.full(m1, 1), np.full(m2, 6)]).astype(np.int64)
    return deg, mask
