"""Seeded multi-edge-type LDPC ensemble (input generator, no decoding arithmetic).

The paper decodes PEG-built MET-LDPC codes whose degree distributions come
from an external reference (Results, "GPU-based error correction speed";
Table 1 gives their edge and node counts).  Those matrices are not available,
so the decoder is exercised on a synthetic ensemble of the same shape:

* ``n_c`` core variable nodes (VNs).  Each has 2 (the first 40 %) or 3
  (the rest) type-1 edges to ``m1 = n_c - R n`` type-1 checks, and ``d2``
  type-2 edges to the ``m2 = n - n_c`` type-2 checks.
* ``m2`` degree-1 VNs; degree-1 VN ``j`` attaches to type-2 check ``j``
  (before relabelling).  Table 1 of the paper shows the same split of
  "updated" (degree > 1) and "ignored" (degree 1) VNs.
* Edges of each type are placed by a seeded socket permutation: the check
  sockets of a type are dealt as evenly as possible (each check gets
  ``floor(E/m)`` or ``ceil(E/m)``), shuffled, and paired with the VN sockets
  in order.  A repeated (VN, check) pair is re-paired by swapping its check
  socket with a uniformly drawn socket of the same type until none is left.
* Finally VN and check labels are shuffled, so that the natural order mixes
  core and degree-1 nodes as a real code would.

The number of checks is ``m = m1 + m2 = n - R n`` (the rate relation
``R = (n - m)/n`` of the Methods section).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Per-rate shape of the ensemble: fraction of core VNs and type-2 edges per
# core VN.
RATE_PRESETS = {
    0.1: dict(core_frac=0.20, d2=20),
    0.05: dict(core_frac=0.12, d2=22),
    0.02: dict(core_frac=0.06, d2=32),
}

EDGE_T1 = 0       # core VN -- type-1 check
EDGE_T2 = 1       # core VN -- type-2 check
EDGE_T2_DEG1 = 2  # degree-1 VN -- type-2 check


@dataclass
class MetGraph:
    """Tanner graph as edge arrays, in natural (relabelled) node numbering."""
    n_vn: int
    n_cn: int
    edge_vn: np.ndarray      # int32 [E]
    edge_cn: np.ndarray      # int32 [E]
    edge_type: np.ndarray    # uint8 [E], EDGE_T1 / EDGE_T2 / EDGE_T2_DEG1
    rate: float = 0.0
    n_core: int = 0
    m1: int = 0
    m2: int = 0
    d2: int = 0
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.edge_vn.shape[0])

    def vn_degree(self) -> np.ndarray:
        return np.bincount(self.edge_vn, minlength=self.n_vn)

    def cn_degree(self) -> np.ndarray:
        return np.bincount(self.edge_cn, minlength=self.n_cn)


def _deal(n_sockets: int, n_checks: int) -> np.ndarray:
    """Check label per socket, each check getting floor or ceil of the mean."""
    base, extra = divmod(n_sockets, n_checks)
    counts = np.full(n_checks, base, dtype=np.int64)
    counts[:extra] += 1
    return np.repeat(np.arange(n_checks, dtype=np.int64), counts)


def _repair_multi_edges(v: np.ndarray, c: np.ndarray, n_checks: int,
                        rng: np.random.Generator) -> np.ndarray:
    """Swap check sockets until no (v, c) pair repeats within this edge type."""
    c = c.copy()
    for _ in range(10000):
        key = v.astype(np.int64) * n_checks + c
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(key.shape[0], dtype=bool)
        dup[order[1:]] = ks[1:] == ks[:-1]
        idx = np.nonzero(dup)[0]
        if idx.size == 0:
            return c
        others = rng.integers(0, c.shape[0], size=idx.size)
        for i, j in zip(idx.tolist(), others.tolist()):
            c[i], c[j] = c[j], c[i]
    raise RuntimeError("multi-edge re-pairing did not finish")


def met_ensemble(n: int, rate: float, core_frac: float, d2: int, seed: int,
                 frac_two: float = 0.4, relabel: bool = True) -> MetGraph:
    """Build the seeded MET ensemble described in the module docstring."""
    n_c = int(round(core_frac * n))
    m2 = n - n_c
    k = int(round(rate * n))
    m1 = n_c - k
    if n_c < 1 or m1 < 1 or m2 < 1 or d2 < 1:
        raise ValueError(f"degenerate ensemble n={n} rate={rate} core_frac={core_frac}")
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), int(n), int(d2)]))

    # type-1 edges: 2 sockets for the first 40 % of core VNs, 3 for the rest
    n_two = int(round(frac_two * n_c))
    deg_t1 = np.full(n_c, 3, dtype=np.int64)
    deg_t1[:n_two] = 2
    v1 = np.repeat(np.arange(n_c, dtype=np.int64), deg_t1)
    c1 = rng.permutation(_deal(v1.shape[0], m1))
    c1 = _repair_multi_edges(v1, c1, m1, rng)

    # type-2 edges from core VNs
    v2 = np.repeat(np.arange(n_c, dtype=np.int64), d2)
    c2 = rng.permutation(_deal(v2.shape[0], m2))
    c2 = _repair_multi_edges(v2, c2, m2, rng)

    # degree-1 VN n_c + j <-> type-2 check j
    v3 = n_c + np.arange(m2, dtype=np.int64)
    c3 = np.arange(m2, dtype=np.int64)

    ev = np.concatenate([v1, v2, v3])
    ec = np.concatenate([c1, m1 + c2, m1 + c3])
    et = np.concatenate([np.full(v1.shape[0], EDGE_T1, np.uint8),
                         np.full(v2.shape[0], EDGE_T2, np.uint8),
                         np.full(v3.shape[0], EDGE_T2_DEG1, np.uint8)])
    m = m1 + m2
    if relabel:
        vlab = rng.permutation(n)
        clab = rng.permutation(m)
        ev = vlab[ev]
        ec = clab[ec]
    order = np.lexsort((ev, ec))
    return MetGraph(n_vn=n, n_cn=m,
                    edge_vn=np.ascontiguousarray(ev[order], dtype=np.int32),
                    edge_cn=np.ascontiguousarray(ec[order], dtype=np.int32),
                    edge_type=np.ascontiguousarray(et[order]),
                    rate=rate, n_core=n_c, m1=m1, m2=m2, d2=d2, seed=seed,
                    meta=dict(core_frac=core_frac, frac_two=frac_two))


def _split(total: int, weights) -> np.ndarray:
    """Integers proportional to weights summing to total (largest remainder),
    each at least 1."""
    w = np.asarray(weights, dtype=np.float64)
    raw = total * w / w.sum()
    out = np.maximum(np.floor(raw).astype(np.int64), 1)
    rest = total - out.sum()
    order = np.argsort(-(raw - np.floor(raw)), kind="stable")
    for i in range(int(rest)):
        out[order[i % len(out)]] += 1
    return out


def met_ensemble_layered(n: int, rate: float, core_frac: float, d2: int, seed: int,
                         frac_two: float = 0.4) -> MetGraph:
    """The same family with layer structure, as codes meant for layered
    decoding are built: the type-2 checks form d2 groups of equal size and
    the k-th type-2 edge of every core VN goes to group k; the type-1 checks
    form three groups (sized in proportion to their edges) and the j-th
    type-1 edge of a core VN goes to group j.  Inside a group the sockets are
    dealt evenly and shuffled as in met_ensemble, so the degree distribution
    is the same; a group holds at most one edge of each core VN, so it is a
    layer (no repeated pairs arise either).  meta["layer_of_check"] gives
    each check's group: the type-2 groups are layers 0 .. d2-1, the type-1
    groups layers d2 .. d2+2."""
    n_c = int(round(core_frac * n))
    m2 = n - n_c
    m1 = n_c - int(round(rate * n))
    if n_c < 1 or m1 < 3 or m2 < d2 or d2 < 1:
        raise ValueError(f"degenerate ensemble n={n} rate={rate} core_frac={core_frac}")
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), int(n), int(d2), 2]))
    n_two = int(round(frac_two * n_c))
    members1 = [np.arange(n_c), np.arange(n_c), np.arange(n_two, n_c)]
    sizes1 = _split(m1, [len(mb) for mb in members1])
    sizes2 = _split(m2, np.ones(d2))
    evs, ecs, ets = [], [], []
    layer = np.zeros(m1 + m2, dtype=np.int32)
    base = 0
    for j, vs in enumerate(members1):
        evs.append(vs)
        ecs.append(base + rng.permutation(_deal(vs.shape[0], int(sizes1[j]))))
        ets.append(np.full(vs.shape[0], EDGE_T1, np.uint8))
        layer[base:base + sizes1[j]] = d2 + j
        base += int(sizes1[j])
    for k in range(d2):
        vs = np.arange(n_c)
        evs.append(vs)
        ecs.append(base + rng.permutation(_deal(n_c, int(sizes2[k]))))
        ets.append(np.full(n_c, EDGE_T2, np.uint8))
        layer[base:base + sizes2[k]] = k
        base += int(sizes2[k])
    # degree-1 VN n_c + j <-> type-2 check m1 + j
    evs.append(n_c + np.arange(m2))
    ecs.append(m1 + np.arange(m2))
    ets.append(np.full(m2, EDGE_T2_DEG1, np.uint8))
    ev, ec, et = np.concatenate(evs), np.concatenate(ecs), np.concatenate(ets)
    m = m1 + m2
    vlab = rng.permutation(n)
    clab = rng.permutation(m)
    ev, ec = vlab[ev], clab[ec]
    lay = np.zeros(m, dtype=np.int32)
    lay[clab] = layer
    order = np.lexsort((ev, ec))
    return MetGraph(n_vn=n, n_cn=m,
                    edge_vn=np.ascontiguousarray(ev[order], dtype=np.int32),
                    edge_cn=np.ascontiguousarray(ec[order], dtype=np.int32),
                    edge_type=np.ascontiguousarray(et[order]),
                    rate=rate, n_core=n_c, m1=m1, m2=m2, d2=d2, seed=seed,
                    meta=dict(core_frac=core_frac, frac_two=frac_two, layer_of_check=lay, n_layers=d2 + 3))


def preset_graph_layered(rate: float, n: int, seed: int) -> MetGraph:
    """The layer-structured ensemble for one of the three code rates."""
    p = RATE_PRESETS[rate]
    return met_ensemble_layered(n, rate, p["core_frac"], p["d2"], seed)


def preset_graph(rate: float, n: int, seed: int) -> MetGraph:
    """The ensemble for one of the three code rates (0.1, 0.05, 0.02)."""
    p = RATE_PRESETS[rate]
    return met_ensemble(n, rate, p["core_frac"], p["d2"], seed)
