"""Check layers for the layered (serial) schedule of belief propagation.

Input generation only, no decoding arithmetic.  The layered schedule
updates the checks one after another in a fixed order, each check seeing the
messages its predecessors in the same iteration have just sent.  Checks that
share no variable node of degree >= 2 can be updated in either order with the
same result (a degree-1 VN has a single check, so it never links two checks),
so a serial order can be grouped into *layers* of such checks, and a whole
layer can be updated at once.

``check_layers`` builds one such grouping: the checks are split by shape
(number of edges to VNs of degree >= 2, number of degree-1 VNs); each shape is
split by first fit in check-index order into layers whose checks share no VN
of degree >= 2; layers are numbered shape after shape, shapes in ascending
order.  ``layer_order`` is the serial check order the layers stand for.
"""
from __future__ import annotations

import numpy as np


def check_layers(graph) -> tuple[np.ndarray, int]:
    """Layer index of every check (int32 [n_cn]) and the number of layers."""
    ev = np.asarray(graph.edge_vn, dtype=np.int64)
    ec = np.asarray(graph.edge_cn, dtype=np.int64)
    n_vn, n_cn = int(graph.n_vn), int(graph.n_cn)
    vdeg = np.bincount(ev, minlength=n_vn)
    core = vdeg[ev] >= 2
    dc = np.bincount(ec[core], minlength=n_cn)
    dd = np.bincount(ec[~core], minlength=n_cn)
    order = np.argsort(ec, kind="stable")
    ptr = np.zeros(n_cn + 1, dtype=np.int64)
    np.cumsum(np.bincount(ec, minlength=n_cn), out=ptr[1:])
    ev_s = ev[order].tolist()
    core_s = core[order].tolist()
    ptr_l = ptr.tolist()
    layer = np.zeros(n_cn, dtype=np.int32)
    base = 0
    for shape in sorted(set(zip(dc.tolist(), dd.tolist()))):
        checks = np.nonzero((dc == shape[0]) & (dd == shape[1]))[0].tolist()
        used = {}          # VN -> bit mask of the layers (of this shape) holding one of its checks
        top = 0
        for c in checks:
            vs = [ev_s[k] for k in range(ptr_l[c], ptr_l[c + 1]) if core_s[k]]
            m = 0
            for v in vs:
                m |= used.get(v, 0)
            L = 0
            while (m >> L) & 1:
                L += 1
            bit = 1 << L
            for v in vs:
                used[v] = used.get(v, 0) | bit
            layer[c] = base + L
            top = max(top, L + 1)
        base += top
    return layer, base


def layer_order(layer_of_check: np.ndarray) -> np.ndarray:
    """Serial check order of a layering: by layer, then by check index."""
    lay = np.asarray(layer_of_check, dtype=np.int64)
    return np.lexsort((np.arange(lay.shape[0]), lay)).astype(np.int32)
