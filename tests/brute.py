"""Brute-force decoders and tiny test codes used to pin the FP64 oracle.

Everything here is exhaustive enumeration over all 2^n words, written from
the definitions (bitwise MAP over the coset {x : H x = s}, block ML) and
independent of the oracle's message-passing code.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np


def graph_from_edges(n_vn: int, n_cn: int, edges) -> SimpleNamespace:
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    return SimpleNamespace(n_vn=n_vn, n_cn=n_cn,
                           edge_vn=edges[:, 0].astype(np.int32),
                           edge_cn=edges[:, 1].astype(np.int32))


def parity_matrix(g) -> np.ndarray:
    H = np.zeros((g.n_cn, g.n_vn), dtype=np.uint8)
    H[g.edge_cn, g.edge_vn] ^= 1
    return H


def all_words(n: int) -> np.ndarray:
    idx = np.arange(1 << n, dtype=np.int64)
    return ((idx[:, None] >> np.arange(n)) & 1).astype(np.uint8)


def coset_mask(H: np.ndarray, s: np.ndarray, words: np.ndarray) -> np.ndarray:
    return np.all((words.astype(np.int64) @ H.T.astype(np.int64)) % 2 == s[None, :], axis=1)


def map_llr(H: np.ndarray, s: np.ndarray, llr: np.ndarray) -> np.ndarray:
    """Bitwise MAP LLR ln P(x_v=0 | y, Hx=s)/P(x_v=1 | y, Hx=s).

    With L = ln p(0)/p(1), the channel likelihood of word x is proportional
    to exp(-sum_v x_v L_v).
    """
    n = H.shape[1]
    W = all_words(n)
    W = W[coset_mask(H, s, W)]
    logw = -(W.astype(np.float64) @ llr.astype(np.float64))
    out = np.empty(n)
    for v in range(n):
        a = logw[W[:, v] == 0]
        b = logw[W[:, v] == 1]
        out[v] = np.logaddexp.reduce(a) - np.logaddexp.reduce(b)
    return out


def ml_decode(H: np.ndarray, s: np.ndarray, llr: np.ndarray) -> np.ndarray:
    """Block maximum-likelihood word in the coset {x : H x = s}."""
    n = H.shape[1]
    W = all_words(n)
    W = W[coset_mask(H, s, W)]
    score = -(W.astype(np.float64) @ llr.astype(np.float64))
    return W[int(np.argmax(score))]


def random_tree_code(rng: np.random.Generator, n_target: int):
    """A cycle-free Tanner graph: every check has degree >= 2, VNs <= n_target."""
    edges = []
    n_vn, n_cn = 1, 0
    while n_vn < n_target:
        # attach a new check below a random existing VN, with 1..3 new VNs
        parent = int(rng.integers(0, n_vn))
        k = int(min(rng.integers(1, 4), n_target - n_vn))
        c = n_cn
        n_cn += 1
        edges.append((parent, c))
        for _ in range(k):
            edges.append((n_vn, c))
            n_vn += 1
        # sometimes hang an extra VN below an existing check (keeps it a tree)
        if n_vn < n_target and n_cn > 0 and rng.random() < 0.3:
            edges.append((n_vn, int(rng.integers(0, n_cn))))
            n_vn += 1
    return graph_from_edges(n_vn, n_cn, edges)


def random_code(rng: np.random.Generator, n: int, m: int, col_w: int = 3):
    """Random sparse H (each VN in col_w distinct checks; cycles allowed)."""
    edges = []
    for v in range(n):
        for c in rng.choice(m, size=min(col_w, m), replace=False):
            edges.append((v, int(c)))
    return graph_from_edges(n, m, edges)


def tanh_rule(llr_others: np.ndarray, s: int) -> float:
    """Textbook check-node rule: (1-2s) 2 atanh(prod tanh(L/2))."""
    return (1 - 2 * s) * 2.0 * np.arctanh(np.prod(np.tanh(llr_others / 2.0)))
