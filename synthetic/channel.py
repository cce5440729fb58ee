"""Seeded channel samples for the decoder (input generator, no decoding arithmetic).

After multidimensional reconciliation the two parties see a virtual
binary-input AWGN channel (Results, "Information reconciliation for CV-QKD
system"): Bob holds bits ``x`` and sends the syndrome ``s = H x`` (Step 1 of
the Methods); Alice observes ``y = (1 - 2x) + sigma * z`` with ``z ~ N(0, 1)``.

``sigma`` is set from the reconciliation efficiency ``beta = R / C`` (Table 1
reports beta per rate).  Table 1's figures follow the Gaussian capacity
``C = 0.5 log2(1 + SNR)``; the decoder's workload uses the BIAWGN capacity
``C(sigma) = 1 - E[log2(1 + exp(-2Y/sigma^2))]`` with ``Y ~ N(1, sigma^2)``
(evaluated with Gauss-Hermite quadrature), which agrees with the Gaussian
formula to about four digits at these SNRs.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .ensemble import MetGraph, preset_graph


def awgn_capacity(snr):
    """Gaussian-input capacity in bit per channel use."""
    return 0.5 * np.log2(1.0 + np.asarray(snr, dtype=np.float64))


def biawgn_capacity(sigma: float, nodes: int = 200) -> float:
    """Capacity of the binary-input AWGN channel with unit amplitude."""
    t, w = np.polynomial.hermite.hermgauss(nodes)
    y = 1.0 + np.sqrt(2.0) * sigma * t
    z = 2.0 * y / (sigma * sigma)
    f = np.logaddexp(0.0, -z) / np.log(2.0)
    return float(1.0 - np.dot(w, f) / np.sqrt(np.pi))


def sigma_for_beta(rate: float, beta: float = 0.90, capacity: str = "biawgn") -> float:
    """Noise standard deviation at which ``rate / C(sigma) == beta``."""
    target = rate / beta
    if not 0.0 < target < 1.0:
        raise ValueError("rate / beta must lie in (0, 1)")
    if capacity == "awgn":
        return float(1.0 / np.sqrt(2.0 ** (2.0 * target) - 1.0))
    if capacity != "biawgn":
        raise ValueError(capacity)
    lo, hi = 1e-2, 1e3          # capacity decreases in sigma
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if biawgn_capacity(mid) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _rng(seed: int, b: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(b)]))


def random_bits(batch: int, n: int, seed: int) -> np.ndarray:
    """Bob's bits, uint8 [batch, n]; codeword b draws from its own stream."""
    x = np.empty((batch, n), dtype=np.uint8)
    for b in range(batch):
        x[b] = _rng(seed, b).integers(0, 2, size=n, dtype=np.uint8)
    return x


def bob_syndrome(graph: MetGraph, x: np.ndarray) -> np.ndarray:
    """Bob's syndrome ``s = H x (mod 2)``, uint8 [batch, m] (sender side)."""
    x = np.atleast_2d(x)
    s = np.zeros((x.shape[0], graph.n_cn), dtype=np.uint8)
    ev = graph.edge_vn.astype(np.int64)
    ec = graph.edge_cn.astype(np.int64)
    for b in range(x.shape[0]):
        counts = np.bincount(ec, weights=x[b, ev].astype(np.float64),
                             minlength=graph.n_cn)
        s[b] = (counts.astype(np.int64) & 1).astype(np.uint8)
    return s


def biawgn_observe(x: np.ndarray, sigma, seed: int) -> np.ndarray:
    """Alice's observation ``y = (1 - 2x) + sigma z`` as float32 [batch, n]."""
    x = np.atleast_2d(x)
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (x.shape[0],))
    y = np.empty(x.shape, dtype=np.float32)
    for b in range(x.shape[0]):
        z = _rng(seed + 7919, b).standard_normal(x.shape[1])
        y[b] = (1.0 - 2.0 * x[b].astype(np.float64) + sig[b] * z).astype(np.float32)
    return y


@dataclass
class Workload:
    graph: MetGraph
    x: np.ndarray        # uint8 [B, n]
    s: np.ndarray        # uint8 [B, m]
    y: np.ndarray        # float32 [B, n]
    sigma: np.ndarray    # float32 [B]
    rate: float
    beta: float
    seed: int


def make_workload(rate: float, n: int, batch: int, graph_seed: int,
                  data_seed: int, beta: float = 0.90, sigma: float | None = None,
                  graph: MetGraph | None = None) -> Workload:
    """Graph, bits, syndromes and observations for one decoding batch."""
    g = graph if graph is not None else preset_graph(rate, n, graph_seed)
    sig = sigma_for_beta(rate, beta) if sigma is None else float(sigma)
    x = random_bits(batch, g.n_vn, data_seed)
    s = bob_syndrome(g, x)
    y = biawgn_observe(x, sig, data_seed)
    return Workload(graph=g, x=x, s=s, y=y,
                    sigma=np.full(batch, sig, dtype=np.float32),
                    rate=rate, beta=beta, seed=data_seed)


def make_uneven_workload(total: int, rates=(0.1, 0.05, 0.02), lengths=(2 ** 16, 2 ** 18, 10 ** 6),
                         seed: int = 3, beta: float = 0.90, graph_seed: int = 40):
    """Codewords whose (rate, length) pair is drawn uniformly per codeword.

    Returns a list of groups ``(rate, n, Workload)``, one per pair that was
    drawn, each with its own graph (seed graph_seed + pair index) and the
    sigma of its rate at efficiency ``beta``.
    """
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), int(total)]))
    pairs = [(r, n) for r in rates for n in lengths]
    draws = rng.integers(0, len(pairs), size=total)
    groups = []
    for k, (r, n) in enumerate(pairs):
        b = int((draws == k).sum())
        if b == 0:
            continue
        wl = make_workload(r, n, b, graph_seed + k, 5000 + 100 * k, beta=beta)
        groups.append((r, n, wl))
    return groups
