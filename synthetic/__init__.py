"""Seeded synthetic inputs for the MET-LDPC decoder and its oracle.

This module is shared by the CUDA decoder's tests/benchmark and by the FP64
oracle's tests.  It holds no belief-propagation arithmetic: it only builds
the workload the decoder is given.

* :mod:`synthetic.ensemble` -- a seeded multi-edge-type (MET) LDPC Tanner
  graph of the shape used for continuous-variable QKD reconciliation
  (core variable nodes of high degree, one degree-1 variable node per
  type-2 check), as edge arrays.
* :mod:`synthetic.channel` -- Bob's random string ``x``, his syndrome
  ``s = H x`` (the sender's side of the protocol, Step 1 of the paper's
  Methods), and Alice's binary-input AWGN observation ``y = (1-2x) + sigma*z``,
  with ``sigma`` solved from a target reconciliation efficiency ``beta``.
* :mod:`synthetic.layers` -- a grouping of the checks into layers of checks
  that share no VN of degree >= 2, which fixes the check order of the layered
  (serial) schedule.
"""
from .ensemble import (MetGraph, met_ensemble, RATE_PRESETS, preset_graph, met_ensemble_layered,
                       preset_graph_layered)
from .channel import (biawgn_capacity, awgn_capacity, sigma_for_beta,
                      random_bits, bob_syndrome, biawgn_observe, Workload,
                      make_workload, make_uneven_workload)
from .layers import check_layers, layer_order

__all__ = [
    "MetGraph", "met_ensemble", "RATE_PRESETS", "preset_graph", "met_ensemble_layered", "preset_graph_layered",
    "biawgn_capacity", "awgn_capacity", "sigma_for_beta", "random_bits",
    "bob_syndrome", "biawgn_observe", "Workload", "make_workload", "make_uneven_workload",
    "check_layers", "layer_order",
]
