"""Autotuner for the decoder: slab width and variable-update variant.

The slab width W (codewords interleaved per 128-byte line group: 8, 16, 32
or 64) trades padding against access granularity: a batch of 11 codewords
fills 69 % of a 16-wide slab but 17 % of a 64-wide one, while wider slabs
move whole 128-byte lines per graph access.  The tuner times a few decoder
iterations for every width on the actual graph and batch size, keeps the
fastest per decoded codeword, and caches the choice in a JSON file keyed by
(graph signature, batch, message type, GPU name).

``DecoderTuner`` widens the search for single-graph decoding without early
termination to the variable-update variant as well: the gather pass or the
accumulation of the new messages inside the check update (which wins with
float messages and loses with half ones on GB300), over the slab widths each
variant allows, and for half messages to the staged check update (operands
brought into shared memory by bulk copies; slower on GB300, where the
direct kernel is instruction-bound).  Plans keep the gather, so they use
``SlabWidthTuner``.
"""
from __future__ import annotations

import json
import os

WIDTHS = (8, 16, 32, 64)


class SlabWidthTuner:
    def __init__(self, cache_path: str | None = None, iters: int = 4, reps: int = 3):
        self.cache_path = cache_path
        self.iters = iters
        self.reps = reps
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)
        self.trials = {}

    def _key(self, graph, batch: int, msg_dtype: str) -> str:
        import torch
        return f"{graph.signature}|{batch}|{msg_dtype}|{torch.cuda.get_device_name()}"

    def choose(self, graph, batch: int, msg_dtype: str = "f16") -> int:
        import torch

        from . import Decoder
        key = self._key(graph, batch, msg_dtype)
        if key in self.cache:
            return int(self.cache[key]["W"])
        dev = torch.device("cuda", torch.cuda.current_device())
        llr = torch.zeros((batch, graph.n_vn), dtype=torch.float32, device=dev)
        syn = torch.zeros((batch, graph.n_cn), dtype=torch.uint8, device=dev)
        times = {}
        for W in WIDTHS:
            dec = Decoder(graph, batch, msg_dtype=msg_dtype, slab_width=W)
            dec.decode(llr, syn, self.iters)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(self.reps):
                dec.decode(llr, syn, self.iters)
            e1.record()
            torch.cuda.synchronize()
            times[W] = e0.elapsed_time(e1) / self.reps
            dec.close()
        best = min(times, key=times.get)
        self.cache[key] = {"W": best, "ms": times}
        self.trials[key] = times
        if self.cache_path:
            os.makedirs(os.path.dirname(os.path.abspath(self.cache_path)), exist_ok=True)
            with open(self.cache_path, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
        return best


class DecoderTuner(SlabWidthTuner):
    """Chooses decoder options (slab width, variable-update variant) by
    timing a few fixed iterations of each candidate on the actual graph and
    batch; cached like the slab width."""

    def _key(self, graph, batch: int, msg_dtype: str) -> str:
        return "dec|" + super()._key(graph, batch, msg_dtype)

    def candidates(self, msg_dtype: str):
        default_w = 64 if msg_dtype == "f16" else 32
        out = [dict(slab_width=w, vn_update="gather") for w in WIDTHS]
        out.append(dict(slab_width=default_w, vn_update="accumulate"))
        if msg_dtype == "f16":
            # check-update operands staged in shared memory (half, width 64)
            out += [dict(slab_width=64, vn_update="gather", staging=m) for m in ("bulk", "bulk_lsu")]
        return out

    def choose_options(self, graph, batch: int, msg_dtype: str = "f16") -> dict:
        import torch

        from . import Decoder, MldError
        key = self._key(graph, batch, msg_dtype)
        if key in self.cache:
            return dict(self.cache[key]["opts"])
        dev = torch.device("cuda", torch.cuda.current_device())
        llr = torch.zeros((batch, graph.n_vn), dtype=torch.float32, device=dev)
        syn = torch.zeros((batch, graph.n_cn), dtype=torch.uint8, device=dev)
        times = []
        for opts in self.candidates(msg_dtype):
            try:
                dec = Decoder(graph, batch, msg_dtype=msg_dtype, **opts)
            except MldError:  # a variant the graph does not allow
                continue
            dec.decode(llr, syn, self.iters)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(self.reps):
                dec.decode(llr, syn, self.iters)
            e1.record()
            torch.cuda.synchronize()
            times.append((e0.elapsed_time(e1) / self.reps, opts))
            dec.close()
        best = min(times, key=lambda t: t[0])[1]
        self.cache[key] = {"opts": best, "ms": [[t, o] for t, o in times]}
        self.trials[key] = times
        if self.cache_path:
            os.makedirs(os.path.dirname(os.path.abspath(self.cache_path)), exist_ok=True)
            with open(self.cache_path, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
        return dict(best)
