"""Batched MET-LDPC belief-propagation decoder for GB300 (sm_103a).

Thin ctypes binding over ``libmetldpc.so`` (C ABI in ``include/metldpc.h``):
argument marshalling only; every decoding step runs in the library's CUDA
kernels.  Device tensors (torch, CUDA) are passed as device pointers on the
current torch stream; numpy arrays or CPU tensors go through the library's
host-staging path and the call waits for the stream before returning.

The library must have been built (``python -m paper_1711_01783_gb300.build``
or ``__graft_entry__.build()``); the first call into the package raises
ImportError if it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmetldpc.so")

MLD_OK = 0
MLD_EINVAL, MLD_ENOMEM, MLD_ECUDA, MLD_ETIMEOUT, MLD_EGRAPH = -1, -2, -3, -4, -5
MLD_MSG_F32, MLD_MSG_F16 = 0, 1
MLD_EARLY_TERM, MLD_DEVICE_PTRS = 0x1, 0x2
MLD_VN_GATHER, MLD_VN_ACCUMULATE = 0, 1
MLD_SCHED_FLOODING, MLD_SCHED_LAYERED = 0, 1
MLD_CHECK_SUM_PRODUCT, MLD_CHECK_MIN_SUM = 0, 1
MLD_STAGE_DIRECT, MLD_STAGE_BULK, MLD_STAGE_BULK_LSU = 0, 1, 2

# Offset (nats) of offset min-sum on the rate-0.1 ensemble: the smallest of
# {0.3, 0.4, 0.5, 0.7, 1.0} that matched sum-product's frame error rate (0 of
# 64 frames, n = 4096) at beta = 0.30.
DEFAULT_MS_OFFSET = 0.7

_STATUS = {MLD_EINVAL: "MLD_EINVAL", MLD_ENOMEM: "MLD_ENOMEM", MLD_ECUDA: "MLD_ECUDA",
           MLD_ETIMEOUT: "MLD_ETIMEOUT", MLD_EGRAPH: "MLD_EGRAPH"}

# Every symbol include/metldpc.h declares.
EXPORTS = ("mld_last_error", "mld_version", "mld_graph_create", "mld_graph_destroy",
           "mld_graph_stats_get", "mld_decoder_create", "mld_decoder_destroy", "mld_decode",
           "mld_decode_y", "mld_decode_status", "mld_decoder_test_stall", "mld_decoder_timing_enable",
           "mld_decoder_timing_read", "mld_decode_noalloc", "mld_plan_create", "mld_plan_launch",
           "mld_plan_stats", "mld_plan_destroy", "mld_decode_multi", "mld_wbp_forward", "mld_wbp_backward",
           "mld_tape_destroy", "mld_phi_eval", "mld_ensemble_size", "mld_ensemble_edges",
           "mld_graph_generate", "mld_graph_set_layers", "mld_graph_layers_get", "mld_md_bob", "mld_md_alice", "mld_peg_edges", "mld_graph_index_arrays")


class MldError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class GraphStats(ctypes.Structure):
    _fields_ = [("n_vn", ctypes.c_int32), ("n_cn", ctypes.c_int32), ("n_edges", ctypes.c_int64),
                ("n_core", ctypes.c_int32), ("n_deg1", ctypes.c_int32), ("e_core", ctypes.c_int64),
                ("max_check_deg", ctypes.c_int32), ("max_vn_deg", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("msg_dtype", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("lmax", ctypes.c_float), ("slab_width", ctypes.c_int32),
                ("vn_update", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("check_rule", ctypes.c_int32), ("ms_offset", ctypes.c_float),
                ("checked", ctypes.c_int32), ("staging", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 6)]


class IndexArrays(ctypes.Structure):
    _fields_ = [(f, ctypes.c_void_p) for f in ("cptr", "col", "dptr", "vptr", "vedge", "unit", "cint")] + \
               [(f"n_{f}", ctypes.c_int64) for f in ("cptr", "col", "dptr", "vptr", "vedge", "unit", "cint")]


class Timing(ctypes.Structure):
    _fields_ = [("check_ms", ctypes.c_double), ("var_ms", ctypes.c_double),
                ("syndrome_ms", ctypes.c_double), ("layout_ms", ctypes.c_double),
                ("check_launches", ctypes.c_int64), ("var_launches", ctypes.c_int64),
                ("syndrome_launches", ctypes.c_int64), ("layout_launches", ctypes.c_int64),
                ("check_timed", ctypes.c_int64), ("var_timed", ctypes.c_int64),
                ("syndrome_timed", ctypes.c_int64), ("layout_timed", ctypes.c_int64)]


class Job(ctypes.Structure):
    _fields_ = [("decoder", ctypes.c_void_p), ("inp", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("syndrome", ctypes.c_void_p), ("batch", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("bits_out", ctypes.c_void_p), ("post_out", ctypes.c_void_p),
                ("converged", ctypes.c_void_p), ("iters_used", ctypes.c_void_p)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_1711_01783_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U32, F = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_float
    sig = {
        "mld_last_error": (ctypes.c_char_p, []),
        "mld_version": (ctypes.c_char_p, []),
        "mld_graph_create": (ctypes.c_int, [P, P, P, I64, I32, I32, ctypes.POINTER(P)]),
        "mld_graph_destroy": (ctypes.c_int, [P]),
        "mld_ensemble_size": (ctypes.c_int, [ctypes.c_double, I32, I32, ctypes.c_double,
                                             ctypes.POINTER(I64), ctypes.POINTER(I32)]),
        "mld_ensemble_edges": (ctypes.c_int, [ctypes.c_double, I32, I32, ctypes.c_double, ctypes.c_uint64,
                                              P, P, P, I64]),
        "mld_graph_generate": (ctypes.c_int, [ctypes.c_double, I32, I32, ctypes.c_uint64, ctypes.POINTER(P)]),
        "mld_graph_stats_get": (ctypes.c_int, [P, ctypes.POINTER(GraphStats)]),
        "mld_graph_set_layers": (ctypes.c_int, [P, P, I32]),
        "mld_graph_layers_get": (ctypes.c_int, [P, P, ctypes.POINTER(I32)]),
        "mld_decoder_create": (ctypes.c_int, [P, ctypes.POINTER(Opts), ctypes.POINTER(P)]),
        "mld_decoder_destroy": (ctypes.c_int, [P]),
        "mld_decode": (ctypes.c_int, [P, P, P, I32, I32, U32, P, P, P, P, P]),
        "mld_decode_y": (ctypes.c_int, [P, P, P, P, I32, I32, U32, P, P, P, P, P]),
        "mld_decode_status": (ctypes.c_int, [P]),
        "mld_decoder_test_stall": (ctypes.c_int, [P, ctypes.c_int32]),
        "mld_decoder_timing_enable": (ctypes.c_int, [P, ctypes.c_int]),
        "mld_decoder_timing_read": (ctypes.c_int, [P, ctypes.POINTER(Timing)]),
        "mld_decode_noalloc": (ctypes.c_int, [P, I32, P, P, I32, I32, U32, P, P, P, P, P]),
        "mld_plan_create": (ctypes.c_int, [P, I32, U32, ctypes.POINTER(P)]),
        "mld_plan_launch": (ctypes.c_int, [P, P]),
        "mld_plan_stats": (ctypes.c_int, [P, ctypes.POINTER(I64)]),
        "mld_plan_destroy": (ctypes.c_int, [P]),
        "mld_decode_multi": (ctypes.c_int, [P, I32, U32, P]),
        "mld_wbp_forward": (ctypes.c_int, [P, P, P, I32, P, I32, I32, I32, P, ctypes.POINTER(P), P]),
        "mld_wbp_backward": (ctypes.c_int, [P, P, P, P, P]),
        "mld_tape_destroy": (ctypes.c_int, [P]),
        "mld_phi_eval": (ctypes.c_int, [I32, P, P, I64, P]),
        "mld_md_bob": (ctypes.c_int, [P, P, I64, P, P, P]),
        "mld_peg_edges": (ctypes.c_int, [I32, I32, P, I32, P, P, I64, P, P, P, ctypes.POINTER(I64)]),
        "mld_graph_index_arrays": (ctypes.c_int, [P, ctypes.POINTER(IndexArrays)]),
        "mld_md_alice": (ctypes.c_int, [P, P, P, P, I32, I64, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library; raises ImportError if it has not been built."""
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def version() -> str:
    return lib().mld_version().decode()


def _check(status: int):
    if status != MLD_OK:
        raise MldError(status, lib().mld_last_error().decode(errors="replace"))


def _torch():
    import torch
    return torch


def _is_cuda_tensor(x) -> bool:
    return getattr(x, "is_cuda", False)


def _stream_handle(stream) -> ctypes.c_void_p:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


# core-VN fraction of the ensemble per code rate (mld_graph_generate's table)
ENSEMBLE_CORE_FRAC = {0.1: 0.20, 0.05: 0.12, 0.02: 0.06}


def ensemble_edges(rate: float, n: int, d2: int, seed: int, core_frac: float | None = None):
    """The library's seeded MET ensemble on the host (mld_ensemble_edges).

    Returns (edge_vn int32, edge_cn int32, edge_type uint8, n_cn); no GPU is
    needed.  ``core_frac`` defaults to the rate's entry of ENSEMBLE_CORE_FRAC.
    """
    cf = ENSEMBLE_CORE_FRAC[rate] if core_frac is None else float(core_frac)
    e, m = ctypes.c_int64(), ctypes.c_int32()
    _check(lib().mld_ensemble_size(float(rate), int(n), int(d2), cf, ctypes.byref(e), ctypes.byref(m)))
    ev = np.empty(e.value, np.int32)
    ec = np.empty(e.value, np.int32)
    et = np.empty(e.value, np.uint8)
    _check(lib().mld_ensemble_edges(float(rate), int(n), int(d2), cf, int(seed), _ptr(ev), _ptr(ec), _ptr(et),
                                    e.value))
    return ev, ec, et, int(m.value)


def peg_edges(deg, mask, prio=None):
    """Progressive-edge-growth edge list (mld_peg_edges, host only).

    deg: int [n_types, n_vn] edges per type and VN; mask: int [n_cn] (bit t:
    the check accepts type t); prio: int [n_cn] tie-break priorities or None.
    Returns (edge_vn int32, edge_cn int32, edge_type uint8) in placement order.
    """
    d = np.ascontiguousarray(deg, dtype=np.int32)
    if d.ndim != 2:
        raise ValueError("deg must be [n_types, n_vn]")
    m = np.ascontiguousarray(mask, dtype=np.uint32)
    p = None if prio is None else np.ascontiguousarray(prio, dtype=np.int32)
    if p is not None and p.shape != m.shape:
        raise ValueError("prio must be [n_cn]")
    total = int(d.astype(np.int64).sum())
    ev = np.empty(total, np.int32)
    ec = np.empty(total, np.int32)
    et = np.empty(total, np.uint8)
    k = ctypes.c_int64()
    _check(lib().mld_peg_edges(d.shape[1], d.shape[0], _ptr(d), m.shape[0], _ptr(m), _ptr(p), total,
                               _ptr(ev), _ptr(ec), _ptr(et), ctypes.byref(k)))
    return ev[:k.value], ec[:k.value], et[:k.value]


class Graph:
    """Tanner graph uploaded to the current CUDA device (mld_graph_create)."""

    def __init__(self, edge_vn, edge_cn, n_vn: int, n_cn: int, edge_type=None):
        import hashlib
        ev = np.ascontiguousarray(edge_vn, dtype=np.int32)
        ec = np.ascontiguousarray(edge_cn, dtype=np.int32)
        et = None if edge_type is None else np.ascontiguousarray(edge_type, dtype=np.uint8)
        if ev.shape != ec.shape or (et is not None and et.shape != ev.shape):
            raise ValueError("edge arrays differ in length")
        hsh = hashlib.sha1(np.array([n_vn, n_cn, ev.shape[0]], np.int64).tobytes())
        hsh.update(ev.tobytes())
        hsh.update(ec.tobytes())
        self.signature = hsh.hexdigest()[:16]
        h = ctypes.c_void_p()
        _check(lib().mld_graph_create(_ptr(ev), _ptr(ec), _ptr(et), ev.shape[0], int(n_vn), int(n_cn),
                                     ctypes.byref(h)))
        self._h = h
        st = GraphStats()
        _check(lib().mld_graph_stats_get(h, ctypes.byref(st)))
        self.stats = {f: getattr(st, f) for f, _ in GraphStats._fields_}
        self.n_vn, self.n_cn = int(n_vn), int(n_cn)

    @classmethod
    def generate(cls, rate: float, n: int, d2: int, seed: int):
        """The library's ensemble graph for rate 0.1 / 0.05 / 0.02 (mld_graph_generate)."""
        import hashlib
        h = ctypes.c_void_p()
        _check(lib().mld_graph_generate(float(rate), int(n), int(d2), int(seed), ctypes.byref(h)))
        self = cls.__new__(cls)
        self._h = h
        st = GraphStats()
        _check(lib().mld_graph_stats_get(h, ctypes.byref(st)))
        self.stats = {f: getattr(st, f) for f, _ in GraphStats._fields_}
        self.n_vn, self.n_cn = int(st.n_vn), int(st.n_cn)
        self.signature = hashlib.sha1(f"ensemble {rate} {n} {d2} {seed}".encode()).hexdigest()[:16]
        return self

    @classmethod
    def from_edges(cls, g):
        """From any object with n_vn, n_cn, edge_vn, edge_cn (and edge_type)."""
        return cls(g.edge_vn, g.edge_cn, g.n_vn, g.n_cn, getattr(g, "edge_type", None))

    def set_layers(self, layer_of_check=None):
        """Layering of the checks for the layered schedule (mld_graph_set_layers);
        None builds the library's default first fit."""
        if layer_of_check is None:
            _check(lib().mld_graph_set_layers(self._h, None, 0))
            return
        lay = np.ascontiguousarray(layer_of_check, dtype=np.int32)
        if lay.shape != (self.n_cn,):
            raise ValueError("layer_of_check must be [n_cn]")
        _check(lib().mld_graph_set_layers(self._h, _ptr(lay), int(lay.max(initial=-1)) + 1))

    def index_arrays(self) -> dict:
        """Device pointers and lengths of the store's index arrays
        (mld_graph_index_arrays)."""
        ia = IndexArrays()
        _check(lib().mld_graph_index_arrays(self._h, ctypes.byref(ia)))
        return {f: getattr(ia, f) for f, _ in IndexArrays._fields_}

    def layers(self):
        """(layer_of_check int32 [n_cn], n_layers) of the current layering."""
        n = ctypes.c_int32()
        out = np.empty(self.n_cn, dtype=np.int32)
        _check(lib().mld_graph_layers_get(self._h, _ptr(out), ctypes.byref(n)))
        return out, int(n.value)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().mld_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Decoder:
    """Device state for decoding up to ``max_batch`` codewords (mld_decoder_create).

    ``vn_update``: "gather" (default; deterministic variable update) or
    "accumulate" (the check update adds its messages to the next
    posteriors; fixed-iteration calls only, see mld_opts).
    ``schedule``: "flooding" (default) or "layered" (checks one layer at a
    time, see Graph.set_layers).
    ``check_rule``: "sum_product" (default) or "min_sum" (offset min-sum with
    ``ms_offset`` nats).
    ``staging``: "direct" (default), "bulk" or "bulk_lsu" (check-update
    operands staged in shared memory by bulk copies where that applies,
    posterior rows by one bulk copy each or by per-thread cp.async; see
    mld_opts)."""

    def __init__(self, graph: Graph, max_batch: int, msg_dtype: str = "f32",
                 lmax: float = 25.0, slab_width: int = 0, vn_update: str = "gather",
                 schedule: str = "flooding", check_rule: str = "sum_product",
                 ms_offset: float = DEFAULT_MS_OFFSET, checked: bool = False, staging: str = "direct"):
        o = Opts()
        o.msg_dtype = {"f32": MLD_MSG_F32, "f16": MLD_MSG_F16}[msg_dtype]
        o.max_batch = int(max_batch)
        o.lmax = float(lmax)
        o.slab_width = int(slab_width)
        o.vn_update = {"gather": MLD_VN_GATHER, "accumulate": MLD_VN_ACCUMULATE}[vn_update]
        o.schedule = {"flooding": MLD_SCHED_FLOODING, "layered": MLD_SCHED_LAYERED}[schedule]
        o.check_rule = {"sum_product": MLD_CHECK_SUM_PRODUCT, "min_sum": MLD_CHECK_MIN_SUM}[check_rule]
        o.ms_offset = float(ms_offset) if check_rule == "min_sum" else 0.0
        o.checked = 1 if checked else 0
        o.staging = {"direct": MLD_STAGE_DIRECT, "bulk": MLD_STAGE_BULK, "bulk_lsu": MLD_STAGE_BULK_LSU}[staging]
        h = ctypes.c_void_p()
        _check(lib().mld_decoder_create(graph.handle, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.graph = graph  # keeps the graph alive
        self.max_batch = int(max_batch)
        self.msg_dtype = msg_dtype

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().mld_decoder_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _outputs(self, B: int, on_device: bool, want_post: bool, out):
        n = self.graph.n_vn
        if out is not None:
            return out
        if on_device:
            torch = _torch()
            dev = torch.device("cuda", torch.cuda.current_device())
            return dict(bits=torch.empty((B, n), dtype=torch.uint8, device=dev),
                        post=torch.empty((B, n), dtype=torch.float32, device=dev) if want_post else None,
                        converged=torch.empty(B, dtype=torch.uint8, device=dev),
                        iters_used=torch.empty(B, dtype=torch.int32, device=dev))
        return dict(bits=np.empty((B, n), dtype=np.uint8),
                    post=np.empty((B, n), dtype=np.float32) if want_post else None,
                    converged=np.empty(B, dtype=np.uint8),
                    iters_used=np.empty(B, dtype=np.int32))

    def _run(self, fn, x, sigma, syndrome, iters, early_term, want_post, out, stream):
        on_dev = _is_cuda_tensor(x)
        if on_dev:
            torch = _torch()
            x = x.contiguous()
            if x.dtype != torch.float32:
                raise TypeError("soft input must be float32")
            syndrome = syndrome.contiguous().to(torch.uint8)
            if sigma is not None:
                sigma = sigma.contiguous().to(torch.float32)
        else:
            x = np.ascontiguousarray(x.numpy() if hasattr(x, "numpy") else x, dtype=np.float32)
            syndrome = np.ascontiguousarray(syndrome.numpy() if hasattr(syndrome, "numpy") else syndrome,
                                            dtype=np.uint8)
            if sigma is not None:
                sigma = np.ascontiguousarray(sigma.numpy() if hasattr(sigma, "numpy") else sigma,
                                             dtype=np.float32).reshape(-1)
        B = int(x.shape[0])
        if tuple(x.shape) != (B, self.graph.n_vn) or tuple(syndrome.shape) != (B, self.graph.n_cn):
            raise ValueError("soft input must be [B, n_vn] and syndrome [B, n_cn]")
        o = self._outputs(B, on_dev, want_post, out)
        flags = (MLD_EARLY_TERM if early_term else 0) | (MLD_DEVICE_PTRS if on_dev else 0)
        sh = _stream_handle(stream)
        args = [self._h, _ptr(x)]
        if fn is lib().mld_decode_y:
            args.append(_ptr(sigma))
        args += [_ptr(syndrome), B, int(iters), flags, _ptr(o["bits"]), _ptr(o.get("post")),
                 _ptr(o["converged"]), _ptr(o["iters_used"]), sh]
        _check(fn(*args))
        if not on_dev:
            torch = _torch()
            (stream or torch.cuda.current_stream()).synchronize()
        return o

    def decode(self, llr, syndrome, iters: int, early_term: bool = False,
               want_post: bool = False, out=None, stream=None):
        """Decode from channel LLRs [B, n]; see mld_decode."""
        return self._run(lib().mld_decode, llr, None, syndrome, iters, early_term, want_post, out, stream)

    def decode_y(self, y, sigma, syndrome, iters: int, early_term: bool = False,
                 want_post: bool = False, out=None, stream=None):
        """Decode from BIAWGN observations y [B, n] and per-codeword sigma [B]."""
        return self._run(lib().mld_decode_y, y, sigma, syndrome, iters, early_term, want_post, out, stream)

    def status(self) -> int:
        return int(lib().mld_decode_status(self._h))

    def test_stall(self, nbytes: int) -> None:
        """Timeout-path test hook (mld_decoder_test_stall)."""
        _check(lib().mld_decoder_test_stall(self._h, int(nbytes)))

    def wbp_forward(self, llr, syndrome, weights, ckpt_k: int = 5, keep_tape: bool = True, stream=None):
        """Weighted BP forward (mld_wbp_forward); returns (soft [B, n], Tape or None)."""
        torch = _torch()
        llr = llr.contiguous().to(torch.float32)
        syndrome = syndrome.contiguous().to(torch.uint8)
        w = weights.detach().contiguous().to(torch.float32)
        T, nt = int(w.shape[0]), int(w.shape[1])
        soft = torch.empty_like(llr)
        h = ctypes.c_void_p()
        _check(lib().mld_wbp_forward(self._h, _ptr(llr), _ptr(syndrome), int(llr.shape[0]), _ptr(w), nt, T,
                                     int(ckpt_k), _ptr(soft), ctypes.byref(h) if keep_tape else None,
                                     _stream_handle(stream)))
        return soft, (Tape(h, self, llr.shape, (T, nt)) if keep_tape else None)

    def timing(self, every: int):
        """Time the kernels of every N-th iteration of later decode calls (0 = off)."""
        _check(lib().mld_decoder_timing_enable(self._h, int(every)))

    def read_timing(self) -> dict:
        """Per-kernel-class device time (ms) and launch counts since the last read."""
        t = Timing()
        _check(lib().mld_decoder_timing_read(self._h, ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in Timing._fields_}


class Tape:
    """Recorded forward of weighted BP, for mld_wbp_backward."""

    def __init__(self, handle, decoder, llr_shape, w_shape):
        self._h = handle
        self.decoder = decoder
        self.llr_shape = tuple(llr_shape)
        self.w_shape = tuple(w_shape)

    def backward(self, dsoft, stream=None):
        torch = _torch()
        dsoft = dsoft.contiguous().to(torch.float32)
        dw = torch.empty(self.w_shape, dtype=torch.float32, device=dsoft.device)
        dllr = torch.empty(self.llr_shape, dtype=torch.float32, device=dsoft.device)
        _check(lib().mld_wbp_backward(self._h, _ptr(dsoft), _ptr(dw), _ptr(dllr), _stream_handle(stream)))
        return dw, dllr

    def close(self):
        if getattr(self, "_h", None):
            lib().mld_tape_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def weighted_bp(decoder, llr, syndrome, weights, ckpt_k: int = 5):
    """Differentiable weighted BP: soft posteriors [B, n] as a function of the
    channel LLRs and the weights [T, n_types] (torch.autograd)."""
    torch = _torch()

    class _WeightedBP(torch.autograd.Function):
        @staticmethod
        def forward(ctx, llr_, w_):
            soft, tape = decoder.wbp_forward(llr_, syndrome, w_, ckpt_k=ckpt_k)
            ctx.tape = tape
            return soft

        @staticmethod
        def backward(ctx, dsoft):
            dw, dllr = ctx.tape.backward(dsoft)
            ctx.tape.close()
            return dllr, dw

    return _WeightedBP.apply(llr, weights)


class Plan:
    """Several jobs (graph + batch + iteration cap) decoded by one captured
    CUDA graph (mld_plan_create / mld_plan_launch).

    ``jobs`` is a list of dicts with keys ``decoder`` (Decoder), ``y`` (CUDA
    float32 [B, n]; observations if ``sigma`` is given, else LLRs), ``sigma``
    (CUDA float32 [B] or None), ``syndrome`` (CUDA uint8 [B, m]) and
    ``max_iters``.  Outputs are allocated here and returned by ``outputs``.
    """

    def __init__(self, jobs, early_term: bool = False, want_post: bool = False):
        torch = _torch()
        self._keep = []
        self.outputs = []
        arr = (Job * max(1, len(jobs)))()
        for i, jb in enumerate(jobs):
            dec = jb["decoder"]
            y = jb["y"].contiguous()
            syn = jb["syndrome"].contiguous().to(torch.uint8)
            sig = jb.get("sigma")
            sig = sig.contiguous().to(torch.float32) if sig is not None else None
            B, n = int(y.shape[0]), dec.graph.n_vn
            o = dict(bits=torch.empty((B, n), dtype=torch.uint8, device=y.device),
                     post=torch.empty((B, n), dtype=torch.float32, device=y.device) if want_post else None,
                     converged=torch.empty(B, dtype=torch.uint8, device=y.device),
                     iters_used=torch.empty(B, dtype=torch.int32, device=y.device))
            self._keep += [dec, y, syn, sig]
            self.outputs.append(o)
            arr[i] = Job(dec.handle.value, y.data_ptr(), sig.data_ptr() if sig is not None else None,
                         syn.data_ptr(), B, int(jb["max_iters"]), o["bits"].data_ptr(),
                         o["post"].data_ptr() if o["post"] is not None else None,
                         o["converged"].data_ptr(), o["iters_used"].data_ptr())
        h = ctypes.c_void_p()
        flags = (MLD_EARLY_TERM if early_term else 0) | MLD_DEVICE_PTRS
        _check(lib().mld_plan_create(ctypes.cast(arr, ctypes.c_void_p), len(jobs), flags, ctypes.byref(h)))
        self._h = h
        n = ctypes.c_int64()
        _check(lib().mld_plan_stats(h, ctypes.byref(n)))
        self.launches = int(n.value)

    def launch(self, stream=None):
        _check(lib().mld_plan_launch(self._h, _stream_handle(stream)))
        return self.outputs

    def close(self):
        if getattr(self, "_h", None):
            lib().mld_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


def decode_noalloc(graph: Graph, llr, syndrome, iters: int, msg_dtype: str = "f32",
                   early_term: bool = False, want_post: bool = False, stream=None):
    """Decode without a decoder object and without allocating device memory
    in the library (mld_decode_noalloc).  Inputs are CUDA tensors; the output
    tensors are allocated here by torch, the library allocates nothing.

    The entry point takes device pointers only, so the inputs are checked
    here before any pointer reaches the library: both must be CUDA tensors
    on one device, ``llr`` float32 [B, n_vn] and ``syndrome`` [B, n_cn]."""
    torch = _torch()
    if not (_is_cuda_tensor(llr) and _is_cuda_tensor(syndrome)):
        raise TypeError("decode_noalloc takes CUDA tensors (device pointers only)")
    if llr.device != syndrome.device:
        raise ValueError("llr and syndrome are on different devices")
    if llr.dtype != torch.float32:
        raise TypeError("llr must be float32")
    if msg_dtype not in ("f32", "f16"):
        raise ValueError("msg_dtype must be 'f32' or 'f16'")
    if llr.dim() != 2 or tuple(llr.shape) != (llr.shape[0], graph.n_vn) \
            or tuple(syndrome.shape) != (llr.shape[0], graph.n_cn):
        raise ValueError("llr must be [B, n_vn] and syndrome [B, n_cn]")
    llr = llr.contiguous()
    syndrome = syndrome.contiguous().to(torch.uint8)
    B, n = int(llr.shape[0]), graph.n_vn
    dev = llr.device
    with torch.cuda.device(dev):
        out = dict(bits=torch.empty((B, n), dtype=torch.uint8, device=dev),
                   post=torch.empty((B, n), dtype=torch.float32, device=dev) if want_post else None,
                   converged=torch.empty(B, dtype=torch.uint8, device=dev),
                   iters_used=torch.empty(B, dtype=torch.int32, device=dev))
        flags = (MLD_EARLY_TERM if early_term else 0) | MLD_DEVICE_PTRS
        dt = {"f32": MLD_MSG_F32, "f16": MLD_MSG_F16}[msg_dtype]
        _check(lib().mld_decode_noalloc(graph.handle, dt, _ptr(llr), _ptr(syndrome), B, int(iters), flags,
                                        _ptr(out["bits"]), _ptr(out["post"]), _ptr(out["converged"]),
                                        _ptr(out["iters_used"]), _stream_handle(stream)))
    return out


def md_bob(y, bits, stream=None):
    """Bob's side of multidimensional reconciliation (mld_md_bob): CUDA float32
    y [..., 8k] and uint8 bits of the same shape -> (alpha [..., 8k], |y| [..., k])."""
    torch = _torch()
    if not (_is_cuda_tensor(y) and _is_cuda_tensor(bits)):
        raise TypeError("md_bob takes CUDA tensors")
    y = y.contiguous().to(torch.float32)
    bits = bits.contiguous().to(torch.uint8)
    if y.shape != bits.shape or y.shape[-1] % 8:
        raise ValueError("y and bits must have one shape whose last dimension is a multiple of 8")
    alpha = torch.empty_like(y)
    ynorm = torch.empty(y.shape[:-1] + (y.shape[-1] // 8,), dtype=torch.float32, device=y.device)
    _check(lib().mld_md_bob(_ptr(y), _ptr(bits), y.numel(), _ptr(alpha), _ptr(ynorm), _stream_handle(stream)))
    return alpha, ynorm


def md_alice(x, alpha, ynorm, noise_var, stream=None):
    """Alice's LLRs of Bob's bits (mld_md_alice): CUDA float32 x, alpha
    [rows, n], ynorm [rows, n/8], noise_var [rows] -> LLR [rows, n]."""
    torch = _torch()
    if not all(_is_cuda_tensor(t) for t in (x, alpha, ynorm, noise_var)):
        raise TypeError("md_alice takes CUDA tensors")
    x = x.contiguous().to(torch.float32)
    alpha = alpha.contiguous().to(torch.float32)
    ynorm = ynorm.contiguous().to(torch.float32)
    noise_var = noise_var.contiguous().to(torch.float32).reshape(-1)
    if x.dim() != 2 or alpha.shape != x.shape or x.shape[1] % 8 or tuple(ynorm.shape) != (x.shape[0], x.shape[1] // 8) \
            or noise_var.shape[0] != x.shape[0]:
        raise ValueError("x, alpha [rows, n], ynorm [rows, n/8], noise_var [rows]")
    llr = torch.empty_like(x)
    _check(lib().mld_md_alice(_ptr(x), _ptr(alpha), _ptr(ynorm), _ptr(noise_var), x.shape[0], x.shape[1],
                              _ptr(llr), _stream_handle(stream)))
    return llr


def phi(x, msg_dtype: str = "f32", stream=None):
    """Device phi(x) = -ln tanh(x/2) as used by the check update of a decoder
    with the given message storage type (float32 CUDA tensor in and out)."""
    torch = _torch()
    x = x.contiguous().to(torch.float32)
    out = torch.empty_like(x)
    dt = {"f32": MLD_MSG_F32, "f16": MLD_MSG_F16}[msg_dtype]
    _check(lib().mld_phi_eval(dt, _ptr(x), _ptr(out), x.numel(), _stream_handle(stream)))
    return out


__all__ = ["Graph", "Decoder", "Plan", "Tape", "weighted_bp", "phi", "decode_noalloc", "ensemble_edges",
           "md_bob", "md_alice", "DEFAULT_MS_OFFSET", "peg_edges",
           "ENSEMBLE_CORE_FRAC", "version", "lib", "MldError", "EXPORTS",
           "LIB_PATH", "NOALLOC_SCRATCH_BYTES"]
