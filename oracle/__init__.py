"""FP64 CPU oracle for syndrome-based sum-product BP (test infrastructure).

TEST INFRASTRUCTURE ONLY: the decoder's tests, the package smoke check and
the benchmark's CPU-baseline leg use this module to check or time the CUDA
decoder.  The decoder itself never imports it, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, FP64, one codeword per
thread); see that file's header for the paper passages it follows and the
readings it takes.  This module compiles it with gcc and wraps it with ctypes.

Layered schedule (``decode_layered``): the same check and variable updates
with the checks taken one at a time in a given order.  Pinned by MAP on
cycle-free graphs, the one-sweep closed form of a repetition chain, the
order-invariance of checks that share no VN, the coset symmetry, exhaustive
ML and the noiseless limit (``tests/test_oracle_layered.py``).

Offset min-sum (``decode_ms``): the flooding decoder with the check update's
magnitude replaced by the smallest other magnitude minus an offset.  Pinned
by the exact degree-2 chain (offset 0), the single-check bound
|r_min-sum| >= |r_sum-product| with equal signs, the offset's closed form on
one check, the coset symmetry, exhaustive ML, the noiseless limit and
planted mistakes (``tests/test_oracle_minsum.py``).

Weighted BP (``wbp``): forward plus a hand-written reverse-mode gradient,
pinned by central finite differences of its own FP64 loss and by the
all-weights-one case equalling plain BP.

Parity status: plain BP is pinned by brute-force bitwise MAP on cycle-free
graphs, the single-check and repetition-chain closed forms, exhaustive ML
on small codes, the coset-symmetry invariant and the noiseless limit
(``tests/test_oracle_pins.py``).  The frame error rate of the synthetic
ensemble has no published value: parity unpinned for that figure.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LMAX = 25.0  # LLR clamp used throughout (a reading: the paper gives no constant)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` next to it (gcc -O3).

    ISO C mode (-std=c11) keeps floating-point contraction off, so the
    optimisation level does not change any result.  No -march=native: the
    oracle must compute the same bits on every host it is built on."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-D_GNU_SOURCE", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, dbl, ptr = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            lib.oracle_phi.restype = dbl
            lib.oracle_phi.argtypes = [dbl]
            lib.oracle_decode.restype = ctypes.c_int
            lib.oracle_decode.argtypes = [i32, i32, i64, ptr, ptr, i32, ptr, ptr,
                                          i32, i32, dbl, ptr, ptr, ptr, ptr, i32]
            lib.oracle_decode_layered.restype = ctypes.c_int
            lib.oracle_decode_layered.argtypes = [i32, i32, i64, ptr, ptr, ptr, i32, ptr, ptr,
                                                  i32, i32, dbl, ptr, ptr, ptr, ptr, i32]
            lib.oracle_decode_ms.restype = ctypes.c_int
            lib.oracle_decode_ms.argtypes = [i32, i32, i64, ptr, ptr, dbl, i32, ptr, ptr,
                                             i32, i32, dbl, ptr, ptr, ptr, ptr, i32]
            lib.oracle_wbp.restype = ctypes.c_int
            lib.oracle_wbp.argtypes = [i32, i32, i64, ptr, ptr, ptr, i32, i32, ptr, ptr, ptr, i32, ptr, dbl,
                                       ptr, ptr, ptr, ptr, i32]
            lib.oracle_syndrome_ok.restype = ctypes.c_int
            lib.oracle_syndrome_ok.argtypes = [i32, i32, i64, ptr, ptr, i32, ptr, ptr, ptr]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def phi(x: float) -> float:
    """phi(x) = -ln tanh(x/2) in FP64."""
    return float(_load().oracle_phi(float(x)))


def channel_llr(y: np.ndarray, sigma) -> np.ndarray:
    """Eq. 1 in LLR form for the BIAWGN observation: L = 2 y / sigma^2 (FP64)."""
    y = np.atleast_2d(np.asarray(y, dtype=np.float64))
    sig = np.asarray(sigma, dtype=np.float64).reshape(-1, 1)
    return 2.0 * y / (sig * sig)


def _edges(graph):
    ev = np.ascontiguousarray(graph.edge_vn, dtype=np.int32)
    ec = np.ascontiguousarray(graph.edge_cn, dtype=np.int32)
    return int(graph.n_vn), int(graph.n_cn), ev, ec


def decode(graph, llr: np.ndarray, syndrome: np.ndarray, iters: int,
           early_term: bool = False, lmax: float = LMAX, threads: int | None = None):
    """Flooding sum-product BP in FP64.

    ``graph`` is any object with ``n_vn``, ``n_cn``, ``edge_vn``, ``edge_cn``.
    ``llr`` is [B, n] (any float type; promoted to FP64), ``syndrome`` [B, m].
    Returns a dict with ``post`` (FP64 [B, n]), ``bits`` (uint8 [B, n]),
    ``converged`` (uint8 [B]) and ``iters_used`` (int32 [B]).
    """
    n, m, ev, ec = _edges(graph)
    L = np.ascontiguousarray(np.atleast_2d(llr), dtype=np.float64)
    S = np.ascontiguousarray(np.atleast_2d(syndrome), dtype=np.uint8)
    B = L.shape[0]
    if L.shape != (B, n) or S.shape != (B, m):
        raise ValueError("shape mismatch")
    post = np.zeros((B, n), dtype=np.float64)
    bits = np.zeros((B, n), dtype=np.uint8)
    conv = np.zeros(B, dtype=np.uint8)
    used = np.zeros(B, dtype=np.int32)
    st = _load().oracle_decode(n, m, ev.shape[0], _p(ev), _p(ec), B, _p(L), _p(S),
                               int(iters), int(bool(early_term)), float(lmax),
                               _p(post), _p(bits), _p(conv), _p(used),
                               int(threads or default_threads()))
    if st != 0:
        raise RuntimeError(f"oracle_decode failed with status {st}")
    return dict(post=post, bits=bits, converged=conv, iters_used=used)


def decode_layered(graph, llr: np.ndarray, syndrome: np.ndarray, iters: int, order,
                   early_term: bool = False, lmax: float = LMAX, threads: int | None = None):
    """Sum-product BP in FP64 with the layered (serial) schedule: the checks
    are updated one at a time in ``order`` (every check once), each from the
    latest messages.  Same inputs and outputs as :func:`decode`."""
    n, m, ev, ec = _edges(graph)
    L = np.ascontiguousarray(np.atleast_2d(llr), dtype=np.float64)
    S = np.ascontiguousarray(np.atleast_2d(syndrome), dtype=np.uint8)
    od = np.ascontiguousarray(order, dtype=np.int32)
    B = L.shape[0]
    if L.shape != (B, n) or S.shape != (B, m) or od.shape != (m,):
        raise ValueError("shape mismatch")
    post = np.zeros((B, n), dtype=np.float64)
    bits = np.zeros((B, n), dtype=np.uint8)
    conv = np.zeros(B, dtype=np.uint8)
    used = np.zeros(B, dtype=np.int32)
    st = _load().oracle_decode_layered(n, m, ev.shape[0], _p(ev), _p(ec), _p(od), B, _p(L), _p(S),
                                       int(iters), int(bool(early_term)), float(lmax),
                                       _p(post), _p(bits), _p(conv), _p(used),
                                       int(threads or default_threads()))
    if st != 0:
        raise RuntimeError(f"oracle_decode_layered failed with status {st}")
    return dict(post=post, bits=bits, converged=conv, iters_used=used)


def decode_ms(graph, llr: np.ndarray, syndrome: np.ndarray, iters: int, offset: float = 0.0,
              early_term: bool = False, lmax: float = LMAX, threads: int | None = None):
    """Offset min-sum in FP64 (flooding schedule): the check update keeps the
    sign rule and takes max(min of the other |q| - offset, 0) as magnitude.
    Same inputs and outputs as :func:`decode`."""
    n, m, ev, ec = _edges(graph)
    L = np.ascontiguousarray(np.atleast_2d(llr), dtype=np.float64)
    S = np.ascontiguousarray(np.atleast_2d(syndrome), dtype=np.uint8)
    B = L.shape[0]
    if L.shape != (B, n) or S.shape != (B, m):
        raise ValueError("shape mismatch")
    post = np.zeros((B, n), dtype=np.float64)
    bits = np.zeros((B, n), dtype=np.uint8)
    conv = np.zeros(B, dtype=np.uint8)
    used = np.zeros(B, dtype=np.int32)
    st = _load().oracle_decode_ms(n, m, ev.shape[0], _p(ev), _p(ec), float(offset), B, _p(L), _p(S),
                                  int(iters), int(bool(early_term)), float(lmax),
                                  _p(post), _p(bits), _p(conv), _p(used), int(threads or default_threads()))
    if st != 0:
        raise RuntimeError(f"oracle_decode_ms failed with status {st}")
    return dict(post=post, bits=bits, converged=conv, iters_used=used)


def decode_y(graph, y: np.ndarray, sigma, syndrome: np.ndarray, iters: int, **kw):
    """Decode from the channel observation y with per-codeword sigma."""
    return decode(graph, channel_llr(y, sigma), syndrome, iters, **kw)


def wbp(graph, llr: np.ndarray, syndrome: np.ndarray, xbits: np.ndarray, weights: np.ndarray,
        edge_type=None, lmax: float = LMAX, threads: int | None = None):
    """Weighted BP (weights [T, n_types] on the variable-to-check messages)
    with the mean-BCE loss against the true bits, and its exact gradient.

    Returns dict(loss, post [B, n], dw [T, n_types], dllr [B, n]).
    """
    n, m, ev, ec = _edges(graph)
    et = np.ascontiguousarray(graph.edge_type if edge_type is None else edge_type, dtype=np.uint8)
    W = np.ascontiguousarray(weights, dtype=np.float64)
    T, nt = W.shape
    L = np.ascontiguousarray(np.atleast_2d(llr), dtype=np.float64)
    S = np.ascontiguousarray(np.atleast_2d(syndrome), dtype=np.uint8)
    X = np.ascontiguousarray(np.atleast_2d(xbits), dtype=np.uint8)
    B = L.shape[0]
    loss = np.zeros(1)
    post = np.zeros((B, n))
    dw = np.zeros((T, nt))
    dllr = np.zeros((B, n))
    st = _load().oracle_wbp(n, m, ev.shape[0], _p(ev), _p(ec), _p(et), nt, B, _p(L), _p(S), _p(X), T,
                            _p(W), float(lmax), _p(loss), _p(post), _p(dw), _p(dllr),
                            int(threads or default_threads()))
    if st != 0:
        raise RuntimeError(f"oracle_wbp failed with status {st}")
    return dict(loss=float(loss[0]), post=post, dw=dw, dllr=dllr)


def syndrome_ok(graph, bits: np.ndarray, syndrome: np.ndarray) -> np.ndarray:
    """Per-codeword flag: H bits == syndrome (mod 2)."""
    n, m, ev, ec = _edges(graph)
    X = np.ascontiguousarray(np.atleast_2d(bits), dtype=np.uint8)
    S = np.ascontiguousarray(np.atleast_2d(syndrome), dtype=np.uint8)
    ok = np.zeros(X.shape[0], dtype=np.uint8)
    st = _load().oracle_syndrome_ok(n, m, ev.shape[0], _p(ev), _p(ec), X.shape[0],
                                    _p(X), _p(S), _p(ok))
    if st != 0:
        raise RuntimeError(f"oracle_syndrome_ok failed with status {st}")
    return ok
