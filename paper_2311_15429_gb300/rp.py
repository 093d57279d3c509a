"""Thin ctypes binding of the C-ABI in include/rp.h.

Argument marshalling only: every function here has the name of the C entry
point it calls, converts torch tensors / numpy arrays to raw pointers, and
raises ``RPError`` on a non-OK status.  All computation happens in librp.so.
``load()`` fails loudly if the library is missing or does not load; there is
no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

from . import build as _build

RP_OK, RP_ERR_ARG, RP_ERR_STATE, RP_ERR_HISTORY, RP_ERR_CUDA, RP_ERR_OOM, \
    RP_ERR_UNSUPPORTED, RP_ERR_TIMEOUT = range(8)
RP_MODE_FFT, RP_MODE_DIRECT, RP_MODE_LOWRANK = 0, 1, 2
RP_FLAG_GROUND_STATE_CLAMP, RP_FLAG_PLAN_ONLY, RP_FLAG_PROFILE, RP_FLAG_DEFER_FAR = 0x1, 0x2, 0x4, 0x8
RP_FLAG_GROUND_STATE_SPLIT = 0x10
RP_FLAG_HISTORY_SPILL = 0x20
RP_FLAG_AUDIT = 0x40
RP_FLAG_PLAIN_SUM = 0x80
RP_FLAG_OVERLAP_PUSH = 0x100
RP_PAIR_FFT, RP_PAIR_DIRECT, RP_PAIR_LOWRANK, RP_PAIR_LEARNED, RP_PAIR_OTHER = 0, 1, 2, 3, 4
(RP_K_RING_PUSH, RP_K_FWD_PLANE, RP_K_FWD_COLUMN, RP_K_MAC_INV_COLUMN, RP_K_INV_PLANE,
 RP_K_DIRECT, RP_K_FAR_CONVERT, RP_K_FAR_GEMM, RP_K_FAR_SCATTER, RP_K_FAR_ANTERP, RP_K_MOMENTS, RP_K_LEARNED,
 RP_K_FAR_INTERP, RP_K_COUNT) = range(14)
MAX_DOMAINS = 256


class rp_config(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("dt", ctypes.c_double), ("history_depth", ctypes.c_int),
                ("mode", ctypes.c_int), ("flags", ctypes.c_uint), ("far_points", ctypes.c_int),
                ("far_distance", ctypes.c_double), ("far_batch", ctypes.c_int), ("mac_warps", ctypes.c_int),
                ("profile_every", ctypes.c_int), ("far_source_points", ctypes.c_int),
                ("device_budget", ctypes.c_longlong), ("mac_stages", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class rp_pair_info_t(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("lag_lo", ctypes.c_int), ("lag_hi", ctypes.c_int),
                ("fft_m", ctypes.c_int * 3), ("r_min", ctypes.c_double), ("r_max", ctypes.c_double)]


class rp_train_config(ctypes.Structure):
    _fields_ = [("learned_distance", ctypes.c_double), ("gate", ctypes.c_double), ("histories", ctypes.c_int),
                ("samples", ctypes.c_int), ("iterations", ctypes.c_int), ("batch", ctypes.c_int),
                ("lr", ctypes.c_float), ("validation", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("reserved", ctypes.c_int * 8)]


class rp_train_report(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int), ("learned", ctypes.c_int), ("train_rows", ctypes.c_longlong),
                ("final_loss", ctypes.c_float), ("train_seconds", ctypes.c_float), ("val_max", ctypes.c_double),
                ("val_mean", ctypes.c_double), ("val_linear_max", ctypes.c_double),
                ("val_linear_mean", ctypes.c_double), ("network_pairs", ctypes.c_int),
                ("reserved", ctypes.c_int * 3)]


class rp_stats(ctypes.Structure):
    _fields_ = [("ndomains", ctypes.c_int), ("npairs_fft", ctypes.c_int),
                ("npairs_direct", ctypes.c_int), ("max_lag", ctypes.c_int),
                ("raw_depth", ctypes.c_int), ("spectral_depth", ctypes.c_int),
                ("step", ctypes.c_longlong), ("device_bytes", ctypes.c_longlong),
                ("spectral_bytes", ctypes.c_longlong), ("kernel_bytes", ctypes.c_longlong),
                ("points", ctypes.c_longlong), ("mac_tma", ctypes.c_int), ("npairs_far", ctypes.c_int),
                ("far_bytes", ctypes.c_longlong), ("mac_warps", ctypes.c_int), ("npairs_learned", ctypes.c_int),
                ("spill_windows", ctypes.c_int), ("reserved", ctypes.c_int), ("host_bytes", ctypes.c_longlong),
                ("audit_rel_l2", ctypes.c_double), ("audit_step", ctypes.c_longlong),
                ("owned_sources", ctypes.c_int), ("npairs_other", ctypes.c_int)]


class RPError(RuntimeError):
    def __init__(self, status: int, message: str = ""):
        self.status = status
        super().__init__(f"{rp_status_str(status)}: {message}" if message else rp_status_str(status))


_lib = None
_V = ctypes.c_void_p
_I = ctypes.c_int
_PP = ctypes.POINTER(ctypes.c_void_p)

# name -> (restype, argtypes); every entry point declared in include/rp.h
SIGNATURES = {
    "rp_create": (_I, [ctypes.POINTER(rp_config), _I, _V, ctypes.POINTER(_V)]),
    "rp_add_domain": (_I, [_V, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I),
                           ctypes.c_double, ctypes.POINTER(_I)]),
    "rp_finalize": (_I, [_V]),
    "rp_own_sources": (_I, [_V, ctypes.POINTER(_I), _I]),
    "rp_push": (_I, [_V, _I, _V, _V]),
    "rp_push_all": (_I, [_V, _PP, _PP]),
    "rp_push_host": (_I, [_V, _I, _V, _V]),
    "rp_push_all_host": (_I, [_V, _PP, _PP]),
    "rp_push_all_event": (_I, [_V, _PP, _PP, _V]),
    "rp_evaluate": (_I, [_V, _PP, _PP]),
    "rp_evaluate_host": (_I, [_V, _PP, _PP]),
    "rp_evaluate_host_noalloc": (_I, [_V, _PP, _PP]),
    "rp_fields": (_I, [_V, _I, _V, _V, _V, _V, _V, _V]),
    "rp_ground_potential": (_I, [_V, _PP, _PP]),
    "rp_gemm_bf16": (_I, [_V, _V, _V, _I, _I, _I, _I, _V]),
    "rp_gemm_tn": (_I, [_V, _V, _V, _I, _I, _I, _I, _I, _I, _I, _V]),
    "rp_mlp_layout": (_I, [_V]),
    "rp_mlp_forward": (_I, [_V, _V, _I, _V, _I]),
    "rp_mlp_grad": (_I, [_V, _V, _V, _I, _V, _V, _I]),
    "rp_learned_desc_size": (_I, []),
    "rp_train_far_model": (_I, [_V, _V, _V]),
    "rp_learned_dataset": (_I, [_V, ctypes.c_double, _V, _V, ctypes.c_double, ctypes.c_ulonglong, _I, _I,
                                ctypes.c_double, ctypes.c_double, _V, _V, _V, _I]),
    "rp_sync": (_I, [_V]),
    "rp_query": (_I, [_V, ctypes.POINTER(rp_stats)]),
    "rp_pair_info": (_I, [_V, _I, _I, ctypes.POINTER(rp_pair_info_t)]),
    "rp_kernel_stats": (_I, [_V, _I, ctypes.POINTER(ctypes.c_longlong),
                             ctypes.POINTER(ctypes.c_double), _I]),
    "rp_kernel_count": (_I, [_V, _I, ctypes.POINTER(ctypes.c_longlong)]),
    "rp_set_profiling": (_I, [_V, _I]),
    "rp_audit_values": (_I, [_V, _I, _V, _I, _V]),
    "rp_audit": (_I, [_V, _PP, _PP, _I, ctypes.c_ulonglong, _V]),
    "rp_selftest_wait": (_I, [_V, ctypes.c_longlong]),
    "rp_graph_capture": (_I, [_V, _PP, _PP, _PP, _PP]),
    "rp_graph_step": (_I, [_V]),
    "rp_kernel_name": (ctypes.c_char_p, [_I]),
    "rp_save_state": (_I, [_V, ctypes.c_char_p]),
    "rp_load_state": (_I, [_V, ctypes.c_char_p]),
    "rp_destroy": (None, [_V]),
    "rp_status_str": (ctypes.c_char_p, [_I]),
    "rp_last_error": (ctypes.c_char_p, [_V]),
}


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load librp.so (building it first if ``build`` and it is stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"librp.so not found at {_build.LIB}; run paper_2311_15429_gb300/build.py")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x) -> int:
    """Raw address of a torch tensor, numpy array or int."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if str(x.dtype) != "torch.float32" or not x.is_contiguous():
            raise ValueError("tensor must be contiguous float32")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        import numpy as np
        if x.dtype != np.float32 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous float32")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _ptr_array(xs: Sequence):
    if isinstance(xs, ctypes.Array):   # made by pointer_array
        return ctypes.cast(xs, _PP), xs
    arr = (ctypes.c_void_p * len(xs))(*[_ptr(x) for x in xs])
    return ctypes.cast(arr, _PP), arr


def pointer_array(xs: Sequence):
    """The per-domain pointer array of a call taking one buffer per domain
    (rp_push_all, rp_push_all_host, rp_evaluate, rp_evaluate_host), built
    once for buffers that are reused: those calls accept it in place of the
    list.  The buffers must outlive it."""
    return (ctypes.c_void_p * len(xs))(*[_ptr(x) for x in xs])


def _check(st: int, ctx=None):
    if st != RP_OK:
        msg = load().rp_last_error(ctx).decode() if ctx else ""
        raise RPError(st, msg)


def rp_status_str(status: int) -> str:
    return load().rp_status_str(status).decode()


def rp_kernel_name(kind: int) -> Optional[str]:
    s = load().rp_kernel_name(kind)
    return s.decode() if s is not None else None


def rp_last_error(ctx) -> str:
    return load().rp_last_error(ctx).decode()


def rp_create(c: float, dt: float, history_depth: int = 0, mode: int = RP_MODE_FFT,
              flags: int = 0, device: int = 0, stream=None, far_distance: float = 0.0,
              far_points: int = 0, far_batch: int = 0, mac_warps: int = 0, profile_every: int = 0,
              far_source_points: int = 0, device_budget: int = 0, mac_stages: int = 0):
    """Returns the context handle.  ``stream``: a torch.cuda.Stream, a raw
    cudaStream_t int, or None for torch's current stream (NULL without torch)."""
    cfg = rp_config(c, dt, history_depth, mode, flags, far_points, far_distance, far_batch, mac_warps,
                    profile_every, far_source_points, device_budget, mac_stages)
    if stream is None and not (flags & RP_FLAG_PLAN_ONLY):
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream(device).cuda_stream
        except ImportError:
            stream = None
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    out = ctypes.c_void_p()
    _check(load().rp_create(ctypes.byref(cfg), device, stream or 0, ctypes.byref(out)))
    return out


def rp_add_domain(ctx, origin, n, h: float) -> int:
    o = (ctypes.c_double * 3)(*[float(v) for v in origin])
    nn = (ctypes.c_int * 3)(*[int(v) for v in n])
    i = ctypes.c_int()
    _check(load().rp_add_domain(ctx, o, nn, float(h), ctypes.byref(i)), ctx)
    return i.value


def rp_own_sources(ctx, ids: Sequence[int]):
    """Source partition: the context owns these source domains and no other."""
    arr = (ctypes.c_int * len(ids))(*[int(i) for i in ids])
    _check(load().rp_own_sources(ctx, arr, len(ids)), ctx)


def rp_finalize(ctx):
    _check(load().rp_finalize(ctx), ctx)


def rp_push(ctx, dom: int, rho, J):
    _check(load().rp_push(ctx, dom, _ptr(rho), _ptr(J)), ctx)


def rp_push_all(ctx, rhos: Sequence, Js: Sequence):
    pr, _a = _ptr_array(rhos)
    pj, _b = _ptr_array(Js)
    _check(load().rp_push_all(ctx, pr, pj), ctx)


def rp_push_all_event(ctx, rhos: Sequence, Js: Sequence, ready=None):
    """rp_push_all under RP_FLAG_OVERLAP_PUSH whose inputs are complete after
    `ready` (a torch.cuda.Event, a raw cudaEvent_t, or None: already complete)."""
    pr, _a = _ptr_array(rhos)
    pj, _b = _ptr_array(Js)
    if ready is not None and hasattr(ready, "cuda_event"):
        ready = ready.cuda_event
    _check(load().rp_push_all_event(ctx, pr, pj, ready or 0), ctx)


def rp_push_host(ctx, dom: int, rho, J):
    _check(load().rp_push_host(ctx, dom, _ptr(rho), _ptr(J)), ctx)


def rp_push_all_host(ctx, rhos: Sequence, Js: Sequence):
    pr, _a = _ptr_array(rhos)
    pj, _b = _ptr_array(Js)
    _check(load().rp_push_all_host(ctx, pr, pj), ctx)


def rp_evaluate(ctx, phis: Sequence, As: Sequence):
    pp, _a = _ptr_array(phis)
    pa, _b = _ptr_array(As)
    _check(load().rp_evaluate(ctx, pp, pa), ctx)


def rp_evaluate_host(ctx, phis: Sequence, As: Sequence):
    pp, _a = _ptr_array(phis)
    pa, _b = _ptr_array(As)
    _check(load().rp_evaluate_host(ctx, pp, pa), ctx)


def rp_evaluate_host_noalloc(ctx, phis: Sequence, As: Sequence):
    pp, _a = _ptr_array(phis)
    pa, _b = _ptr_array(As)
    _check(load().rp_evaluate_host_noalloc(ctx, pp, pa), ctx)


def rp_ground_potential(ctx, phis: Sequence, As: Sequence):
    """Under RP_FLAG_GROUND_STATE_SPLIT: the static potential P(0) into device
    buffers phis[n] (N_n floats) and As[n] (3 N_n floats)."""
    pp, _a = _ptr_array(phis)
    pa, _b = _ptr_array(As)
    _check(load().rp_ground_potential(ctx, pp, pa), ctx)


def rp_fields(ctx, dom: int, phi, A, A1, A2, E, B=None):
    """E = -grad phi - (1/c) dA/dt and B = curl A on domain ``dom`` (App. B):
    device buffers phi [N], A / A1 / A2 [3N] (steps l, l-1, l-2; A2 may be
    None), E [3N], B [3N] or None."""
    _check(load().rp_fields(ctx, dom, _ptr(phi), _ptr(A), _ptr(A1), _ptr(A2), _ptr(E), _ptr(B)), ctx)


def rp_gemm_bf16(A, B, D, device: int = 0, stream=None):
    """D = A @ B.T on the tensor cores: A (M x K) and B (N x K) bfloat16 CUDA
    tensors, D (M x N) float32."""
    M, K = A.shape
    N = B.shape[0]
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(device).cuda_stream
    for t in (A, B, D):
        if not t.is_contiguous():
            raise ValueError("operands must be contiguous")
    _check(load().rp_gemm_bf16(A.data_ptr(), B.data_ptr(), D.data_ptr(), M, N, K, device, stream))


RP_DTYPE_BF16, RP_DTYPE_FP16 = 0, 1


def rp_gemm_tn(A, B, D, terms: int = 1, splits: int = 0, device: int = 0, stream=None):
    """D = A @ B.T on the tensor cores for bfloat16 or float16 A and B (the
    same type).  terms=3: A is (M x 2K) = [A_hi | A_lo], B is (N x 2K) =
    [B_hi | B_lo], and D = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T.
    splits=0 picks the split-K count."""
    import torch
    M, W = A.shape
    N = B.shape[0]
    K = W // 2 if terms == 3 else W
    if A.dtype != B.dtype or A.dtype not in (torch.bfloat16, torch.float16):
        raise ValueError("A and B must both be bfloat16 or both float16")
    dtype = RP_DTYPE_FP16 if A.dtype == torch.float16 else RP_DTYPE_BF16
    if stream is None:
        stream = torch.cuda.current_stream(device).cuda_stream
    for t in (A, B, D):
        if not t.is_contiguous():
            raise ValueError("operands must be contiguous")
    _check(load().rp_gemm_tn(A.data_ptr(), B.data_ptr(), D.data_ptr(), M, N, K, dtype, terms, splits, device,
                             stream))


def rp_mlp_layout():
    """(layer widths [5], number of weights) of the learned far field's network."""
    dims = (ctypes.c_int * 5)()
    n = load().rp_mlp_layout(dims)
    return list(dims), n


def _f32(a):
    import numpy as _np
    return _np.ascontiguousarray(a, dtype=_np.float32)


def rp_mlp_forward(weights, x, device: int = 0):
    """Network outputs [rows][d4] for inputs x [rows][d0] (host arrays)."""
    import numpy as _np
    dims, nw = rp_mlp_layout()
    w, x = _f32(weights), _f32(x)
    if w.size != nw or x.ndim != 2 or x.shape[1] != dims[0]:
        raise ValueError("shape mismatch")
    y = _np.zeros((x.shape[0], dims[4]), dtype=_np.float32)
    _check(load().rp_mlp_forward(w.ctypes.data, x.ctypes.data, x.shape[0], y.ctypes.data, device))
    return y


def rp_mlp_grad(weights, x, t, device: int = 0):
    """(loss, dL/dW as one array) of the network on inputs x and targets t."""
    import numpy as _np
    dims, nw = rp_mlp_layout()
    w, x, t = _f32(weights), _f32(x), _f32(t)
    g = _np.zeros(nw, dtype=_np.float32)
    loss = ctypes.c_float()
    _check(load().rp_mlp_grad(w.ctypes.data, x.ctypes.data, t.ctypes.data, x.shape[0], g.ctypes.data,
                              ctypes.byref(loss), device))
    return float(loss.value), g


def rp_learned_dataset(n_s, h_s, Lt, direction, Rc, seed, histories, samples, c, dt, device: int = 0):
    """(X [rows][d0], Y [rows][d4], desc [histories][rp_learned_desc_size()])
    of the learned field's training data for one geometry."""
    import numpy as _np
    dims, _ = rp_mlp_layout()
    rows = histories * samples * 4
    X = _np.zeros((rows, dims[0]), dtype=_np.float32)
    Y = _np.zeros((rows, dims[4]), dtype=_np.float32)
    D = _np.zeros((histories, load().rp_learned_desc_size()), dtype=_np.float64)
    ns = (ctypes.c_int * 3)(*[int(v) for v in n_s])
    lt = (ctypes.c_double * 3)(*[float(v) for v in Lt])
    dr = (ctypes.c_double * 3)(*[float(v) for v in direction])
    _check(load().rp_learned_dataset(ns, float(h_s), lt, dr, float(Rc), int(seed), int(histories), int(samples),
                                     float(c), float(dt), X.ctypes.data, Y.ctypes.data, D.ctypes.data, device))
    return X, Y, D


def rp_train_far_model(ctx, learned_distance: float, gate: float = 0.0, histories: int = 0, samples: int = 0,
                       iterations: int = 0, batch: int = 0, lr: float = 0.0, validation: int = 0, seed: int = 1):
    """Train the learned far field on the context's far pairs; returns the report as a dict."""
    cfg = rp_train_config(learned_distance, gate, histories, samples, iterations, batch, lr, validation, seed)
    rep = rp_train_report()
    _check(load().rp_train_far_model(ctx, ctypes.byref(cfg), ctypes.byref(rep)), ctx)
    return {name: getattr(rep, name) for name, _ in rp_train_report._fields_ if name != "reserved"}


def rp_sync(ctx):
    _check(load().rp_sync(ctx), ctx)


def rp_query(ctx) -> dict:
    s = rp_stats()
    _check(load().rp_query(ctx, ctypes.byref(s)), ctx)
    return {name: getattr(s, name) for name, _ in rp_stats._fields_ if name != "reserved"}


def rp_pair_info(ctx, target: int, source: int) -> dict:
    p = rp_pair_info_t()
    _check(load().rp_pair_info(ctx, target, source, ctypes.byref(p)), ctx)
    return {"kind": p.kind, "lag_lo": p.lag_lo, "lag_hi": p.lag_hi, "fft_m": tuple(p.fft_m),
            "r_min": p.r_min, "r_max": p.r_max}


def rp_kernel_stats(ctx, kind: int, reset: bool = False):
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    _check(load().rp_kernel_stats(ctx, kind, ctypes.byref(n), ctypes.byref(ms), int(reset)), ctx)
    return n.value, ms.value


def rp_graph_capture(ctx, rhos: Sequence, Js: Sequence, phis: Sequence, As: Sequence):
    """Record push_all + evaluate on these device buffers as a CUDA graph."""
    a, _a = _ptr_array(rhos)
    b, _b = _ptr_array(Js)
    c, _c = _ptr_array(phis)
    d, _d = _ptr_array(As)
    _check(load().rp_graph_capture(ctx, a, b, c, d), ctx)


def rp_graph_step(ctx):
    _check(load().rp_graph_step(ctx), ctx)


def rp_selftest_wait(ctx, limit_cycles: int):
    _check(load().rp_selftest_wait(ctx, int(limit_cycles)), ctx)


def rp_set_profiling(ctx, every: int):
    """Per-launch CUDA events on the launches of steps s % every == 0 (every >= 1), or off (0)."""
    _check(load().rp_set_profiling(ctx, int(every)), ctx)


def rp_audit_values(ctx, target: int, nodes):
    """FP64 potentials [len(nodes)][4] at node ids of domain ``target``
    (RP_FLAG_AUDIT), computed on the GPU from the context's history."""
    import numpy as _np
    n = _np.ascontiguousarray(nodes, dtype=_np.int64).reshape(-1)
    out = _np.zeros((n.size, 4), dtype=_np.float64)
    _check(load().rp_audit_values(ctx, int(target), n.ctypes.data, int(n.size), out.ctypes.data), ctx)
    return out


def rp_audit(ctx, phis: Sequence, As: Sequence, nodes_per_domain: int, seed: int = 0):
    """rel-L2 [ndomains][4] of the outputs against the GPU's FP64 sums at
    sampled nodes (RP_FLAG_AUDIT)."""
    import numpy as _np
    pp, _a = _ptr_array(phis)
    pa, _b = _ptr_array(As)
    out = _np.zeros((len(phis), 4), dtype=_np.float64)
    _check(load().rp_audit(ctx, pp, pa, int(nodes_per_domain), int(seed), out.ctypes.data), ctx)
    return out


def rp_kernel_count(ctx, kind: int) -> int:
    n = ctypes.c_longlong()
    _check(load().rp_kernel_count(ctx, kind, ctypes.byref(n)), ctx)
    return n.value


def rp_save_state(ctx, path: str):
    _check(load().rp_save_state(ctx, path.encode()), ctx)


def rp_load_state(ctx, path: str):
    _check(load().rp_load_state(ctx, path.encode()), ctx)


def rp_destroy(ctx):
    if ctx:
        load().rp_destroy(ctx)


class RetardedPotentials:
    """Owns one context: domains from ``synth.Domain``-like objects (origin,
    n, h), device output buffers as torch tensors, and the push / evaluate
    calls of a time step."""

    def __init__(self, domains, c: float, dt: float, history_depth: int = 0,
                 mode: int = RP_MODE_FFT, flags: int = 0, device: int = 0, stream=None,
                 far_distance: float = 0.0, far_points: int = 0, far_batch: int = 0,
                 mac_warps: int = 0, profile_every: int = 0, far_source_points: int = 0,
                 device_budget: int = 0, owned_sources: Optional[Sequence[int]] = None, mac_stages: int = 0):
        import torch
        self.domains = list(domains)
        self.ctx = rp_create(c, dt, history_depth, mode, flags, device, stream, far_distance,
                             far_points, far_batch, mac_warps, profile_every, far_source_points,
                             device_budget, mac_stages)
        try:
            for d in self.domains:
                rp_add_domain(self.ctx, d.origin, d.n, d.h)
            if owned_sources is not None:
                rp_own_sources(self.ctx, owned_sources)
            rp_finalize(self.ctx)
        except Exception:
            rp_destroy(self.ctx)
            self.ctx = None
            raise
        if flags & RP_FLAG_PLAN_ONLY:
            self.phi = self.A = None
        else:
            dev = torch.device("cuda", device)
            self.phi = [torch.empty(d.N, dtype=torch.float32, device=dev) for d in self.domains]
            self.A = [torch.empty(3 * d.N, dtype=torch.float32, device=dev) for d in self.domains]

    def push(self, dom: int, rho, J):
        rp_push(self.ctx, dom, rho, J)

    def push_all(self, rhos, Js):
        rp_push_all(self.ctx, rhos, Js)

    def evaluate(self):
        rp_evaluate(self.ctx, self.phi, self.A)
        return self.phi, self.A

    def sync(self):
        rp_sync(self.ctx)

    def train_far_model(self, learned_distance: float, **kw):
        return rp_train_far_model(self.ctx, learned_distance, **kw)

    def query(self):
        return rp_query(self.ctx)

    def pair_info(self, t, s):
        return rp_pair_info(self.ctx, t, s)

    def close(self):
        if self.ctx:
            rp_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
