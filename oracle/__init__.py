"""FP64 CPU oracle for the retarded potentials (test infrastructure only).

The oracle is the plain direct retarded sum of the paper (Eq. 2 summed over
sub-domains as in Eqs. 3-4, discretised as in Eq. 8 with the hat-function
time interpolation of Eq. 7; Eqs. 11-12 give the same number), written in C
(``rp_oracle.c``) and called through ctypes.  Only ``tests/``, the package's
``smoke()`` check and ``bench.py``'s CPU-baseline leg may import this module;
the CUDA library neither links nor imports it, and it shares no code with it.

Parity status per function:
  * ``eval_points_windows`` -- ``eval_points`` with a stored window per
    domain (so that a far source needs only the samples around its delay);
    the same code path as ``eval_points``, which calls it with one window.
  * ``eval_positions`` -- the same sums at arbitrary points; pinned by the
    static Coulomb limit and the retarded phase lag at far points, and by
    agreement with ``eval_points`` where the points are grid nodes of a
    domain with no own source (``tests/test_oracle_learned.py``).
  * ``learned`` -- the learned far field's steps (moments, canonical frame,
    delay window, network, re-interpolation); see that module's header.
  * ``eval_points`` -- pinned by the closed forms and brute-force forms in
    ``tests/test_oracle_pins.py`` (static Coulomb limit of a Gaussian, the
    O(h^2) self-cell constant, retarded phase lag of a breathing monopole,
    the Lorenz gauge condition, the Eq. 12 Delta-S form, reciprocity,
    linearity and time-shift invariance).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rp_oracle.c")
_LIB = os.path.join(_HERE, "_build", "librp_oracle.so")

OK, ERR_HISTORY, ERR_ARG, ERR_COINCIDENT = 0, 1, 2, 3
_ERRORS = {ERR_HISTORY: "sample outside the stored history",
           ERR_ARG: "bad argument",
           ERR_COINCIDENT: "nodes of two domains coincide"}

_lib = None


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {_ERRORS.get(code, 'unknown')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (IEEE arithmetic, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path: str):
    """Load a compiled oracle and declare its C signatures."""
    lib = ctypes.CDLL(path)
    lib.rpo_eval.restype = ctypes.c_int
    lib.rpo_eval.argtypes = [
        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_double, ctypes.c_double, ctypes.c_int,
        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.rpo_eval_windows.restype = ctypes.c_int
    lib.rpo_eval_windows.argtypes = [
        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_double, ctypes.c_double, ctypes.c_int,
        ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.rpo_eval_positions.restype = ctypes.c_int
    lib.rpo_eval_positions.argtypes = [
        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
        ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
        ctypes.c_double, ctypes.c_double, ctypes.c_int,
        ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    lib.rpo_cube_average_constant.restype = ctypes.c_double
    lib.rpo_cube_average_constant.argtypes = []
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(_LIB)
    return _lib


def cube_average_constant() -> float:
    """C such that the cell-averaged self weight is C*h^2."""
    return _load().rpo_cube_average_constant()


def history_needed(origins, ns, hs, c: float, dt: float) -> int:
    """How many steps back the sums read: the retarded time of the farthest
    node pair, R_max/c, falls between samples floor(R_max/(c dt)) and that + 1
    before the evaluated step (Eq. 7's hat interpolation reads both), so the
    history must reach that many steps back.  R_max is the distance between
    the farthest corners of two domains' node lattices, over all ordered
    pairs (self pairs included)."""
    ndom = len(hs)
    o = np.asarray(origins, dtype=np.float64).reshape(ndom, 3)
    n = np.asarray(ns, dtype=np.float64).reshape(ndom, 3)
    h = np.asarray(hs, dtype=np.float64).reshape(ndom, 1)
    lo, hi = o, o + h * (n - 1)
    worst = 0
    for t in range(ndom):
        for s in range(ndom):
            far = np.maximum(np.abs(hi[t] - lo[s]), np.abs(hi[s] - lo[t]))
            worst = max(worst, int(np.floor(np.sqrt(np.sum(far * far)) / (c * dt))) + 1)
    return worst


def eval_points(origins: np.ndarray, ns: np.ndarray, hs: Sequence[float],
                hists: Sequence[np.ndarray], hist_first: int,
                c: float, dt: float, target: int, step: int, nodes,
                clamp: bool = False) -> np.ndarray:
    """Retarded (phi, Ax, Ay, Az) at ``nodes`` of domain ``target`` and time index ``step``.

    ``hists[n]`` is an array [T][4][N_n] (float32 or float64, one dtype for
    all domains) holding the samples of time indices hist_first..hist_first+T-1.
    Returns an array [len(nodes)][4] in float64.
    """
    lib = _load()
    ndom = len(hists)
    origins = np.ascontiguousarray(origins, dtype=np.float64).reshape(ndom, 3)
    ns = np.ascontiguousarray(ns, dtype=np.int32).reshape(ndom, 3)
    hs = np.ascontiguousarray(hs, dtype=np.float64).reshape(ndom)
    is_f64 = hists[0].dtype == np.float64
    want = np.float64 if is_f64 else np.float32
    T = hists[0].shape[0]
    arrs = []
    for d, a in enumerate(hists):
        a = np.ascontiguousarray(a, dtype=want)
        N = int(np.prod(ns[d]))
        if a.shape != (T, 4, N):
            raise ValueError(f"history of domain {d} has shape {a.shape}, expected {(T, 4, N)}")
        arrs.append(a)
    ptrs = (ctypes.c_void_p * ndom)(*[a.ctypes.data for a in arrs])
    nodes = np.ascontiguousarray(nodes, dtype=np.int64).reshape(-1)
    out = np.zeros((nodes.size, 4), dtype=np.float64)
    rc = lib.rpo_eval(ndom, origins.ctypes.data, ns.ctypes.data, hs.ctypes.data,
                      ctypes.cast(ptrs, ctypes.c_void_p), int(is_f64), int(hist_first), int(T),
                      float(c), float(dt), int(bool(clamp)), int(target), int(step),
                      int(nodes.size), nodes.ctypes.data, out.ctypes.data)
    if rc != OK:
        raise OracleError(rc)
    return out


def eval_points_windows(origins, ns, hs, hists, firsts, c: float, dt: float, target: int, step: int,
                        nodes, clamp: bool = False) -> np.ndarray:
    """``eval_points`` with a separate stored window per domain: ``hists[n]``
    [T_n][4][N_n] holds the samples of time indices firsts[n] .. firsts[n]+T_n-1
    (one dtype for all).  Returns [len(nodes)][4] float64."""
    lib = _load()
    ndom = len(hists)
    origins = np.ascontiguousarray(origins, dtype=np.float64).reshape(ndom, 3)
    ns = np.ascontiguousarray(ns, dtype=np.int32).reshape(ndom, 3)
    hs = np.ascontiguousarray(hs, dtype=np.float64).reshape(ndom)
    is_f64 = hists[0].dtype == np.float64
    want = np.float64 if is_f64 else np.float32
    arrs = [np.ascontiguousarray(a, dtype=want) for a in hists]
    for d, a in enumerate(arrs):
        if a.ndim != 3 or a.shape[1:] != (4, int(np.prod(ns[d]))):
            raise ValueError(f"history of domain {d} has shape {a.shape}")
    first = np.ascontiguousarray(firsts, dtype=np.int64).reshape(ndom)
    lens = np.ascontiguousarray([a.shape[0] for a in arrs], dtype=np.int32)
    ptrs = (ctypes.c_void_p * ndom)(*[a.ctypes.data for a in arrs])
    nodes = np.ascontiguousarray(nodes, dtype=np.int64).reshape(-1)
    out = np.zeros((nodes.size, 4), dtype=np.float64)
    rc = lib.rpo_eval_windows(ndom, origins.ctypes.data, ns.ctypes.data, hs.ctypes.data,
                              ctypes.cast(ptrs, ctypes.c_void_p), int(is_f64), first.ctypes.data, lens.ctypes.data,
                              float(c), float(dt), int(bool(clamp)), int(target), int(step),
                              int(nodes.size), nodes.ctypes.data, out.ctypes.data)
    if rc != OK:
        raise OracleError(rc)
    return out


def eval_points_windows_parallel(origins, ns, hs, hists, firsts, c, dt, target, step, nodes, threads=None):
    """``eval_points_windows`` with the nodes split across host threads
    (ctypes releases the GIL).  Returns (values, threads used)."""
    from concurrent.futures import ThreadPoolExecutor
    nodes = np.asarray(nodes, dtype=np.int64).reshape(-1)
    nthr = max(1, min(threads or os.cpu_count() or 1, nodes.size))
    chunks = np.array_split(nodes, nthr)
    with ThreadPoolExecutor(nthr) as ex:
        parts = list(ex.map(lambda ch: eval_points_windows(origins, ns, hs, hists, firsts, c, dt, target, step, ch),
                            chunks))
    return np.concatenate(parts, axis=0), nthr


def eval_positions(origins, ns, hs, hists, hist_first: int, c: float, dt: float, step: int,
                   positions, clamp: bool = False) -> np.ndarray:
    """Retarded (phi, Ax, Ay, Az) at arbitrary points ``positions`` [P][3]
    (bohr) from every domain, at time index ``step``.  Returns [P][4] float64."""
    lib = _load()
    ndom = len(hists)
    origins = np.ascontiguousarray(origins, dtype=np.float64).reshape(ndom, 3)
    ns = np.ascontiguousarray(ns, dtype=np.int32).reshape(ndom, 3)
    hs = np.ascontiguousarray(hs, dtype=np.float64).reshape(ndom)
    is_f64 = hists[0].dtype == np.float64
    want = np.float64 if is_f64 else np.float32
    T = hists[0].shape[0]
    arrs = [np.ascontiguousarray(a, dtype=want) for a in hists]
    for d, a in enumerate(arrs):
        if a.shape != (T, 4, int(np.prod(ns[d]))):
            raise ValueError(f"history of domain {d} has shape {a.shape}")
    ptrs = (ctypes.c_void_p * ndom)(*[a.ctypes.data for a in arrs])
    pos = np.ascontiguousarray(positions, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((pos.shape[0], 4), dtype=np.float64)
    rc = lib.rpo_eval_positions(ndom, origins.ctypes.data, ns.ctypes.data, hs.ctypes.data,
                                ctypes.cast(ptrs, ctypes.c_void_p), int(is_f64), int(hist_first), int(T),
                                float(c), float(dt), int(bool(clamp)), int(step), int(pos.shape[0]),
                                pos.ctypes.data, out.ctypes.data)
    if rc != OK:
        raise OracleError(rc)
    return out


def eval_points_parallel(origins, ns, hs, hists, hist_first, c, dt, target, step, nodes,
                         clamp=False, threads=None):
    """``eval_points`` with the node list split across host threads.

    ctypes releases the GIL for the duration of the C call, so each thread
    runs the same single-threaded oracle on its share of the nodes in
    parallel, reading the one shared copy of the history.
    Returns (values [len(nodes)][4], threads used).
    """
    from concurrent.futures import ThreadPoolExecutor
    nodes = np.asarray(nodes, dtype=np.int64).reshape(-1)
    nthr = threads or os.cpu_count() or 1
    nthr = max(1, min(nthr, nodes.size))
    if nthr == 1:
        return eval_points(origins, ns, hs, hists, hist_first, c, dt, target, step, nodes,
                           clamp=clamp), 1
    chunks = np.array_split(nodes, nthr)
    with ThreadPoolExecutor(nthr) as ex:
        parts = list(ex.map(lambda ch: eval_points(origins, ns, hs, hists, hist_first, c, dt,
                                                   target, step, ch, clamp=clamp), chunks))
    return np.concatenate(parts, axis=0), nthr


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
