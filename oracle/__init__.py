"""CPU oracle for speculative distance-1 coloring (Algorithms 1 and 2 of the paper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library under
``paper_1205_3809_gb300`` never does, and the two share no code: this package
wraps ``oracle.c`` (plain single-threaded C) with ctypes and numpy marshalling.

Every function cites the passage it follows; what pins each one (outside
itself) is listed at the top of ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_LEARNED = os.path.join(_HERE, "learned.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_SRC_ASYNC = os.path.join(_HERE, "async_omp.c")
_LIB_ASYNC = os.path.join(_HERE, "libasync_omp.so")

ORC_OK = 0
ORC_ERR_MAX_ROUNDS = -4


def build(force: bool = False) -> str:
    """Compile liboracle.so (single-threaded, -O2, no FMA contraction) and, apart
    from it, libasync_omp.so (the paper's OpenMP form, a timed baseline only)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_LEARNED))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-Wall",
               "-o", _LIB, _SRC, _SRC_LEARNED, "-lm"]
        subprocess.run(cmd, check=True)
    if force or not os.path.exists(_LIB_ASYNC) or os.path.getmtime(_LIB_ASYNC) < os.path.getmtime(_SRC_ASYNC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall", "-o", _LIB_ASYNC, _SRC_ASYNC]
        try:  # an optional baseline: without OpenMP the rest still builds
            subprocess.run(cmd, check=True)
        except (OSError, subprocess.CalledProcessError) as e:
            print(f"oracle: libasync_omp.so not built ({e}); the OpenMP baseline is unavailable",
                  file=sys.stderr)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            build()
        lib = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        i32 = ctypes.c_int32
        lib.orc_greedy.argtypes = [i32, vp, vp, vp, vp, vp]
        lib.orc_iterative.argtypes = [i32, vp, vp, vp, i32, i32, vp, vp, vp, vp, i32, vp]
        lib.orc_chromatic_number.argtypes = [i32, vp, vp, vp]
        lib.orc_largest_first_order.argtypes = [i32, vp, vp]
        lib.orc_smallest_last_order.argtypes = [i32, vp, vp, vp, vp]
        lib.orc_features.argtypes = [i32, vp, vp, vp]
        lib.orc_mlp_forward.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp]
        lib.orc_bf16_array.argtypes = [vp, ctypes.c_int64, vp]
        for f in (lib.orc_greedy, lib.orc_iterative, lib.orc_chromatic_number,
                  lib.orc_largest_first_order, lib.orc_smallest_last_order, lib.orc_features,
                  lib.orc_mlp_forward, lib.orc_bf16_array, lib.orc_mlp_param_count):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _csr(rowptr, colidx):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    return rowptr, colidx, int(rowptr.shape[0] - 1)


@dataclass
class Coloring:
    colors: np.ndarray          # int32[n], 1-based
    ncolors: int
    rounds: int
    round_sizes: np.ndarray     # int32[rounds]: |U| at the start of each round
    settle_round: np.ndarray    # int32[n]: round after which v left U for good
    status: int = ORC_OK


def greedy(rowptr, colidx, order=None):
    """Algorithm 1 (Greedy, Sec. 3.1): first-fit in `order` (None = 0..n-1).

    Returns (colors int32[n], ncolors).
    """
    rowptr, colidx, n = _csr(rowptr, colidx)
    color = np.zeros(max(n, 0), np.int32)
    nc = ctypes.c_int32()
    order_a = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    rc = _load().orc_greedy(n, _ptr(rowptr), _ptr(colidx), _ptr(order_a), _ptr(color),
                            ctypes.byref(nc))
    if rc != ORC_OK:
        raise RuntimeError(f"orc_greedy failed: {rc}")
    return color, int(nc.value)


def iterative(rowptr, colidx, priority=None, mode: str = "sync",
              max_rounds: int = 0, allow_max_rounds: bool = False) -> Coloring:
    """Algorithm 2 (Iterative, Sec. 3.2) as synchronous rounds (mode="sync") or run
    by one thread (mode="sequential", Phase 1 reads live colors in precedence order).

    priority: uint32[n] or None (None = index order).  Ties break by index.
    """
    rowptr, colidx, n = _csr(rowptr, colidx)
    m = {"sync": 0, "sequential": 1}[mode]
    color = np.zeros(max(n, 0), np.int32)
    settle = np.zeros(max(n, 0), np.int32)
    cap = max(n, 1) if max_rounds <= 0 else max_rounds
    sizes = np.zeros(cap, np.int32)
    nc, rounds = ctypes.c_int32(), ctypes.c_int32()
    prio = None if priority is None else np.ascontiguousarray(priority, dtype=np.uint32)
    rc = _load().orc_iterative(n, _ptr(rowptr), _ptr(colidx), _ptr(prio), m, max_rounds,
                               _ptr(color), ctypes.byref(nc), ctypes.byref(rounds),
                               _ptr(sizes), cap, _ptr(settle))
    if rc != ORC_OK and not (allow_max_rounds and rc == ORC_ERR_MAX_ROUNDS):
        raise RuntimeError(f"orc_iterative failed: {rc}")
    r = int(rounds.value)
    return Coloring(colors=color, ncolors=int(nc.value), rounds=r,
                    round_sizes=sizes[:min(r, cap)].copy(), settle_round=settle, status=rc)


def chromatic_number(rowptr, colidx) -> int:
    """Exact chromatic number by backtracking (n <= 20)."""
    rowptr, colidx, n = _csr(rowptr, colidx)
    chi = ctypes.c_int32()
    rc = _load().orc_chromatic_number(n, _ptr(rowptr), _ptr(colidx), ctypes.byref(chi))
    if rc != ORC_OK:
        raise RuntimeError(f"orc_chromatic_number failed: {rc}")
    return int(chi.value)


def largest_first_order(rowptr) -> np.ndarray:
    """Vertices by degree descending, ties by index."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    n = int(rowptr.shape[0] - 1)
    order = np.zeros(n, np.int32)
    rc = _load().orc_largest_first_order(n, _ptr(rowptr), _ptr(order))
    if rc != ORC_OK:
        raise RuntimeError(f"orc_largest_first_order failed: {rc}")
    return order


def smallest_last_order(rowptr, colidx):
    """Smallest-last ordering; returns (order, removal_degree)."""
    rowptr, colidx, n = _csr(rowptr, colidx)
    order = np.zeros(n, np.int32)
    rdeg = np.zeros(n, np.int32)
    rc = _load().orc_smallest_last_order(n, _ptr(rowptr), _ptr(colidx), _ptr(order), _ptr(rdeg))
    if rc != ORC_OK:
        raise RuntimeError(f"orc_smallest_last_order failed: {rc}")
    return order, rdeg
