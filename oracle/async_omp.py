"""The paper's multicore form of Algorithm 2 (asynchronous Phase 1, OpenMP
threads; Sec. 3.2, Sec. 4), wrapped for timing beside the GPU path.

TEST AND BASELINE INFRASTRUCTURE ONLY (``tests/`` and the CPU-baseline leg of
``bench.py``).  Its result depends on the thread schedule, so it is judged by
validity only; ``python -m oracle.async_omp`` times it on an R-MAT-B graph and
prints one JSON line (``bench.py`` runs it in a child process with a time limit).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import sys
import time

import numpy as np

from . import _LIB_ASYNC, build

_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_ASYNC):
            build()
        lib = ctypes.CDLL(_LIB_ASYNC)
        vp, i32 = ctypes.c_void_p, ctypes.c_int32
        lib.orc_async_omp.argtypes = [i32, vp, vp, vp, i32, i32, vp, vp, vp]
        lib.orc_async_omp.restype = ctypes.c_int
        _lib = lib
    return _lib


def color(rowptr, colidx, priority=None, threads: int = 0, max_rounds: int = 0):
    """Returns (colors int32[n], ncolors, rounds, status)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    n = int(rowptr.shape[0]) - 1
    out = np.zeros(max(n, 0), np.int32)
    prio = None if priority is None else np.ascontiguousarray(priority, dtype=np.uint32)
    nc, rd = ctypes.c_int32(), ctypes.c_int32()
    ptr = lambda a: None if a is None or a.size == 0 else ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    rc = _load().orc_async_omp(n, ptr(rowptr), ptr(colidx), ptr(prio), int(threads), int(max_rounds), ptr(out),
                               ctypes.byref(nc), ctypes.byref(rd))
    return out, int(nc.value), int(rd.value), int(rc)


def valid(rowptr, colidx, colors) -> bool:
    """A proper coloring with 1 <= color(v) <= deg(v) + 1."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    deg = np.diff(rowptr)
    if colors.size and (colors.min() < 1 or np.any(colors > deg + 1)):
        return False
    src = np.repeat(np.arange(colors.size, dtype=np.int64), deg)
    return not np.any(colors[src] == colors[np.asarray(colidx, dtype=np.int64)])


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import graphgen as gg
    g = gg.rmat(args.scale, 8, gg.RMAT_B, args.seed)
    color(np.zeros(2, np.int32), np.zeros(0, np.int32))  # load the library outside the timed call
    t = time.perf_counter()
    colors, nc, rd, rc = color(g.rowptr, g.colidx, threads=args.threads)
    s = time.perf_counter() - t
    threads = args.threads if args.threads > 0 else int(os.environ.get("OMP_NUM_THREADS") or os.cpu_count() or 1)
    print(json.dumps({"value": g.m / s, "unit": "edges/s", "seconds": round(s, 3), "threads": threads,
                      "ncolors": nc, "rounds": rd, "status": rc,
                      "valid": bool(rc == 0 and valid(g.rowptr, g.colidx, colors)),
                      "sample": f"R-MAT-B scale {args.scale} seed {args.seed}: {g.m} edges, one run"}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
