"""Seeded synthetic graph inputs, shared by the CUDA path's tests/bench and the oracle.

Holds none of the coloring method's arithmetic: it only builds simple symmetric
int32 CSR graphs (rows sorted, no self loops, no duplicates) from a counter-based
SplitMix64 stream, so a given (generator, parameters, seed) gives the same graph
on any machine and any thread count.  R-MAT follows Sec. 4.1 of the paper; the
random id shuffle follows Sec. 5.1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")

# Quadrant probabilities of the paper's three R-MAT families (Sec. 4.1).
RMAT_ER = (0.25, 0.25, 0.25, 0.25)
RMAT_G = (0.45, 0.15, 0.15, 0.25)
RMAT_B = (0.55, 0.15, 0.15, 0.15)


def build(force: bool = False) -> str:
    """Compile libgraphgen.so with gcc (OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-std=c11", "-Wall", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            build()
        lib = ctypes.CDLL(_LIB)
        P32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))
        I64P = ctypes.POINTER(ctypes.c_int64)
        lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                                P32, P32, I64P]
        lib.gg_gnm.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, P32, P32, I64P]
        lib.gg_grid2d.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32,
                                  P32, P32, I64P]
        lib.gg_rgg.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_uint64, P32, P32, I64P]
        lib.gg_csr_from_edges.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, P32, P32, I64P]
        lib.gg_permutation.argtypes = [ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p]
        lib.gg_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_draw.restype = ctypes.c_uint64
        lib.gg_free.argtypes = [ctypes.c_void_p]
        lib.gg_num_threads.restype = ctypes.c_int
        for f in (lib.gg_rmat, lib.gg_gnm, lib.gg_grid2d, lib.gg_rgg, lib.gg_csr_from_edges,
                  lib.gg_permutation):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class Graph:
    """Simple undirected graph as a symmetric CSR: rowptr (n+1), colidx (2m)."""
    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.colidx.shape[0])

    @property
    def m(self) -> int:
        """Undirected edge count, as the paper counts edges (Table 2)."""
        return self.nnz // 2

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.rowptr.astype(np.int64))

    @property
    def max_degree(self) -> int:
        return int(self.degrees.max()) if self.n > 0 else 0


def _take(fn, *args, n: int, name: str) -> Graph:
    lib = _load()
    rp = ctypes.POINTER(ctypes.c_int32)()
    ci = ctypes.POINTER(ctypes.c_int32)()
    nnz = ctypes.c_int64()
    rc = fn(*args, ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(nnz))
    if rc != 0:
        raise ValueError(f"graph generator {name} failed with code {rc}")
    try:
        rowptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
        colidx = (np.ctypeslib.as_array(ci, shape=(nnz.value,)).copy()
                  if nnz.value > 0 else np.zeros(0, np.int32))
    finally:
        lib.gg_free(ctypes.cast(rp, ctypes.c_void_p))
        lib.gg_free(ctypes.cast(ci, ctypes.c_void_p))
    return Graph(n=n, rowptr=rowptr, colidx=colidx, name=name)


def rmat(scale: int, edge_factor: int, abcd, seed: int, permute: bool = True) -> Graph:
    """R-MAT graph (Sec. 4.1) with 2**scale vertices and edge_factor*2**scale samples."""
    a, b, c, d = abcd
    return _take(_load().gg_rmat, scale, edge_factor, a, b, c, d, seed, 1 if permute else 0,
                 n=1 << scale, name=f"rmat(s={scale},ef={edge_factor},{abcd},seed={seed})")


def gnm(n: int, m: int, seed: int) -> Graph:
    """Uniform simple graph with exactly m undirected edges."""
    return _take(_load().gg_gnm, n, m, seed, n=n, name=f"gnm(n={n},m={m},seed={seed})")


def grid2d(rows: int, cols: int, seed: int = 0, permute: bool = True) -> Graph:
    """rows x cols 5-point mesh, ids shuffled when permute is set."""
    return _take(_load().gg_grid2d, rows, cols, seed, 1 if permute else 0, n=rows * cols,
                 name=f"grid2d({rows}x{cols},seed={seed})")


def rgg(n: int, seed: int, avg_degree: float = 8.0) -> Graph:
    """Random geometric graph in the unit square with radius sqrt(avg_degree/(pi n))."""
    radius = min(1.0, float(np.sqrt(avg_degree / (np.pi * max(n, 1)))))
    return _take(_load().gg_rgg, n, radius, seed, n=n, name=f"rgg(n={n},seed={seed})")


def from_edges(n: int, u, v, name: str = "edges") -> Graph:
    """Simple symmetric CSR from an undirected edge list (loops/duplicates dropped)."""
    u = np.ascontiguousarray(np.asarray(u, dtype=np.int32))
    v = np.ascontiguousarray(np.asarray(v, dtype=np.int32))
    assert u.shape == v.shape
    return _take(_load().gg_csr_from_edges, n, u.shape[0], u.ctypes.data, v.ctypes.data,
                 n=n, name=name)


def permutation(n: int, seed: int) -> np.ndarray:
    """Pseudo-random permutation of range(n) (keyed Feistel bijection)."""
    out = np.empty(n, np.int32)
    rc = _load().gg_permutation(n, seed, out.ctypes.data)
    if rc != 0:
        raise ValueError("permutation failed")
    return out


def draws(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Raw 64-bit SplitMix64 draws of a stream, for seeded test data."""
    lib = _load()
    return np.array([lib.gg_draw(seed, stream, start + i) for i in range(count)], dtype=np.uint64)


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """Same graph with vertex i renamed perm[i]."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees)
    return from_edges(g.n, perm[src], perm[g.colidx], name=g.name + "+relabel")


# ---- small named shapes used by tests (edge lists only, no method arithmetic)

def path(n: int) -> Graph:
    k = np.arange(max(n - 1, 0))
    return from_edges(n, k, k + 1, name=f"path({n})")


def cycle(n: int) -> Graph:
    k = np.arange(n)
    return from_edges(n, k, (k + 1) % n, name=f"cycle({n})")


def star(n: int, hub: int) -> Graph:
    leaves = np.array([v for v in range(n) if v != hub], dtype=np.int32)
    return from_edges(n, np.full(leaves.shape, hub), leaves, name=f"star({n},hub={hub})")


def complete(n: int) -> Graph:
    iu = np.triu_indices(n, 1)
    return from_edges(n, iu[0], iu[1], name=f"K{n}")


def complete_bipartite(a: int, b: int) -> Graph:
    u, v = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return from_edges(a + b, u.ravel(), v.ravel(), name=f"K{a},{b}")


def edgeless(n: int) -> Graph:
    return from_edges(n, [], [], name=f"edgeless({n})")


def num_threads() -> int:
    return int(_load().gg_num_threads())


# ---- the batched workload: many small graphs of mixed families

BATCH_FAMILIES = ("grid2d", "rgg", "rmat_g")


def batch_mix(count: int, seed: int, n_min: int = 1000, n_max: int = 200000):
    """`count` graphs with sizes log-uniform in [n_min, n_max], families in turn
    drawn from 2-D 5-point grids (rows x cols about n), random geometric graphs
    (average degree 8) and R-MAT-G (edge factor 8; 2^round(log2 n) vertices,
    since R-MAT's recursive quadrants define a power of two).  Graph i uses
    SplitMix64 streams (seed, 41..43) at counter i."""
    u = draws(seed, 41, count)
    fam = draws(seed, 42, count)
    gseed = draws(seed, 43, count)
    lo, hi = np.log(float(n_min)), np.log(float(n_max))
    out = []
    for i in range(count):
        x = float(u[i] >> np.uint64(11)) / float(1 << 53)
        n = int(round(np.exp(lo + x * (hi - lo))))
        s = int(gseed[i] & np.uint64(0x7FFFFFFF))
        kind = BATCH_FAMILIES[int(fam[i] % np.uint64(3))]
        if n < 2:
            g = edgeless(max(n, 0))
        elif kind == "grid2d":
            rows = max(1, int(round(np.sqrt(n))))
            g = grid2d(rows, max(1, int(round(n / rows))), s)
        elif kind == "rgg":
            g = rgg(n, s)
        else:
            g = rmat(max(1, int(round(np.log2(n)))), 8, RMAT_G, s)
        out.append(g)
    return out
