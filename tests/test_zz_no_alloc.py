"""gc_color_noalloc, the entry point for callers that cannot allocate memory
while they run (a framework whose caching allocator holds the device's memory,
a service with a fixed memory plan, code that must not let cudaMalloc /
cudaFree synchronise the device).  Its workspace is a fixed file-scope device
array shared by all calls, so two calls in a row must give the same colors as
gc_color_ex, and a graph too large for the array must be refused.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gcpkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1205_3809_gb300 as m
    m.library()
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


def _noalloc(gcpkg, rp, ci, prio=None):
    lib = gcpkg.library()
    n = rp.numel() - 1
    out = torch.full((n,), -1, dtype=torch.int32, device=rp.device)
    nc, rd = ctypes.c_int32(), ctypes.c_int32()
    stream = torch.cuda.current_stream(rp.device)
    rc = lib.gc_color_noalloc(_ptr(rp), _ptr(ci), n, _ptr(prio), _ptr(out), ctypes.byref(nc),
                              ctypes.byref(rd), ctypes.c_void_p(stream.cuda_stream))
    return rc, out, nc.value, rd.value


@pytest.mark.parametrize("with_priority", [False, True])
def test_noalloc_matches_gc_color_ex_on_two_calls(gcpkg, with_priority):
    graphs = [gg.rmat(14, 8, gg.RMAT_B, 3), gg.gnm(10000, 50000, 1), gg.complete(300)]
    for g in graphs:
        rp, ci = _dev(g.rowptr), _dev(g.colidx)
        prio = None
        if with_priority:
            keys = (gg.draws(5, 9, g.n) >> np.uint64(56)).astype(np.uint32)
            prio = _dev(keys.view(np.int32))
        ref = gcpkg.color(rp, ci, prio)  # gc_color_ex, library-managed workspace
        for _ in range(2):
            rc, out, nc, rd = _noalloc(gcpkg, rp, ci, prio)
            assert rc == gcpkg.GC_OK, gcpkg.strerror(rc)
            assert torch.equal(out, ref.colors), g.name
            assert nc == ref.ncolors and rd == ref.rounds, g.name


def test_noalloc_refuses_graph_beyond_its_buffer(gcpkg):
    cap = int(gcpkg.library().gc_noalloc_capacity_bytes())
    n = cap // 16  # more than the per-vertex workspace the fixed buffer can hold
    g = gg.edgeless(n)
    rc, _, _, _ = _noalloc(gcpkg, _dev(g.rowptr), _dev(g.colidx))
    assert rc == gcpkg.GC_ERR_TOO_LARGE
    # and a graph that fits still works afterwards
    small = gg.gnm(2000, 8000, 3)
    rp, ci = _dev(small.rowptr), _dev(small.colidx)
    rc, out, nc, rd = _noalloc(gcpkg, rp, ci)
    ref = gcpkg.color(rp, ci)
    assert rc == gcpkg.GC_OK and torch.equal(out, ref.colors) and rd == ref.rounds
