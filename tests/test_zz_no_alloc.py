"""gc_color_noalloc, the entry point for callers that cannot allocate memory
while they run (a framework whose caching allocator holds the device's memory,
a service with a fixed memory plan, code that must not let cudaMalloc /
cudaFree synchronise the device).  Its workspace is a fixed file-scope device
array shared by all calls, so two calls in a row must give what the oracle
and gc_color_ex give, a graph too large for the array must be refused, and the
calls must allocate nothing: checked in a child process of its own, so that
what other tests allocated does not matter.

This file is named so that pytest collects it last; none of its checks
depends on that.
"""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def _noalloc(gcpkg, rp, ci, prio=None, out=None):
    lib = gcpkg.library()
    n = rp.numel() - 1
    if out is None:
        out = torch.full((n,), -1, dtype=torch.int32, device=rp.device)
    nc, rd = ctypes.c_int32(), ctypes.c_int32()
    stream = torch.cuda.current_stream(rp.device)
    rc = lib.gc_color_noalloc(_ptr(rp), _ptr(ci), n, _ptr(prio), _ptr(out), ctypes.byref(nc),
                              ctypes.byref(rd), ctypes.c_void_p(stream.cuda_stream))
    return rc, out, nc.value, rd.value


@pytest.mark.parametrize("with_priority", [False, True])
def test_noalloc_matches_oracle_and_gc_color_ex_on_two_calls(gcpkg, with_priority):
    graphs = [gg.rmat(14, 8, gg.RMAT_B, 3), gg.gnm(10000, 50000, 1), gg.complete(300)]
    for g in graphs:
        rp, ci = _dev(g.rowptr), _dev(g.colidx)
        keys = prio = None
        if with_priority:
            keys = (gg.draws(5, 9, g.n) >> np.uint64(56)).astype(np.uint32)
            prio = _dev(keys.view(np.int32))
        want = oracle.iterative(g.rowptr, g.colidx, keys)
        ref = gcpkg.color(rp, ci, prio)  # gc_color_ex, library-managed workspace
        for _ in range(2):
            rc, out, nc, rd = _noalloc(gcpkg, rp, ci, prio)
            assert rc == gcpkg.GC_OK, gcpkg.strerror(rc)
            assert np.array_equal(out.cpu().numpy(), want.colors), g.name
            assert (nc, rd) == (want.ncolors, want.rounds), g.name
            assert torch.equal(out, ref.colors) and (nc, rd) == (ref.ncolors, ref.rounds), g.name


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
    want = oracle.iterative(small.rowptr, small.colidx)
    assert rc == gcpkg.GC_OK and np.array_equal(out.cpu().numpy(), want.colors) and rd == want.rounds


_CHILD = r"""
import ctypes, json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import graphgen as gg
import paper_1205_3809_gb300 as m
lib = m.library()
dev = torch.device("cuda:0")
torch.cuda.set_device(dev)
g = gg.rmat(14, 8, gg.RMAT_B, 3)
rp = torch.from_numpy(g.rowptr).to(dev)
ci = torch.from_numpy(g.colidx).to(dev)
keys = torch.from_numpy((gg.draws(5, 9, g.n) >> np.uint64(56)).astype(np.uint32).view(np.int32)).to(dev)
outs = [torch.empty(g.n, dtype=torch.int32, device=dev) for _ in range(4)]
s = torch.cuda.current_stream(dev)
def call(prio, out):
    nc, rd = ctypes.c_int32(), ctypes.c_int32()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = lib.gc_color_noalloc(p(rp), p(ci), g.n, None if prio is None else p(prio), p(out),
                              ctypes.byref(nc), ctypes.byref(rd), ctypes.c_void_p(s.cuda_stream))
    return rc, nc.value, rd.value
# first calls on this device: they look up the array's address and load the
# library's kernels (with and without a priority array); then measure
first = [call(None, outs[0]), call(keys, outs[1])]
torch.cuda.synchronize()
free0, _ = torch.cuda.mem_get_info()
res0, ws0 = torch.cuda.memory_reserved(), int(lib.gc_workspace_bytes())
later = [call(None, outs[2]), call(keys, outs[3]), call(None, outs[2])]
torch.cuda.synchronize()
free1, _ = torch.cuda.mem_get_info()
print(json.dumps({"rc": [r[0] for r in first + later], "free": [free0, free1],
                  "reserved": [res0, torch.cuda.memory_reserved()],
                  "workspace": [ws0, int(lib.gc_workspace_bytes())],
                  "same": bool(torch.equal(outs[0], outs[2]) and torch.equal(outs[1], outs[3]))}))
"""


def test_noalloc_allocates_nothing_in_a_fresh_process(gcpkg):
    """In a process of its own (nothing allocated by other tests): after the
    first calls, further calls change neither the device's free memory nor the
    library's workspace (which stays empty: no gc_color_ex call was made) nor
    torch's reserved memory."""
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["rc"] == [0] * 5
    assert d["workspace"] == [0, 0]
    assert d["reserved"][0] == d["reserved"][1]
    assert d["free"][0] == d["free"][1], d["free"]
    assert d["same"]
