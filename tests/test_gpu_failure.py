"""Failure paths, made to happen without faulting or hanging the GPU.

* A grid barrier that gives up: the testing option barrier_poll_limit makes
  the bounded wait between rounds stop after one poll, so blocks that are not
  the last to arrive record GC_ERR_TIMEOUT and leave; every wait in the kernel
  stays bounded.  The call must report GC_ERR_TIMEOUT, and the next call must
  be bit-exact with the oracle (the state a call uses is reset by the call).
* Device memory that cannot be had: the testing option workspace_limit_mb
  refuses to grow the workspace (the host-side stand-in for a failing
  cudaMalloc).  The call must report GC_ERR_OOM without touching the workspace
  it already holds, and a call without the limit must then succeed.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

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


def _exact(gcpkg, g, res):
    ref = oracle.iterative(g.rowptr, g.colidx)
    assert (res.ncolors, res.rounds) == (ref.ncolors, ref.rounds)
    assert np.array_equal(res.colors.cpu().numpy(), ref.colors)


def test_barrier_gives_up_then_next_call_is_exact(gcpkg):
    g = gg.rmat(16, 8, gg.RMAT_B, 3)  # dozens of rounds, hundreds of blocks per barrier
    rp, ci = _dev(g.rowptr), _dev(g.colidx)
    with pytest.raises(gcpkg.GcError) as e:
        gcpkg.color(rp, ci, options={"barrier_poll_limit": 1})
    assert e.value.code == gcpkg.GC_ERR_TIMEOUT
    _exact(gcpkg, g, gcpkg.color(rp, ci))
    # the other loop forms take no grid barrier, so the option changes nothing there
    _exact(gcpkg, g, gcpkg.color(rp, ci, options={"barrier_poll_limit": 1, "loop_mode": 1}))


def test_workspace_refused_then_recovers(gcpkg):
    g = gg.rmat(15, 8, gg.RMAT_B, 3)  # needs several MiB of workspace
    rp, ci = _dev(g.rowptr), _dev(g.colidx)
    gcpkg.release()
    with pytest.raises(gcpkg.GcError) as e:
        gcpkg.color(rp, ci, options={"workspace_limit_mb": 1})
    assert e.value.code == gcpkg.GC_ERR_OOM
    held = gcpkg.workspace_bytes()
    assert held < (1 << 20)  # nothing beyond the limit was allocated
    _exact(gcpkg, g, gcpkg.color(rp, ci))
    grown = gcpkg.workspace_bytes()
    assert grown > (1 << 20)
    # a workspace that is already big enough needs no growth: the limit does not bite
    _exact(gcpkg, g, gcpkg.color(rp, ci, options={"workspace_limit_mb": 1}))
    assert gcpkg.workspace_bytes() == grown


def test_host_entry_point_refused(gcpkg):
    g = gg.rmat(15, 8, gg.RMAT_B, 3)
    gcpkg.release()
    with pytest.raises(gcpkg.GcError) as e:
        gcpkg.color_host(g.rowptr, g.colidx, options={"workspace_limit_mb": 1})
    assert e.value.code == gcpkg.GC_ERR_OOM
    res = gcpkg.color_host(g.rowptr, g.colidx)
    ref = oracle.iterative(g.rowptr, g.colidx)
    assert (res.ncolors, res.rounds) == (ref.ncolors, ref.rounds)
    assert np.array_equal(np.asarray(res.colors), ref.colors)


@pytest.mark.parametrize("mode", [1, 2])
def test_batch_plan_refused(gcpkg, mode):
    gs = [gg.gnm(20000, 80000, 7 + i) for i in range(8)]  # several MiB of plan workspace
    rp_c, ci_c, voff, eoff = gcpkg.pack_batch((h.rowptr, h.colidx) for h in gs)
    rp_d, ci_d = _dev(rp_c), _dev(ci_c)
    with pytest.raises(gcpkg.GcError) as e:
        gcpkg.Batch(rp_d, ci_d, voff, eoff, options={"batch_mode": mode, "workspace_limit_mb": 1})
    assert e.value.code == gcpkg.GC_ERR_OOM
    b = gcpkg.Batch(rp_d, ci_d, voff, eoff, options={"batch_mode": mode})
    b.run()
    b.status()
    cols = b.colors.cpu().numpy()
    for i, h in enumerate(gs):
        ref = oracle.iterative(h.rowptr, h.colidx)
        assert np.array_equal(cols[voff[i]:voff[i + 1]], ref.colors)
    b.close()
