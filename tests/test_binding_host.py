"""Host-side logic of the Python binding (no GPU): the batched input layout,
argument checks that fire before any device call, and the option arrays."""
import numpy as np
import pytest

import graphgen as gg

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gcpkg():
    import paper_1205_3809_gb300 as m
    try:
        m.build()
    except Exception as e:  # noqa: BLE001 - no nvcc: nothing here needs the library's kernels
        pytest.skip(f"cannot build libgc.so: {e}")
    return m


def test_pack_batch_layout(gcpkg):
    gs = [gg.path(4), gg.edgeless(0), gg.star(5, 0), gg.edgeless(2)]
    rp, ci, voff, eoff = gcpkg.pack_batch((g.rowptr, g.colidx) for g in gs)
    assert voff.tolist() == [0, 4, 4, 9, 11] and eoff.tolist() == [0, 6, 6, 14, 14]
    assert rp.dtype == np.int32 and ci.dtype == np.int32 and voff.dtype == np.int64
    assert rp.size == voff[-1] + len(gs) and ci.size == eoff[-1]
    for i, g in enumerate(gs):   # graph g's rowptr at voff[g] + g, its colidx at eoff[g]
        assert np.array_equal(rp[voff[i] + i: voff[i + 1] + i + 1], g.rowptr)
        assert np.array_equal(ci[eoff[i]: eoff[i + 1]], g.colidx)
    empty = gcpkg.pack_batch([])
    assert empty[0].size == 0 and empty[2].tolist() == [0] and empty[3].tolist() == [0]


def test_cpu_tensors_are_refused_before_any_device_call(gcpkg):
    g = gg.path(5)
    rp, ci = torch.from_numpy(g.rowptr), torch.from_numpy(g.colidx)
    with pytest.raises(ValueError, match="CUDA"):
        gcpkg.color(rp, ci)
    with pytest.raises(ValueError, match="G\\+1"):
        gcpkg.Batch(rp, ci, np.array([0, 5]), np.array([0, 4, 8]))
    with pytest.raises(ValueError, match="CUDA"):
        gcpkg.Batch(rp, ci, np.array([0, 5]), np.array([0, 8]))


def test_option_arrays(gcpkg):
    arr = gcpkg._options_array(gcpkg.BATCH_TUNE_CANDIDATES)
    assert len(arr) == len(gcpkg.BATCH_TUNE_CANDIDATES)
    modes = [arr[i].batch_mode for i in range(len(arr))]
    assert modes.count(2) == 3 and modes.count(1) == len(gcpkg.TUNE_CANDIDATES)
    assert arr[0].local_shared_bytes == 0 and arr[1].local_shared_bytes == 132 * 1024
    o = gcpkg._options({"batch_mode": 2, "local_thread_degree": -1})
    assert (o.batch_mode, o.local_thread_degree, o.small_max_degree) == (2, -1, 0)
    assert gcpkg._options(None) is None
