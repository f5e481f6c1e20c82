"""Host side of the autotuner: the degree signature and the JSON cache (no GPU)."""
import json

import numpy as np

import paper_1205_3809_gb300 as gc


def test_degree_signature_shape():
    sig = gc._degree_signature(np.array([0, 1, 1, 3, 7, 8]))
    # n, sum, max, then shares of log2(deg+1) buckets 0 (deg 0), 1 (deg 1-2), 2 (3-6), 3 (7-14)
    assert sig[:3] == [6, 20, 8]
    assert sig[3:] == [round(1 / 6, 2), round(2 / 6, 2), round(1 / 6, 2), round(2 / 6, 2)]
    assert gc._degree_signature(np.zeros(0)) == [0, 0, 0]


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("GC_TUNE_CACHE", str(path))
    assert gc._cache_io("k") is None
    gc._cache_io("k", {"best": {"small_max_degree": 8}, "table": []})
    gc._cache_io("k2", {"best": {}, "table": []})
    assert gc._cache_io("k")["best"] == {"small_max_degree": 8}
    assert set(json.load(open(path))) == {"k", "k2"}
    path.write_text("not json")
    assert gc._cache_io("k") is None          # a damaged cache is ignored, not fatal


def test_candidates_are_valid_options():
    for c in gc.TUNE_CANDIDATES:
        assert 1 <= c["small_max_degree"] <= c["medium_max_degree"] <= 256
        assert c["small_max_degree"] <= 32 and c["block_threads"] in (128, 256)
    o = gc._options_array(gc.TUNE_CANDIDATES[:2])
    assert o[1].medium_max_degree == gc.TUNE_CANDIDATES[1]["medium_max_degree"]


def test_pack_batch_layout():
    a = (np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32))
    e = (np.array([0], np.int32), np.zeros(0, np.int32))
    b = (np.array([0, 0, 0, 0], np.int32), np.zeros(0, np.int32))
    rp, ci, voff, eoff = gc.pack_batch([a, e, b])
    assert rp.tolist() == [0, 1, 2, 0, 0, 0, 0, 0]
    assert ci.tolist() == [1, 0]
    assert voff.tolist() == [0, 2, 2, 5] and eoff.tolist() == [0, 2, 2, 2]
