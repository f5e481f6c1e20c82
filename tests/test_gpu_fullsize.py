"""The benchmark's full-size graphs, colored the way bench.py times them, against
the oracle's stored results (tests/golden/fullsize.json, written by
tests/golden/make_fullsize.py from graphgen/ and oracle/ only): colors (SHA-256
of the int32 array), color count, round count and |U_r| of every round, plus
what holds at any size (a proper coloring, 1 <= color <= degree + 1).

R-MAT-ER scale 22 (seed 2), R-MAT-B scale 24 (seed 3, the main workload, also
through the host-buffer entry point that the end-to-end leg times) and
R-MAT-G scale 23 (seed 5), index priority.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize.json")

CASES = {
    "rmat_er_s22_seed2": lambda: gg.rmat(22, 8, gg.RMAT_ER, 2),
    "rmat_b_s24_seed3": lambda: gg.rmat(24, 8, gg.RMAT_B, 3),
    "rmat_g_s23_seed5": lambda: gg.rmat(23, 8, gg.RMAT_G, 5),
}


@pytest.fixture(scope="module")
def gcpkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1205_3809_gb300 as m
    m.library()
    return m


def _sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).astype("<i4").tobytes()).hexdigest()


def _check(g, exp, colors, ncolors, rounds, sizes=None):
    assert _sha(colors) == exp["colors_sha256"]
    assert (ncolors, rounds) == (exp["ncolors"], exp["rounds"])
    if sizes is not None:
        assert list(map(int, sizes)) == exp["round_sizes"]
    assert np.all((colors >= 1) & (colors <= g.degrees + 1))
    src = np.repeat(np.arange(g.n, dtype=np.int32), g.degrees)
    assert not np.any(colors[src] == colors[g.colidx]), "monochromatic edge"


@pytest.mark.parametrize("name", list(CASES))
def test_full_size_matches_stored_oracle_result(gcpkg, name):
    exp = json.load(open(GOLDEN)).get(name)
    if exp is None:
        pytest.skip(f"no stored oracle result for {name}")
    g = CASES[name]()
    graph_sha = hashlib.sha256(g.rowptr.astype("<i4").tobytes() + g.colidx.astype("<i4").tobytes()).hexdigest()
    assert graph_sha == exp["graph_sha256"]
    rp, ci = torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.colidx).cuda()
    res = gcpkg.color(rp, ci, options={"telemetry": 1}, round_sizes=True)  # the bench's launch configuration
    _check(g, exp, res.colors.cpu().numpy(), res.ncolors, res.rounds, res.round_sizes)
    # the per-round device times cover every round
    ns = gcpkg.last_round_ns()
    assert ns.shape[0] == res.rounds and ns[0] == 0 and np.all(ns[1:] > 0)
    if name == "rmat_b_s24_seed3":
        # the end-to-end leg: pinned host buffers in, colors out
        h_out = torch.empty(g.n, dtype=torch.int32).pin_memory()
        r2 = gcpkg.color_host(torch.from_numpy(g.rowptr).pin_memory(), torch.from_numpy(g.colidx).pin_memory(),
                              out=h_out)
        _check(g, exp, h_out.numpy(), r2.ncolors, r2.rounds)
    del rp, ci
    gcpkg.release()
