"""Write tests/golden/fullsize.json: the oracle's result on the full-size
synthetic workloads (index priority, and the shipped learned priority with
keys the oracle computes itself), stored as a SHA-256 of the int32 colors plus
ncolors, rounds, |U_r| of every round and the degree volume of every round
(the sum of deg(v) over U_r, which the bench's fixed byte accounting needs).
Calls only graphgen/ and oracle/.

    python tests/golden/make_fullsize.py [name ...]
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

WORKLOADS = {
    # R-MAT-ER scale 22 (4,194,304 vertices, edge factor 8), (0.25,0.25,0.25,0.25), seed 2
    "rmat_er_s22_seed2": lambda: gg.rmat(22, 8, gg.RMAT_ER, 2),
    # R-MAT-B scale 24 (16,777,216 vertices, edge factor 8), (0.55,0.15,0.15,0.15), seed 3
    "rmat_b_s24_seed3": lambda: gg.rmat(24, 8, gg.RMAT_B, 3),
    # R-MAT-G scale 23 (8,388,608 vertices, edge factor 8), (0.45,0.15,0.15,0.25), seed 5
    "rmat_g_s23_seed5": lambda: gg.rmat(23, 8, gg.RMAT_G, 5),
    # the larger R-MAT-B graphs of Table 4 (scales 25-27), same recipe, seed 3
    "rmat_b_s25_seed3": lambda: gg.rmat(25, 8, gg.RMAT_B, 3),
    "rmat_b_s26_seed3": lambda: gg.rmat(26, 8, gg.RMAT_B, 3),
    "rmat_b_s27_seed3": lambda: gg.rmat(27, 8, gg.RMAT_B, 3),
}


# learned priority: the shipped network's keys (computed by the oracle), then the same rounds
LEARNED = {"rmat_b_s24_seed3_learned": "rmat_b_s24_seed3", "rmat_g_s23_seed5_learned": "rmat_g_s23_seed5"}


def learned_keys(g):
    import json as _json
    from oracle import learned as L
    path = os.path.join(ROOT, "paper_1205_3809_gb300", "priority_mlp_rmat_g.json")
    params = np.asarray(_json.load(open(path))["params"], dtype=np.float32)
    return L.learned_keys(g.rowptr, g.colidx, params)


def degree_volumes(g, r):
    """vol_k = sum of deg(v) over U_k, k = 1..rounds (v is in U_k iff it settled in round k or later)."""
    by_round = np.bincount(r.settle_round, weights=g.degrees.astype(np.float64), minlength=r.rounds + 1)
    return [int(x) for x in np.cumsum(by_round[::-1])[::-1][1:r.rounds + 1]]


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).astype("<i4").tobytes()).hexdigest()


def main(names):
    path = os.path.join(ROOT, "tests", "golden", "fullsize.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    for name in names:
        g = WORKLOADS[LEARNED.get(name, name)]()
        t = time.time()
        keys = learned_keys(g) if name in LEARNED else None
        r = oracle.iterative(g.rowptr, g.colidx, keys)
        out[name] = {
            "n": g.n, "nnz": g.nnz,
            "graph_sha256": hashlib.sha256(g.rowptr.astype("<i4").tobytes()
                                           + g.colidx.astype("<i4").tobytes()).hexdigest(),
            "colors_sha256": sha(r.colors), "ncolors": r.ncolors, "rounds": r.rounds,
            "round_sizes": r.round_sizes.tolist(),
            "round_degree_volumes": degree_volumes(g, r),
            "oracle_seconds": round(time.time() - t, 1),
        }
        print(name, out[name]["ncolors"], out[name]["rounds"], out[name]["oracle_seconds"], flush=True)
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS) + list(LEARNED))
