"""Train the vertex-priority network on the GPU and write its parameter file.

Training set: R-MAT-G graphs (quadrants 0.45/0.15/0.15/0.25, edge factor 8,
Sec. 4.1), scales 14 to 18 in turn, seeds 10000 + i.  Labels: the oracle
computes both orderings the paper cites for Greedy (Sec. 1, Sec. 3.1),
smallest-last (Matula and Beck) and largest-first, colors the graph with
serial Greedy in each, and the ordering that uses fewer colors (smallest-last
on a tie) gives every vertex its target, log2(1 + its position in that
ordering).  Features are computed by the library's GPU kernel
and the network is trained by its GPU kernels (gc_mlp_train_step: fused
gradient of the mean squared error, then Adam).

Evaluation (written into the file): colors and rounds of index priority and
of the learned priority on R-MAT-G scale 23 seed 5 and R-MAT-B scale 24 seed 3,
beside serial Greedy in smallest-last and largest-first order (oracle).

Usage: python tests/train_priority_mlp.py --out paper_1205_3809_gb300/priority_mlp_rmat_g.json
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402


def _targets(job):
    """Worker: targets of one training graph and the ordering that labelled it
    (oracle, one thread)."""
    scale, seed = job
    from oracle import learned as L
    g = gg.rmat(scale, 8, gg.RMAT_G, seed)
    return L.ordering_targets(g.rowptr, g.colidx)


def _greedy_colors(job):
    """Worker: serial Greedy colors in smallest-last and largest-first order."""
    kind, scale, seed = job
    import oracle
    abcd = {"G": gg.RMAT_G, "B": gg.RMAT_B}[kind]
    g = gg.rmat(scale, 8, abcd, seed)
    sl, _ = oracle.smallest_last_order(g.rowptr, g.colidx)
    lf = oracle.largest_first_order(g.rowptr)
    return {"smallest_last": oracle.greedy(g.rowptr, g.colidx, sl)[1],
            "largest_first": oracle.greedy(g.rowptr, g.colidx, lf)[1]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=512)
    ap.add_argument("--min-scale", type=int, default=14)
    ap.add_argument("--max-scale", type=int, default=18)
    ap.add_argument("--seed-base", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--init-seed", type=int, default=1)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--no-eval", action="store_true")
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_1205_3809_gb300", "priority_mlp_rmat_g.json"))
    a = ap.parse_args()

    gg.build()
    import oracle
    oracle.build()
    os.environ.setdefault("OMP_NUM_THREADS", "1")  # inherited by the spawned workers
    ctx = mp.get_context("spawn")
    nsc = a.max_scale - a.min_scale + 1
    jobs = [(a.min_scale + i % nsc, a.seed_base + i) for i in range(a.graphs)]
    evals = [("G", 23, 5), ("B", 24, 3)]
    t0 = time.time()
    with ctx.Pool(a.workers) as pool:
        greedy_async = None if a.no_eval else pool.map_async(_greedy_colors, evals)
        labelled = pool.map(_targets, jobs, chunksize=1)
        targets = [t for t, _ in labelled]
        labels = {"smallest_last": 0, "largest_first": 0}
        for _, lab in labelled:
            labels[lab["ordering"]] += 1
        print("labels:", labels, flush=True)
        t_labels = time.time() - t0
        os.environ.pop("OMP_NUM_THREADS", None)

        import torch
        import paper_1205_3809_gb300 as gc
        dev = torch.device("cuda:0")
        feats = []
        for (scale, seed), t in zip(jobs, targets):
            g = gg.rmat(scale, 8, gg.RMAT_G, seed)
            f = gc.features(torch.from_numpy(g.rowptr).to(dev), torch.from_numpy(g.colidx).to(dev))
            assert f.shape[0] == t.shape[0]
            feats.append(f.cpu().numpy())
        x = np.concatenate(feats)
        t = np.concatenate(targets)
        n = x.shape[0]
        perm = gg.permutation(n, a.seed_base)
        xd = torch.from_numpy(x[perm]).to(dev)
        td = torch.from_numpy(t[perm]).to(dev)
        del x, feats

        d = gg.draws(a.init_seed, 7, gc.MLP_PARAMS)
        u = (d >> np.uint64(11)).astype(np.float64) / float(1 << 53)
        fan_in = np.concatenate([np.full(32 * 6, 6), np.full(32, 6), np.full(32 * 32, 32), np.full(32, 32),
                                 np.full(32, 32), [32]]).astype(np.float64)
        init = ((2.0 * u - 1.0) * np.sqrt(3.0 / fan_in)).astype(np.float32)
        tr = gc.MlpTrainer(torch.from_numpy(init).to(dev), lr=a.lr)
        steps_per_epoch = max(1, n // a.batch)
        history = []
        t1 = time.time()
        for ep in range(a.epochs):
            tr.lr = a.lr * (0.5 * (1.0 + np.cos(np.pi * ep / a.epochs)))
            acc = torch.zeros(1, dtype=torch.float64, device=dev)
            for s in range(steps_per_epoch):
                off = s * a.batch
                acc += tr.step(xd[off:off + a.batch], td[off:off + a.batch]).double()
            history.append(float(acc.item()) / (steps_per_epoch * a.batch))
            print(f"epoch {ep}: lr {tr.lr:.2e} mse {history[-1]:.5f}", flush=True)
        torch.cuda.synchronize()
        t_train = time.time() - t1
        params = tr.params.cpu().numpy()

        ev = {}
        if not a.no_eval:
            greedy = greedy_async.get()
            for (kind, scale, seed), gr in zip(evals, greedy):
                abcd = {"G": gg.RMAT_G, "B": gg.RMAT_B}[kind]
                g = gg.rmat(scale, 8, abcd, seed)
                rp, ci = torch.from_numpy(g.rowptr).to(dev), torch.from_numpy(g.colidx).to(dev)
                plain = gc.color(rp, ci)
                learned = gc.color_learned(rp, ci, tr.params)
                ev[f"rmat_{kind.lower()}_s{scale}_seed{seed}"] = {
                    "plain": {"ncolors": plain.ncolors, "rounds": plain.rounds},
                    "learned": {"ncolors": learned.ncolors, "rounds": learned.rounds},
                    "greedy_serial": gr}
                print(kind, scale, ev[f"rmat_{kind.lower()}_s{scale}_seed{seed}"], flush=True)

    doc = {
        "format": "gc-priority-mlp-1",
        "layout": "W1[32][6] | b1[32] | W2[32][32] | b2[32] | W3[32] | b3 (float32)",
        "features": "L(deg), floor(log2(1+deg)), L(floor(sum nbr deg / deg)), L(max nbr deg), "
                    "L(sum nbr deg), L(min nbr deg); L = Mitchell log2(1+x), 16 fraction bits",
        "target": ("log2(1 + position in the ordering, smallest-last or largest-first (oracle), whose serial "
                   "Greedy coloring of the graph uses fewer colors; smallest-last on a tie) "
                   "(smaller = colored earlier)"),
        "labels": labels,
        "training": {"graphs": a.graphs, "family": "R-MAT-G (0.45,0.15,0.15,0.25) edge factor 8",
                     "scales": [a.min_scale, a.max_scale], "seeds": [a.seed_base, a.seed_base + a.graphs - 1],
                     "samples": int(n), "epochs": a.epochs, "batch": a.batch, "lr": a.lr,
                     "lr_schedule": "cosine per epoch", "optimizer": "Adam(0.9, 0.999, 1e-8)",
                     "init": "uniform(+-sqrt(3/fan_in)), SplitMix64 seed %d stream 7" % a.init_seed,
                     "mse_per_epoch": history, "label_seconds": round(t_labels, 1),
                     "train_seconds": round(t_train, 2)},
        "eval": ev,
        "params": [float(v) for v in params],
    }
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    with open(a.out, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", a.out, flush=True)


if __name__ == "__main__":
    main()
