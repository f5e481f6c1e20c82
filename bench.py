#!/usr/bin/env python
"""Benchmark: edges colored per second and colors used on R-MAT-B scale 24.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one full coloring (gc_color through the C ABI: setup scan, round 1,
every later round until the worklist is empty) of the synthetic R-MAT-B graph
(scale 24, edge factor 8, quadrant probabilities (0.55, 0.15, 0.15, 0.15),
seed 3, ids permuted), with the graph already resident in HBM.  The L2 is
flushed (256 MB write) before every step, outside the step's CUDA events.
Prints one JSON line (rank 0).  Multi-GPU runs color one replica per rank
("replicas only": the method has no exchange step to shard).

Beside it, the same line carries every other configuration of the benchmark
set, each timed the same way with its own clock record and roofline: the
learned priority on the same graph, G(n=10,000, m=50,000), R-MAT-ER scale 22,
the batch of 4,096 graphs, and R-MAT-G scale 23 with index and learned
priority (`configs`).

--impl reference times the CPU oracle (plain single-threaded C, test
infrastructure) on the host cores, on bounded samples of the same workload.
"""
import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen as gg  # noqa: E402

METRIC = "edges colored/sec and colors used, R-MAT-B scale 24 on 1 GB300, learned vs plain"
WORKLOAD = ("R-MAT-B scale 24: 16,777,216 vertices, edge factor 8, (a,b,c,d)=(0.55,0.15,0.15,0.15), "
            "seed 3, duplicates and self loops removed, ids permuted; symmetric int32 CSR; "
            "plain index priority; synchronous rounds")
SCALE, EF, ABCD, SEED = 24, 8, gg.RMAT_B, 3
# bounded CPU samples of the same recipe at smaller scale
CPU_BASELINE_SCALE = 22
REFERENCE_STEP_SCALE = 20

# Random 16-bit gathers from an L2-resident table, driven by a streamed int32
# index array (`python bench.py --measure-l2-ceiling`, GB300).
L2_GATHER_CEILING = 208.0  # G gathers/s, 32 MB table (the scale-24 color state)
L2_SECTOR_CEILING = 234.0  # G sectors/s: the same run counted in L2 sectors (gathers + index stream)
# Per-launch ncu counters of the rounds kernel on the bench workload, with the
# command that took them and the code they belong to.
PROFILE_JSON = os.path.join(ROOT, "profiles", "rounds_persistent_kernel_rmat_b_s24.json")
GOLDEN_JSON = os.path.join(ROOT, "tests", "golden", "fullsize.json")

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def cpu_model() -> str:
    """The host CPU's model string, as far as the OS reports it."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine() or "unknown"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), \
        int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value of x over all ranks (each rank times its own replica; the
    job is as slow as its slowest rank).  One all-reduce on an initialised group."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, steps: int, world: int, max_seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * steps * units_per_rank / max_seconds


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (every 100 ms) while the timed region runs."""

    def __init__(self, gpu_id):
        self.proc = None
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self, t0, t1):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        for t, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or not (t0 - 0.15 <= t <= t1 + 0.15):
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(REASONS, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- oracle leg

def oracle_rate(scale, runs=1):
    """Single-threaded CPU oracle on R-MAT-B at `scale` (same recipe): edges/s."""
    import oracle
    oracle.build()
    g = gg.rmat(scale, EF, ABCD, SEED)
    times = []
    for _ in range(runs):
        t = time.perf_counter()
        r = oracle.iterative(g.rowptr, g.colidx)
        times.append(time.perf_counter() - t)
    return g, r, times


def batch_cpu_baseline(graphs, stride=64):
    """The single-threaded oracle on every `stride`-th graph of a batch (a bounded
    sample of the same workload): edges/s, with what the sample was."""
    import oracle
    oracle.build()
    sample = graphs[::stride]
    m = sum(g.m for g in sample)
    t = time.perf_counter()
    for g in sample:
        oracle.iterative(g.rowptr, g.colidx)
    s = time.perf_counter() - t
    return {"value": m / s if s > 0 else None, "unit": "edges/s", "cores": 1, "kind": "oracle",
            "sample": f"every {stride}th graph of the batch: {len(sample)} graphs, {m} edges, {s:.1f} s",
            "host": {"cpus": os.cpu_count(), "machine": platform.machine(), "model": cpu_model()}}


def paper_async_openmp(scale):
    """The paper's own multicore method (asynchronous Algorithm 2, OpenMP, all host
    cores) on the CPU-baseline graph, in a child process with a time limit;
    checked for validity only.  Never fails the bench: a problem is reported."""
    try:
        r = subprocess.run([sys.executable, "-m", "oracle.async_omp", "--scale", str(scale), "--seed", "3"],
                           cwd=ROOT, capture_output=True, text=True, timeout=300)
        if r.returncode != 0:
            return {"unavailable": f"exit {r.returncode}: {r.stderr.strip()[-200:]}"}
        out = json.loads(r.stdout.strip().splitlines()[-1])
        out["note"] = ("Algorithm 2 as the paper runs it on multicore CPUs: asynchronous Phase 1, "
                       "schedule-dependent, validity-checked")
        return out
    except (subprocess.TimeoutExpired, ValueError, IndexError, OSError) as e:
        return {"unavailable": f"{type(e).__name__}: {e}"[:200]}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    g = gg.rmat(REFERENCE_STEP_SCALE, EF, ABCD, SEED)
    for _ in range(args.warmup):
        oracle.iterative(g.rowptr, g.colidx)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        r = oracle.iterative(g.rowptr, g.colidx)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = g.m * args.steps / total
    sample = (f"R-MAT-B scale {REFERENCE_STEP_SCALE} (same recipe: edge factor 8, seed 3), "
              f"{g.m} edges, one full oracle run per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "ncolors": r.ncolors, "rounds": r.rounds,
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------- roofline bits

def algorithmic_bytes_rounds(sizes, vols, elem):
    """Bytes one launch of the rounds kernel must move (rounds k >= 2).

    sizes[k-1] = |U_k|, vols[k-1] = A_k, the active-list entries round k reads
    (A_2 = full rows; later rounds read only neighbours not yet settled).
    Per round k: active list 4*A_k + neighbour colors elem*A_k + worklist
    tuples 16|U_k| + own color elem|U_k| + static masks 32|U_k| (k >= 3);
    writes: survivors 4*A_{k+1}, next tuples 16|U_{k+1}|, static masks
    32|U_{k+1}|, next color elem|U_k|, final int32 color 4 per settled vertex.
    """
    total = 0
    R = len(sizes)
    for k in range(2, R + 1):
        u, a = int(sizes[k - 1]), int(vols[k - 1])
        un = int(sizes[k]) if k < R else 0
        an = int(vols[k]) if k < R else 0
        reads = 4 * a + elem * a + 16 * u + elem * u + (32 * u if k >= 3 else 0)
        writes = 4 * an + 16 * un + 32 * un + elem * u + 4 * (u - un)
        total += reads + writes
    return total


def fixed_bytes_rounds(sizes, degree_vols):
    """Bytes of rounds k >= 2 under the fixed full-row accounting, the same for
    every implementation of the method: per round k over W = U_k, the worklist
    4|W|, the rowptr pair 8|W|, colidx and the neighbours' colors 8 vol(W)
    (vol(W) = sum of deg(v) over W, whole rows), the own color 4|W| and the
    appends of the next round 8|U_{k+1}|."""
    total = 0
    R = len(sizes)
    for k in range(2, R + 1):
        u, un = int(sizes[k - 1]), (int(sizes[k]) if k < R else 0)
        total += 16 * u + 8 * int(degree_vols[k - 1]) + 8 * un
    return total


def fixed_bytes_call(n, nnz, sizes, degree_vols):
    """Fixed whole-row bytes of a whole coloring: pass 1 over V (rowptr 4(n+1),
    colidx 4 nnz, own color 4n, appends 8|U_2|), the rounds k >= 2
    (fixed_bytes_rounds), color init 4n and the max reduction 4n."""
    u2 = int(sizes[1]) if len(sizes) > 1 else 0
    return 4 * (n + 1) + 4 * nnz + 4 * n + 8 * u2 + fixed_bytes_rounds(sizes, degree_vols) + 8 * n


def stored_degree_volumes(n, nnz, sizes):
    """Per-round degree volumes of this workload as the oracle computed them
    (stored with its other full-size results by tests/golden/make_fullsize.py),
    when the run's |U_k| are the stored ones; else None."""
    if not os.path.exists(GOLDEN_JSON):
        return None
    for entry in json.load(open(GOLDEN_JSON)).values():
        if (entry.get("n") == n and entry.get("nnz") == nnz and entry.get("round_sizes") == [int(x) for x in sizes]
                and "round_degree_volumes" in entry):
            return entry["round_degree_volumes"]
    return None


def algorithmic_bytes_batch(N, NNZ, sizes, vols, elem):
    """Bytes one batched run must move, all of its kernels together.

    Rebase: colidx read and written (8*NNZ).  Pass 1 (round 1 and round 2's
    Phase 1): rowptr 4(N+1) and colidx 4*NNZ read; both color buffers
    2*elem*N, final color and settle round 8 per vertex settled in round 1,
    a tuple 16|U_2| written.  Rounds k >= 2: algorithmic_bytes_rounds, plus
    the settle round 4 per vertex they settle.  Reduce: final colors and
    settle rounds read, 8N.
    """
    u2 = int(sizes[1]) if len(sizes) > 1 else 0
    rebase = 8 * NNZ
    pass1 = 4 * (N + 1) + 4 * NNZ + 2 * elem * N + 8 * (N - u2) + 16 * u2
    rounds = algorithmic_bytes_rounds(sizes, vols, elem) + 4 * u2
    reduce = 8 * N
    return rebase + pass1 + rounds + reduce


def algorithmic_bytes_batch_blocks(N, sizes, vols):
    """Bytes one batched run with one thread block per graph must move to and
    from device memory (its colors live in shared memory).

    Round k reads the rows of U_k: colidx 4*vol_k and rowptr 8 per vertex, and
    (k >= 2) the worklist 4|U_k|; it appends U_{k+1} with new colors (8 per
    vertex) and reads them back once for the color update.  The final colors
    are written once, 4N.  vol_1 is nnz (every row), |U_1| = N.
    """
    total = 4 * N
    R = len(sizes)
    for k in range(1, R + 1):
        u, a = int(sizes[k - 1]), int(vols[k - 1])
        un = int(sizes[k]) if k < R else 0
        total += 4 * a + 8 * u + (4 * u if k >= 2 else 0) + 16 * un
    return total


def gathers_rounds(vols):
    """Random neighbour-color reads of the rounds kernel (one per active entry)."""
    return int(sum(int(x) for x in vols[1:]))


def kernel_code_hash(path: str) -> str:
    """SHA-256 of a CUDA source's code: comments and blank lines removed, so a
    change to the text around the code does not void a profile of the code."""
    import re
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    lines = [ln.rstrip() for ln in src.splitlines() if ln.strip()]
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def load_profile(kernel_src, path=PROFILE_JSON):
    """The per-launch ncu counters of the rounds kernel (with the command that
    took them), or {} if that file is missing or the kernel's code has changed
    since the capture."""
    if not os.path.exists(path):
        return {}
    d = json.load(open(path))
    return d if d.get("kernel_code_sha256") == kernel_code_hash(kernel_src) else {}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# -------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    import paper_1205_3809_gb300 as gcpkg

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (there is no CPU path)")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    gcpkg.library()

    t = time.time()
    g = gg.rmat(args.scale, EF, ABCD, SEED)
    log(f"[rank {rank}] graph n={g.n} m={g.m} maxdeg={g.max_degree} generated in {time.time() - t:.1f}s")
    rp = torch.from_numpy(g.rowptr).to(dev)
    ci = torch.from_numpy(g.colidx).to(dev)
    out = torch.empty(g.n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    opts = {"telemetry": 1}

    def step():
        return gcpkg.color(rp, ci, out=out, options=opts, stream=stream)

    for _ in range(args.warmup):
        flush.zero_()
        res = step()
    torch.cuda.synchronize(dev)

    props = torch.cuda.get_device_properties(dev)
    gpu_id = "GPU-" + str(getattr(props, "uuid", "")) if getattr(props, "uuid", None) else str(local)
    sampler = ClockSampler(gpu_id)
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.time()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kernel_ms = []
    launches = 0
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        res = step()
        ends[i].record(stream)
        kernel_ms.append(gcpkg.last_phase_ms()[2])
        launches += gcpkg.last_launch_count()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    t1 = time.time()
    clocks = sampler.stop(t0, t1)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_s = sum(step_ms) / 1e3
    total_s = max_over_ranks(total_s, world, dev)
    value = job_rate(g.m, args.steps, world, total_s)

    sizes, vols = gcpkg.last_round_stats()
    elem = 2  # 16-bit color state (the library restarts with 32 bits only past 32767 colors)
    active_bytes = algorithmic_bytes_rounds(sizes, vols, elem)
    degree_vols = stored_degree_volumes(g.n, g.nnz, sizes)
    alg_bytes = fixed_bytes_rounds(sizes, degree_vols) if degree_vols else active_bytes
    kms = statistics.mean(kernel_ms)
    achieved = alg_bytes / (kms / 1e3) / 1e9
    peak, peak_kind = peaks()
    prof = load_profile(os.path.join(ROOT, "paper_1205_3809_gb300", "csrc", "gc_device.cuh"))
    per_launch = prof.get("per_launch", {})
    traffic = (per_launch["dram__bytes_read.sum"] + per_launch["dram__bytes_write.sum"]
               if "dram__bytes_read.sum" in per_launch and "dram__bytes_write.sum" in per_launch else None)
    sectors = per_launch.get("lts__t_sectors.sum")
    gathers = gathers_rounds(vols)
    gather_rate = gathers / (kms / 1e3) / 1e9

    # end to end through the host-buffer entry point (pinned buffers)
    e2e = None
    if not args.no_e2e:
        h_rp = torch.from_numpy(g.rowptr).pin_memory()
        h_ci = torch.from_numpy(g.colidx).pin_memory()
        h_out = torch.empty(g.n, dtype=torch.int32).pin_memory()
        for _ in range(2):
            gcpkg.color_host(h_rp, h_ci, out=h_out, stream=stream)
        torch.cuda.synchronize(dev)
        e_ms = []
        for _ in range(max(3, args.steps // 5)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r2 = gcpkg.color_host(h_rp, h_ci, out=h_out, stream=stream)
            b.record(stream)
            b.synchronize()
            e_ms.append(a.elapsed_time(b))
        assert np.array_equal(h_out.numpy(), out.cpu().numpy()) and r2.ncolors == res.ncolors
        e2e = {"value": g.m / (statistics.mean(e_ms) / 1e3), "unit": "edges/s",
               "h2d_bytes_per_step": 4 * (g.n + 1) + 4 * g.nnz, "d2h_bytes_per_step": 4 * g.n + 8,
               "ms_per_step": statistics.mean(e_ms)}

    learned = None if args.no_learned else measure_learned(gcpkg, rp, ci, g, flush, stream, args)
    asynchronous = None if args.no_learned else measure_async(gcpkg, rp, ci, g, flush, stream, args)
    configs = None
    if not args.no_configs and world == 1:
        del rp, ci
        torch.cuda.empty_cache()
        configs = measure_configs(gcpkg, flush, stream, args, gpu_id)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cg, cr, ct = oracle_rate(CPU_BASELINE_SCALE)
        import oracle
        t = time.perf_counter()
        _, greedy_colors = oracle.greedy(cg.rowptr, cg.colidx)
        greedy_s = time.perf_counter() - t
        cpu = {"value": cg.m / ct[0], "unit": "edges/s", "cores": 1, "kind": "oracle",
               "sample": (f"R-MAT-B scale {CPU_BASELINE_SCALE} (same recipe, seed 3): {cg.m} edges, "
                          f"one full run, {ct[0]:.1f} s, {cr.rounds} rounds, {cr.ncolors} colors"),
               "host": {"cpus": os.cpu_count(), "machine": platform.machine(), "model": cpu_model()},
               "greedy_serial": {"value": cg.m / greedy_s, "unit": "edges/s", "seconds": round(greedy_s, 3),
                                 "ncolors": greedy_colors,
                                 "note": "Algorithm 1 in index order, one core (the sequential baseline)"},
               "paper_async_openmp": paper_async_openmp(CPU_BASELINE_SCALE)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "ncolors": res.ncolors, "rounds": res.rounds,
            "config": {"workload": WORKLOAD if args.scale == SCALE else
                       WORKLOAD.replace("scale 24", f"scale {args.scale}").replace("16,777,216", f"{g.n:,}"),
                       "n": g.n, "m": g.m, "max_degree": g.max_degree,
                       "priority": "index (plain)", "loop": "persistent cooperative launch",
                       "color_state_bits": 8 * elem,
                       "l2": "inputs larger than L2 (colidx 1.07 GB) and L2 flushed (256 MB write) "
                             "before every step, outside its events",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "kernel": "rounds_persistent_kernel",
                         "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "traffic_source": ({"file": os.path.relpath(PROFILE_JSON, ROOT),
                                             "command": prof.get("command"), "workload": prof.get("workload")}
                                            if traffic is not None else None),
                         "algorithmic_bytes": alg_bytes, "kernel_ms": kms,
                         "accounting": ("whole rows: fixed per-round bytes of the method (worklist, rowptr, "
                                        "colidx and neighbour colors of every row of U_k, own color, appends)"
                                        if degree_vols else "active entries (this implementation's reads)"),
                         "active_entries": {"algorithmic_bytes": active_bytes,
                                            "achieved": active_bytes / (kms / 1e3) / 1e9,
                                            "frac": active_bytes / (kms / 1e3) / 1e9 / peak},
                         "l2_gathers": {"count": gathers, "achieved_G_per_s": gather_rate,
                                        "ceiling_G_per_s": L2_GATHER_CEILING,
                                        "frac": gather_rate / L2_GATHER_CEILING},
                         "l2_sectors": None if sectors is None else {
                             "count": sectors, "achieved_G_per_s": sectors / (kms / 1e3) / 1e9,
                             "ceiling_G_per_s": L2_SECTOR_CEILING,
                             "frac": sectors / (kms / 1e3) / 1e9 / L2_SECTOR_CEILING,
                             "source": os.path.relpath(PROFILE_JSON, ROOT)}},
            "cpu_baseline": cpu,
            "learned": learned,
            "asynchronous": asynchronous,
            "configs": configs,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def config_roofline(n, nnz, sizes, vols, kms):
    """Roofline of the rounds kernel for one configuration: the fixed whole-row
    bytes when the oracle's degree volumes of that workload are stored, else
    this implementation's active-entry bytes (said in `accounting`)."""
    peak, peak_kind = peaks()
    degree_vols = stored_degree_volumes(n, nnz, sizes)
    alg = fixed_bytes_rounds(sizes, degree_vols) if degree_vols else algorithmic_bytes_rounds(sizes, vols, 2)
    achieved = alg / (kms / 1e3) / 1e9 if kms > 0 else None
    return {"bound": "hbm", "kernel": "rounds_persistent_kernel", "achieved": achieved, "peak": peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": None if achieved is None else achieved / peak,
            "traffic": None, "algorithmic_bytes": alg, "kernel_ms": kms,
            "accounting": ("whole rows: fixed per-round bytes of the method (oracle degree volumes)"
                           if degree_vols else "active entries (this implementation's reads)")}


def time_config(gcpkg, g, workload, flush, stream, steps, warmup, gpu_id, learned=False):
    """One configuration of the benchmark set, timed like the main line: CUDA
    events around each step on the launching stream, L2 flushed before each
    step outside the events, nvidia-smi clocks sampled over the timed steps.
    learned: the step is features -> network -> keys -> coloring under the keys
    (the shipped network), as one step."""
    import torch
    dev = flush.device
    rp = torch.from_numpy(g.rowptr).to(dev)
    ci = torch.from_numpy(g.colidx).to(dev)
    out = torch.empty(g.n, dtype=torch.int32, device=dev)
    opts = {"telemetry": 1}
    if learned:
        params = gcpkg.load_priority_model(device=dev)
        feats = torch.empty((g.n, 6), dtype=torch.float32, device=dev)
        scores = torch.empty(g.n, dtype=torch.float32, device=dev)
        keys = torch.empty(g.n, dtype=torch.int32, device=dev)

    def step():
        if learned:
            gcpkg.features(rp, ci, out=feats, stream=stream)
            gcpkg.mlp_forward(params, feats, out=scores, stream=stream)
            gcpkg.priority_keys(scores, out=keys, stream=stream)
            return gcpkg.color(rp, ci, keys, out=out, options=opts, stream=stream)
        return gcpkg.color(rp, ci, out=out, options=opts, stream=stream)

    for _ in range(warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(gpu_id)
    time.sleep(0.3)
    t0 = time.time()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kernel_ms, launches = [], 0
    for a, e in evs:
        flush.zero_()
        a.record(stream)
        res = step()
        e.record(stream)
        kernel_ms.append(gcpkg.last_phase_ms()[2])
        launches += gcpkg.last_launch_count() + (3 if learned else 0)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop(t0, time.time())
    ms = statistics.mean(a.elapsed_time(e) for a, e in evs)
    sizes, vols = gcpkg.last_round_stats()
    kms = statistics.mean(kernel_ms)
    return {"workload": workload, "n": g.n, "m": g.m, "max_degree": g.max_degree,
            "priority": "learned (features, network, keys inside the step)" if learned else "index (plain)",
            "value": g.m / (ms / 1e3), "unit": "edges/s", "ms_per_step": ms, "steps": steps,
            "ncolors": res.ncolors, "rounds": res.rounds, "gpu_launches": launches,
            "roofline": config_roofline(g.n, g.nnz, sizes, vols, kms), "clocks": clocks}


def measure_configs(gcpkg, flush, stream, args, gpu_id):
    """The other configurations of the benchmark set, each timed on its own."""
    steps, warmup = max(5, args.steps // 2), 3
    out = {}
    t = time.time()
    g = gg.gnm(10000, 50000, 1)
    out["c0_gnm_10k_50k"] = time_config(gcpkg, g, "G(n=10,000, m=50,000), seed 1; index priority", flush, stream,
                                        steps, warmup, gpu_id)
    g = gg.rmat(22, EF, gg.RMAT_ER, 2)
    out["c1_rmat_er_s22"] = time_config(
        gcpkg, g, "R-MAT-ER scale 22: 4,194,304 vertices, edge factor 8, (0.25,0.25,0.25,0.25), seed 2, "
        "ids permuted; index priority", flush, stream, steps, warmup, gpu_id)
    g = gg.rmat(23, EF, gg.RMAT_G, 5)
    wl = "R-MAT-G scale 23: 8,388,608 vertices, edge factor 8, (0.45,0.15,0.15,0.25), seed 5, ids permuted"
    c4 = {"plain": time_config(gcpkg, g, wl + "; index priority", flush, stream, steps, warmup, gpu_id)}
    if os.path.exists(gcpkg.PRIORITY_MODEL):
        c4["learned"] = time_config(gcpkg, g, wl + "; learned priority", flush, stream, steps, warmup, gpu_id,
                                    learned=True)
        c4["learned_no_more_colors_than_plain"] = c4["learned"]["ncolors"] <= c4["plain"]["ncolors"]
    out["c4_rmat_g_s23"] = c4
    del g
    log(f"configs c0/c1/c4 in {time.time() - t:.1f}s")
    if not args.no_batch:
        t = time.time()
        out["c3_batched_4096"] = measure_batched(gcpkg, args.batch_graphs, flush, stream, steps, warmup, gpu_id,
                                                 options={}, use_graph=True, e2e_steps=3)
        log(f"config c3 in {time.time() - t:.1f}s")
    return out


def measure_learned(gcpkg, rp, ci, g, flush, stream, args):
    """The learned-priority form on the same graph: features -> network -> keys ->
    coloring under those keys, timed as one step with CUDA events on the
    launching stream (L2 flushed before each step), phases split by events."""
    import torch
    if not os.path.exists(gcpkg.PRIORITY_MODEL):
        return {"unavailable": "no trained model file"}
    params = gcpkg.load_priority_model(device=rp.device)
    n = g.n
    feats = torch.empty((n, 6), dtype=torch.float32, device=rp.device)
    scores = torch.empty(n, dtype=torch.float32, device=rp.device)
    keys = torch.empty(n, dtype=torch.int32, device=rp.device)
    lout = torch.empty(n, dtype=torch.int32, device=rp.device)

    def step(ev=None):
        gcpkg.features(rp, ci, out=feats, stream=stream)
        if ev:
            ev[1].record(stream)
        gcpkg.mlp_forward(params, feats, out=scores, stream=stream)
        if ev:
            ev[2].record(stream)
        gcpkg.priority_keys(scores, out=keys, stream=stream)
        if ev:
            ev[3].record(stream)
        return gcpkg.color(rp, ci, keys, out=lout, stream=stream)

    for _ in range(3):
        flush.zero_()
        res = step()
    torch.cuda.synchronize()
    k = max(5, args.steps // 3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(k)]
    launches = 0
    for i in range(k):
        flush.zero_()
        evs[i][0].record(stream)
        res = step(evs[i])
        evs[i][4].record(stream)
        launches += 3 + gcpkg.last_launch_count()
    torch.cuda.synchronize()
    tot = [e[0].elapsed_time(e[4]) for e in evs]
    phase = [statistics.mean(e[j].elapsed_time(e[j + 1]) for e in evs) for j in range(4)]
    ms = statistics.mean(tot)
    return {"value": g.m / (ms / 1e3), "unit": "edges/s", "ms_per_step": ms, "steps": k,
            "ncolors": res.ncolors, "rounds": res.rounds,
            "phase_ms": {"features": phase[0], "mlp_forward": phase[1], "keys": phase[2],
                         "coloring": phase[3]},
            "model": os.path.basename(gcpkg.PRIORITY_MODEL) + " (trained on R-MAT-G scales 14-18)",
            "gpu_launches": launches}


def measure_async(gcpkg, rp, ci, g, flush, stream, args):
    """The asynchronous form of Algorithm 2 on the same graph (Phase 1 reads live
    colors; schedule-dependent, valid by construction), for colors and rounds beside
    the synchronous form."""
    import torch
    out = torch.empty(g.n, dtype=torch.int32, device=rp.device)
    for _ in range(2):
        flush.zero_()
        res = gcpkg.color_async(rp, ci, out=out, stream=stream)
    torch.cuda.synchronize()
    ms, cols, rds = [], [], []
    for _ in range(max(3, args.steps // 5)):
        flush.zero_()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res = gcpkg.color_async(rp, ci, out=out, stream=stream)
        e.record(stream)
        e.synchronize()
        ms.append(a.elapsed_time(e))
        cols.append(res.ncolors)
        rds.append(res.rounds)
    return {"value": g.m / (statistics.mean(ms) / 1e3), "unit": "edges/s", "ms_per_step": statistics.mean(ms),
            "steps": len(ms), "ncolors": cols, "rounds": rds,
            "note": "Phase 1 reads live colors (the paper's shared-memory form); colors vary run to run"}


def measure_batched(gcpkg, count, flush, stream, steps, warmup, gpu_id, options, use_graph=True, e2e_steps=3,
                    cpu_baseline=False):
    """The batched workload: `count` graphs (sizes log-uniform in [1,000, 200,000];
    2-D grids, random geometric graphs and R-MAT-G in turn; seed 4) colored in
    one persistent launch, replayed as a CUDA graph; each step timed with CUDA
    events (L2 flushed before it), clocks sampled over the timed steps."""
    import torch
    dev = flush.device
    t = time.time()
    gs = gg.batch_mix(count, 4)
    rp, ci, voff, eoff = gcpkg.pack_batch((g.rowptr, g.colidx) for g in gs)
    m_total = int(sum(g.m for g in gs))
    log(f"batch of {len(gs)} graphs: N={voff[-1]} nnz={eoff[-1]} m={m_total} generated in {time.time() - t:.1f}s")
    rp_d, ci_d = torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev)
    b = gcpkg.Batch(rp_d, ci_d, voff, eoff, options=options)
    for _ in range(warmup):
        flush.zero_()
        b.run(graph=use_graph)
    b.status()
    sampler = ClockSampler(gpu_id)
    time.sleep(0.3)
    torch.cuda.synchronize(dev)
    t0 = time.time()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, e in evs:
        flush.zero_()
        a.record(stream)
        b.run(graph=use_graph)
        e.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop(t0, time.time())
    max_rounds, max_colors = b.status()
    ms = [a.elapsed_time(e) for a, e in evs]
    run_s = sum(ms) / 1e3 / len(ms)
    sizes, vols, bits = b.round_stats()
    N, NNZ = int(voff[-1]), int(eoff[-1])
    peak, peak_kind = peaks()
    if b.mode == 2:
        # device memory this mode moves (its colors live in shared memory) sets the fraction;
        # the method's fixed whole-row bytes (this mode reads whole rows, so its volumes are
        # the accounting's vol_k) go beside it
        moved = algorithmic_bytes_batch_blocks(N, sizes, vols)
        fixed = fixed_bytes_call(N, NNZ, sizes, vols)
        roof = {"bound": "hbm", "kernel": "whole run (byte-color and 32-bit passes of batch_local_kernel)",
                "batch_mode": 2, "achieved": moved / run_s / 1e9, "peak": peak, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": moved / run_s / 1e9 / peak, "traffic": None,
                "algorithmic_bytes": moved, "run_ms": 1e3 * run_s, "color_state_bits": bits,
                "accounting": "device-memory bytes this mode moves: rows, worklists, final colors",
                "fixed_whole_row": {"algorithmic_bytes": fixed, "achieved": fixed / run_s / 1e9,
                                    "frac": fixed / run_s / 1e9 / peak,
                                    "note": "the method's whole-row bytes over every graph, neighbour colors "
                                            "counted although this mode reads them from shared memory"},
                "shared_memory_gathers": {"count": int(sum(int(x) for x in vols)),
                                          "achieved_G_per_s": sum(int(x) for x in vols) / run_s / 1e9}}
    else:
        alg = algorithmic_bytes_batch(N, NNZ, sizes, vols, bits // 8)
        gathers = gathers_rounds(vols)
        roof = {"bound": "hbm", "kernel": "whole run (rebase, pass 1, rounds, reduce)", "batch_mode": 1,
                "achieved": alg / run_s / 1e9, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": alg / run_s / 1e9 / peak, "traffic": None, "algorithmic_bytes": alg,
                "run_ms": 1e3 * run_s, "color_state_bits": bits,
                "accounting": "this implementation's reads and writes",
                "l2_gathers": {"count": gathers, "achieved_G_per_s": gathers / run_s / 1e9,
                               "ceiling_G_per_s": L2_GATHER_CEILING,
                               "frac": gathers / run_s / 1e9 / L2_GATHER_CEILING}}
    roof["round_sizes"] = [int(x) for x in sizes]
    # end to end: host buffers in, colors and per-graph counts out
    h_rp, h_ci = torch.from_numpy(rp).pin_memory(), torch.from_numpy(ci).pin_memory()
    h_col = torch.empty(N, dtype=torch.int32).pin_memory()
    h_nc = torch.empty(len(gs), dtype=torch.int32).pin_memory()
    e_ms = []
    for i in range(e2e_steps + 1):  # the first run is a warm-up (first use of the pinned buffers)
        flush.zero_()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rp_d.copy_(h_rp, non_blocking=True)
        ci_d.copy_(h_ci, non_blocking=True)
        b.run(graph=use_graph)
        h_col.copy_(b.colors, non_blocking=True)
        h_nc.copy_(b.ncolors, non_blocking=True)
        e.record(stream)
        e.synchronize()
        if i > 0:
            e_ms.append(a.elapsed_time(e))
    out = {
        "workload": (f"batch of {len(gs)} graphs, sizes log-uniform in [1,000, 200,000], 2-D grids / random "
                     "geometric (avg degree 8) / R-MAT-G edge factor 8 in turn, seed 4; one persistent launch "
                     + ("replayed as a CUDA graph" if use_graph else "(plain launches)")),
        "graphs": len(gs), "N": N, "nnz": NNZ, "m": m_total,
        "value": m_total / run_s, "unit": "edges/s", "ms_per_step": 1e3 * run_s, "steps": steps,
        "options": options, "batch_mode": b.mode, "max_rounds": max_rounds, "max_colors": max_colors,
        "workspace_bytes": b.workspace_bytes, "gpu_launches": b.launch_count * steps,
        "l2": "inputs larger than L2 and L2 flushed (256 MB write) before every step",
        "roofline": roof, "clocks": clocks,
        "e2e": {"value": m_total / (statistics.mean(e_ms) / 1e3), "unit": "edges/s",
                "h2d_bytes_per_step": 4 * (rp.size + ci.size), "d2h_bytes_per_step": 4 * (N + len(gs)),
                "ms_per_step": statistics.mean(e_ms)},
    }
    if cpu_baseline:
        out["cpu_baseline"] = batch_cpu_baseline(gs)
    b.close()
    return out


def run_batched(args):
    """`--batched`: the batch of 4,096 graphs as its own JSON line, options picked
    by the autotuner (unless --no-autotune)."""
    import torch
    import paper_1205_3809_gb300 as gcpkg

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    gcpkg.library()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    props = torch.cuda.get_device_properties(dev)
    gpu_id = "GPU-" + str(props.uuid) if getattr(props, "uuid", None) else "0"
    best, table = ({"batch_mode": args.batch_mode} if args.batch_mode else {}), []
    if not args.no_autotune:
        gs = gg.batch_mix(args.batch_graphs, 4)
        rp, ci, voff, eoff = gcpkg.pack_batch((g.rowptr, g.colidx) for g in gs)
        t = time.time()
        best, table = gcpkg.autotune_batch(torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev), voff, eoff,
                                           reps=2)
        log(f"autotune {time.time() - t:.1f}s: best {best}")
        del gs, rp, ci
        torch.cuda.empty_cache()
    r = measure_batched(gcpkg, args.batch_graphs, flush, stream, args.steps, args.warmup, gpu_id, best,
                        use_graph=args.batch_launch == "graph", e2e_steps=max(3, args.steps // 3),
                        cpu_baseline=not args.no_cpu_baseline)
    line = {"metric": "edges colored/sec, batch of 4,096 graphs on 1 GB300", "value": r["value"], "unit": "edges/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "graphs", "N", "nnz", "m", "options", "batch_mode", "max_rounds",
                                         "max_colors", "workspace_bytes", "l2")},
            "roofline": r["roofline"], "autotune": [{"options": o, "ms": round(t_, 3)} for o, t_ in table],
            "e2e": r["e2e"], "gpu_launches": r["gpu_launches"], "clocks": r["clocks"],
            "cpu_baseline": r.get("cpu_baseline")}
    print(json.dumps(line), flush=True)


def measure_l2_ceiling():
    import shutil
    import tempfile
    src = os.path.join(ROOT, "l2_gather_probe.cu")
    tmp = tempfile.mkdtemp(prefix="gc_probe_")
    exe = os.path.join(tmp, "l2_gather_probe")
    try:
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
        subprocess.run([exe], check=True)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="time only the main workload (no c0/c1/c3/c4 sub-objects)")
    ap.add_argument("--no-batch", action="store_true", help="leave the batched configuration out of `configs`")
    ap.add_argument("--batched", action="store_true",
                    help="time the 4,096-graph batched workload instead (one JSON line)")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--batch-launch", choices=["graph", "plain"], default="graph",
                    help="batched runs as a replayed CUDA graph or as plain launches")
    ap.add_argument("--no-autotune", action="store_true",
                    help="batched: use the library's default options instead of tuning")
    ap.add_argument("--batch-mode", type=int, choices=[0, 1, 2], default=0,
                    help="batched, with --no-autotune: gc_options.batch_mode (0: the library chooses)")
    ap.add_argument("--scale", type=int, default=SCALE,
                    help="R-MAT-B scale (24 is the benchmark; smaller scales are for profiling)")
    ap.add_argument("--measure-l2-ceiling", action="store_true",
                    help="build and run the random-gather ceiling probe, then exit")
    args = ap.parse_args()
    if args.measure_l2_ceiling:
        measure_l2_ceiling()
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.batched:
        run_batched(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
