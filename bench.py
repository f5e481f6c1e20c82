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
# index array, measured on this machine's GB300 (profiles/l2_random_gather.md).
L2_GATHER_CEILING = 208.0  # G gathers/s, 32 MB table (the scale-24 color state)
L2_SECTOR_CEILING = 234.0  # G sectors/s: the same run counted in L2 sectors (gathers + index stream)

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
    (tests/golden/fullsize.json, written by tests/golden/make_fullsize.py), when
    the run's |U_k| are the stored ones; else None."""
    path = os.path.join(ROOT, "tests", "golden", "fullsize.json")
    if not os.path.exists(path):
        return None
    for entry in json.load(open(path)).values():
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


def load_profile_fields(kernel_src):
    """Per-launch counters of the rounds kernel from the committed ncu summary
    (`- key: value` lines), or {} if the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "rounds_persistent_kernel_rmat_b.md")
    if not os.path.exists(path):
        return {}
    want = kernel_code_hash(kernel_src)
    fields = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    return fields if fields.get("kernel_code_sha256") == want else {}


def load_traffic(kernel_src):
    """Per-launch DRAM bytes of the rounds kernel (full size), or None."""
    try:
        return int(load_profile_fields(kernel_src)["traffic_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def load_l2_sectors(kernel_src):
    """Per-launch L2 sectors of the rounds kernel at full size (a one-pass capture), or None."""
    try:
        return int(load_profile_fields(kernel_src)["l2_sectors_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


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
    traffic = load_traffic(os.path.join(ROOT, "paper_1205_3809_gb300", "csrc", "gc_device.cuh"))
    gathers = gathers_rounds(vols)
    gather_rate = gathers / (kms / 1e3) / 1e9
    sectors = load_l2_sectors(os.path.join(ROOT, "paper_1205_3809_gb300", "csrc", "gc_device.cuh"))

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
                             "source": "lts__t_sectors.sum of one full-size launch (profiles/)"}},
            "cpu_baseline": cpu,
            "learned": learned,
            "asynchronous": asynchronous,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


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


def run_batched(args):
    """The batched workload: 4,096 graphs (sizes log-uniform in [1,000, 200,000]; 2-D
    grids, random geometric graphs and R-MAT-G in turn; seed 4) colored in one
    persistent launch replayed as a CUDA graph, options picked by the autotuner."""
    import torch
    import paper_1205_3809_gb300 as gcpkg

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    gcpkg.library()
    t = time.time()
    gs = gg.batch_mix(args.batch_graphs, 4)
    rp, ci, voff, eoff = gcpkg.pack_batch((g.rowptr, g.colidx) for g in gs)
    m_total = int(sum(g.m for g in gs))
    log(f"batch of {len(gs)} graphs: N={voff[-1]} nnz={eoff[-1]} m={m_total} generated in {time.time() - t:.1f}s")
    rp_d, ci_d = torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev)
    stream = torch.cuda.current_stream(dev)
    t = time.time()
    if args.no_autotune:
        best, table = ({"batch_mode": args.batch_mode} if args.batch_mode else {}), []
    else:
        best, table = gcpkg.autotune_batch(rp_d, ci_d, voff, eoff, reps=2)
    log(f"autotune {time.time() - t:.1f}s: best {best}")
    use_graph = args.batch_launch == "graph"
    b = gcpkg.Batch(rp_d, ci_d, voff, eoff, options=best)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        flush.zero_()
        b.run(graph=use_graph)
    b.status()
    props = torch.cuda.get_device_properties(dev)
    sampler = ClockSampler("GPU-" + str(props.uuid) if getattr(props, "uuid", None) else "0")
    time.sleep(0.3)
    torch.cuda.synchronize(dev)
    t0 = time.time()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, e in evs:
        flush.zero_()
        a.record(stream)
        b.run(graph=use_graph)
        e.record(stream)
    torch.cuda.synchronize(dev)
    t1 = time.time()
    clocks = sampler.stop(t0, t1)
    max_rounds, max_colors = b.status()
    ms = [a.elapsed_time(e) for a, e in evs]
    total_s = sum(ms) / 1e3
    sizes, vols, bits = b.round_stats()
    N, NNZ = int(voff[-1]), int(eoff[-1])
    if b.mode == 2:
        # this mode reads whole rows, so its round volumes are the fixed accounting's vol_k
        alg_bytes = fixed_bytes_call(N, NNZ, sizes, vols)
        moved_bytes = algorithmic_bytes_batch_blocks(N, sizes, vols)
    else:
        alg_bytes = moved_bytes = algorithmic_bytes_batch(N, NNZ, sizes, vols, bits // 8)
    run_s = total_s / len(evs)
    peak, peak_kind = peaks()
    gathers = gathers_rounds(vols)
    # end to end: host buffers in, colors and per-graph counts out
    h_rp, h_ci = torch.from_numpy(rp).pin_memory(), torch.from_numpy(ci).pin_memory()
    h_col = torch.empty(int(voff[-1]), dtype=torch.int32).pin_memory()
    h_nc = torch.empty(len(gs), dtype=torch.int32).pin_memory()
    e_ms = []
    for _ in range(max(3, args.steps // 3)):
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
        e_ms.append(a.elapsed_time(e))
    line = {
        "metric": "edges colored/sec, batch of 4,096 graphs on 1 GB300", "value": len(evs) * m_total / total_s,
        "unit": "edges/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"batch of {len(gs)} graphs, sizes log-uniform in [1,000, 200,000], 2-D grids / "
                               "random geometric (avg degree 8) / R-MAT-G edge factor 8 in turn, seed 4; one "
                               "persistent launch " + ("replayed as a CUDA graph" if use_graph else
                                                        "(plain launches)"),
                   "graphs": len(gs), "N": int(voff[-1]), "nnz": int(eoff[-1]), "m": m_total,
                   "options": best, "max_rounds": max_rounds, "max_colors": max_colors,
                   "workspace_bytes": b.workspace_bytes,
                   "l2": "inputs larger than L2 and L2 flushed (256 MB write) before every step"},
        "roofline": {"bound": "hbm",
                     "kernel": ("whole run (byte-color and 32-bit passes of batch_local_kernel)" if b.mode == 2
                                else "whole run (rebase, pass 1, rounds, reduce)"),
                     "batch_mode": b.mode,
                     "achieved": alg_bytes / run_s / 1e9, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": alg_bytes / run_s / 1e9 / peak, "traffic": None,
                     "algorithmic_bytes": alg_bytes, "run_ms": 1e3 * run_s, "color_state_bits": bits,
                     "accounting": ("whole rows: fixed bytes of the method over every graph (neighbour colors "
                                    "counted as the method's reads, though this mode keeps them in shared memory)"
                                    if b.mode == 2 else "this implementation's reads and writes"),
                     "device_memory_bytes": moved_bytes,
                     "round_sizes": [int(x) for x in sizes],
                     **({"shared_memory_gathers": {
                         "count": int(sum(int(x) for x in vols)),
                         "achieved_G_per_s": sum(int(x) for x in vols) / run_s / 1e9,
                         "note": "neighbour colors read from shared memory, all rounds"}} if b.mode == 2 else
                        {"l2_gathers": {"count": gathers, "achieved_G_per_s": gathers / run_s / 1e9,
                                        "ceiling_G_per_s": L2_GATHER_CEILING,
                                        "frac": gathers / run_s / 1e9 / L2_GATHER_CEILING}})},
        "autotune": [{"options": o, "ms": round(t_, 3)} for o, t_ in table],
        "e2e": {"value": m_total / (statistics.mean(e_ms) / 1e3), "unit": "edges/s",
                "h2d_bytes_per_step": 4 * (rp.size + ci.size), "d2h_bytes_per_step": 4 * (int(voff[-1]) + len(gs)),
                "ms_per_step": statistics.mean(e_ms)},
        "gpu_launches": b.launch_count * args.steps,
        "clocks": clocks,
        "cpu_baseline": None if args.no_cpu_baseline else batch_cpu_baseline(gs),
    }
    print(json.dumps(line), flush=True)
    b.close()


def measure_l2_ceiling():
    import shutil
    import tempfile
    src = os.path.join(ROOT, "paper_1205_3809_gb300", "csrc", "l2_gather_probe.cu")
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
