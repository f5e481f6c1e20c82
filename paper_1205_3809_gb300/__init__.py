"""GB300-native speculative distance-1 graph coloring (Algorithm 2, "Iterative",
Sec. 3.2 of Catalyurek et al., arXiv 1205.3809), synchronous rounds.

This module is the Python binding of ``libgc.so``: it marshals arguments for the
C ABI declared in ``include/gc.h`` and does nothing else.  Every step of the
coloring runs in the library's CUDA kernels; there is no CPU path, and calling
anything here without the compiled library raises ``GcLibraryMissing``.
PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_INCLUDE = os.path.join(_ROOT, "include")
LIB_PATH = os.environ.get("GC_LIB_PATH") or os.path.join(_HERE, "libgc.so")

GC_OK = 0
GC_ERR_INVALID = -1
GC_ERR_CUDA = -2
GC_ERR_OOM = -3
GC_ERR_MAX_ROUNDS = -4
GC_ERR_TIMEOUT = -5
GC_ERR_BAD_GRAPH = -6
GC_ERR_TOO_LARGE = -7

# Every symbol include/gc.h declares.
EXPORTED = ("gc_color", "gc_color_ex", "gc_color_host", "gc_validate_csr", "gc_strerror",
            "gc_last_cuda_error", "gc_release", "gc_workspace_bytes", "gc_last_launch_count",
            "gc_last_round_stats", "gc_last_phase_ms", "gc_last_round_ns", "gc_color_noalloc",
            "gc_noalloc_capacity_bytes",
            "gc_features", "gc_mlp_param_count", "gc_mlp_forward", "gc_mlp_grad", "gc_mlp_adam",
            "gc_priority_keys", "gc_mlp_train_step", "gc_batch_create", "gc_batch_run",
            "gc_batch_launch_graph", "gc_batch_status", "gc_batch_destroy", "gc_batch_workspace_bytes",
            "gc_batch_launch_count", "gc_tune", "gc_batch_tune", "gc_color_async", "gc_batch_features",
            "gc_batch_round_stats", "gc_batch_mode", "gc_color_batched")


class GcLibraryMissing(RuntimeError):
    pass


class GcError(RuntimeError):
    def __init__(self, code: int, where: str, cuda_error: int = 0):
        self.code = code
        self.cuda_error = cuda_error
        msg = f"{where}: {strerror(code)} (gc_status {code})"
        if cuda_error:
            msg += f", cudaError {cuda_error}"
        super().__init__(msg)


def _sources():
    return [os.path.join(_CSRC, f) for f in sorted(os.listdir(_CSRC)) if f.endswith((".cu", ".cuh"))]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libgc.so for sm_103a with nvcc (in-tree)."""
    srcs = _sources() + [os.path.join(_INCLUDE, "gc.h")]
    if (not force and os.path.exists(LIB_PATH)
            and all(os.path.getmtime(LIB_PATH) >= os.path.getmtime(s) for s in srcs)):
        return LIB_PATH
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
           "-Xcompiler", "-fPIC", "-shared", "-I", _INCLUDE, "--threads", "3", "-o", LIB_PATH + ".tmp",
           os.path.join(_CSRC, "gc.cu"), os.path.join(_CSRC, "gc_mlp.cu"), os.path.join(_CSRC, "gc_async.cu")]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(LIB_PATH + ".tmp", LIB_PATH)
    return LIB_PATH


class Options(ctypes.Structure):
    """Mirror of ``gc_options`` (gc.h).  0 selects each default."""
    _fields_ = [("small_max_degree", ctypes.c_int32), ("medium_max_degree", ctypes.c_int32),
                ("max_rounds", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("loop_mode", ctypes.c_int32), ("color_bits", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("telemetry", ctypes.c_int32),
                ("narrow_color_limit", ctypes.c_int32), ("tail_volume", ctypes.c_int32),
                ("batch_mode", ctypes.c_int32), ("local_thread_degree", ctypes.c_int32),
                ("local_shared_bytes", ctypes.c_int32), ("barrier_poll_limit", ctypes.c_int32),
                ("workspace_limit_mb", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GcLibraryMissing(
                f"{LIB_PATH} is not built; run __graft_entry__.build() or paper_1205_3809_gb300.build()")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32 = ctypes.c_void_p, ctypes.c_int32
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.gc_color.argtypes = [vp, vp, i32, vp, vp, i32p, i32p]
        lib.gc_color_ex.argtypes = [vp, vp, i32, vp, vp, i32p, i32p, vp, ctypes.POINTER(Options),
                                    vp, i32]
        lib.gc_color_host.argtypes = [vp, vp, i32, vp, vp, i32p, i32p, vp, ctypes.POINTER(Options)]
        lib.gc_validate_csr.argtypes = [vp, vp, i32, vp]
        lib.gc_strerror.argtypes = [ctypes.c_int]
        lib.gc_strerror.restype = ctypes.c_char_p
        lib.gc_workspace_bytes.restype = ctypes.c_size_t
        lib.gc_last_launch_count.restype = ctypes.c_int64
        lib.gc_last_round_stats.argtypes = [vp, vp, i32]
        lib.gc_color_noalloc.argtypes = [vp, vp, i32, vp, vp, i32p, i32p, vp]
        lib.gc_color_noalloc.restype = ctypes.c_int
        lib.gc_noalloc_capacity_bytes.restype = ctypes.c_size_t
        i64, f32 = ctypes.c_int64, ctypes.c_float
        lib.gc_features.argtypes = [vp, vp, i32, vp, vp]
        lib.gc_mlp_forward.argtypes = [vp, vp, i64, vp, vp]
        lib.gc_mlp_grad.argtypes = [vp, vp, vp, i64, f32, vp, vp, vp]
        lib.gc_mlp_adam.argtypes = [vp, vp, vp, vp, i32, f32, f32, f32, f32, vp]
        lib.gc_priority_keys.argtypes = [vp, i64, vp, vp]
        lib.gc_mlp_train_step.argtypes = [vp, vp, vp, vp, vp, vp, vp, i64, i32, f32, f32, f32, f32, vp]
        lib.gc_mlp_train_step.restype = ctypes.c_int
        for f in (lib.gc_features, lib.gc_mlp_forward, lib.gc_mlp_grad, lib.gc_mlp_adam,
                  lib.gc_priority_keys, lib.gc_mlp_param_count):
            f.restype = ctypes.c_int
        lib.gc_batch_create.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, vp, ctypes.POINTER(Options), vp,
                                        ctypes.POINTER(vp)]
        lib.gc_batch_run.argtypes = [vp, vp]
        lib.gc_batch_launch_graph.argtypes = [vp, vp]
        lib.gc_batch_status.argtypes = [vp, vp, i32p, i32p]
        lib.gc_batch_destroy.argtypes = [vp]
        lib.gc_batch_workspace_bytes.argtypes = [vp]
        lib.gc_batch_workspace_bytes.restype = ctypes.c_size_t
        lib.gc_batch_features.argtypes = [vp, vp, vp]
        lib.gc_batch_round_stats.argtypes = [vp, vp, vp, i32, vp, vp]
        lib.gc_batch_round_stats.restype = ctypes.c_int
        lib.gc_batch_mode.argtypes = [vp]
        lib.gc_batch_mode.restype = ctypes.c_int
        lib.gc_color_batched.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(Options)]
        lib.gc_color_batched.restype = ctypes.c_int
        lib.gc_batch_features.restype = ctypes.c_int
        lib.gc_batch_launch_count.argtypes = [vp]
        lib.gc_batch_launch_count.restype = ctypes.c_int64
        for f in (lib.gc_batch_create, lib.gc_batch_run, lib.gc_batch_launch_graph, lib.gc_batch_status,
                  lib.gc_batch_destroy):
            f.restype = ctypes.c_int
        fp = ctypes.POINTER(ctypes.c_float)
        lib.gc_tune.argtypes = [vp, vp, i32, vp, vp, ctypes.POINTER(Options), i32, i32, vp, fp, i32p]
        lib.gc_batch_tune.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, vp, ctypes.POINTER(Options), i32, i32, vp,
                                      fp, i32p]
        lib.gc_tune.restype = ctypes.c_int
        lib.gc_color_async.argtypes = [vp, vp, i32, vp, vp, i32p, i32p, i32, vp]
        lib.gc_color_async.restype = ctypes.c_int
        lib.gc_batch_tune.restype = ctypes.c_int
        lib.gc_last_phase_ms.argtypes = [vp, i32]
        lib.gc_last_round_ns.argtypes = [vp, i32]
        for f in (lib.gc_color, lib.gc_color_ex, lib.gc_color_host, lib.gc_validate_csr,
                  lib.gc_last_cuda_error, lib.gc_release, lib.gc_last_round_stats,
                  lib.gc_last_phase_ms, lib.gc_last_round_ns):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def library():
    """The loaded ctypes handle of libgc.so."""
    return _load()


def strerror(code: int) -> str:
    try:
        return _load().gc_strerror(code).decode()
    except GcLibraryMissing:
        return f"gc_status {code}"


def _options(opts) -> Optional[Options]:
    if opts is None:
        return None
    if isinstance(opts, Options):
        return opts
    o = Options()
    for k, v in dict(opts).items():
        setattr(o, k, int(v))
    return o


@dataclass
class Result:
    colors: object            # torch.Tensor (device) or np.ndarray (host call)
    ncolors: int
    rounds: int
    round_sizes: Optional[np.ndarray] = field(default=None)
    status: int = GC_OK


def _dev_ptr(t, dtype, name, numel):
    import torch
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    return ctypes.c_void_p(t.data_ptr()) if t.numel() > 0 else None


def color(rowptr, colidx, priority=None, *, out=None, options=None, stream=None,
          round_sizes: bool = False, check: bool = True) -> Result:
    """Color a symmetric int32 CSR graph held on the GPU (``gc_color_ex``).

    rowptr: int32 CUDA tensor (n+1); colidx: int32 CUDA tensor (nnz);
    priority: optional uint32 keys as an int32 or uint32 CUDA tensor (n), smaller
    key = higher precedence, ties by index; out: optional int32 CUDA tensor (n).
    """
    import torch
    lib = _load()
    n = int(rowptr.numel()) - 1
    if n < 0:
        raise ValueError("rowptr must have n+1 >= 1 entries")
    rp = _dev_ptr(rowptr, torch.int32, "rowptr", None)
    ci = _dev_ptr(colidx, torch.int32, "colidx", None)
    pr = None
    if priority is not None:
        if priority.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
            raise ValueError("priority must be a 32-bit integer tensor")
        pr = _dev_ptr(priority, priority.dtype, "priority", n)
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=rowptr.device)
    co = _dev_ptr(out, torch.int32, "out", n)
    if stream is None:
        stream = torch.cuda.current_stream(rowptr.device)
    sh = ctypes.c_void_p(stream.cuda_stream)
    nc, rd = ctypes.c_int32(), ctypes.c_int32()
    cap = 0
    rs_buf = None
    if round_sizes:
        o = _options(options)
        cap = min(o.max_rounds if o is not None and o.max_rounds > 0 else max(n, 1), 1 << 20)
        rs_buf = np.zeros(cap, np.int32)
    opt = _options(options)
    with torch.cuda.device(rowptr.device):
        rc = lib.gc_color_ex(rp, ci, n, pr, co, ctypes.byref(nc), ctypes.byref(rd), sh,
                             ctypes.byref(opt) if opt is not None else None,
                             ctypes.c_void_p(rs_buf.ctypes.data) if rs_buf is not None else None,
                             cap)
    if rc != GC_OK and check:
        raise GcError(rc, "gc_color_ex", lib.gc_last_cuda_error())
    res = Result(colors=out, ncolors=int(nc.value), rounds=int(rd.value))
    if rs_buf is not None:
        res.round_sizes = rs_buf[:min(res.rounds, cap)].copy()
    res.status = rc
    return res


def color_async(rowptr, colidx, priority=None, *, out=None, max_rounds: int = 0, stream=None,
                check: bool = True) -> Result:
    """Asynchronous Algorithm 2 (``gc_color_async``): schedule-dependent colors, valid
    by construction; the comparison point for the synchronous ``color``."""
    import torch
    lib = _load()
    n = int(rowptr.numel()) - 1
    rp = _dev_ptr(rowptr, torch.int32, "rowptr", None)
    ci = _dev_ptr(colidx, torch.int32, "colidx", None)
    pr = None if priority is None else _dev_ptr(priority, priority.dtype, "priority", n)
    if out is None:
        out = torch.empty(max(n, 0), dtype=torch.int32, device=rowptr.device)
    co = _dev_ptr(out, torch.int32, "out", max(n, 0))
    nc, rd = ctypes.c_int32(), ctypes.c_int32()
    with torch.cuda.device(rowptr.device):
        rc = lib.gc_color_async(rp, ci, n, pr, co, ctypes.byref(nc), ctypes.byref(rd), int(max_rounds),
                                _stream_handle(stream, rowptr.device))
    if rc != GC_OK and check:
        raise GcError(rc, "gc_color_async", lib.gc_last_cuda_error())
    return Result(colors=out, ncolors=int(nc.value), rounds=int(rd.value), status=rc)


def color_host(rowptr: np.ndarray, colidx: np.ndarray, priority=None, *, out=None,
               options=None, stream=None) -> Result:
    """Color a graph held in host memory (``gc_color_host``): the library copies the
    inputs to the device, colors, and copies the colors back into ``out``."""
    lib = _load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32) if not _is_pinned_tensor(rowptr) else rowptr
    n = int(rowptr.shape[0]) - 1
    if out is None:
        out = np.empty(max(n, 0), np.int32)
    nc, rd = ctypes.c_int32(), ctypes.c_int32()
    opt = _options(options)
    sh = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    rc = lib.gc_color_host(_host_ptr(rowptr), _host_ptr(colidx), n,
                           _host_ptr(priority) if priority is not None else None,
                           _host_ptr(out), ctypes.byref(nc), ctypes.byref(rd), sh,
                           ctypes.byref(opt) if opt is not None else None)
    if rc != GC_OK:
        raise GcError(rc, "gc_color_host", lib.gc_last_cuda_error())
    return Result(colors=out, ncolors=int(nc.value), rounds=int(rd.value))


def _is_pinned_tensor(x) -> bool:
    return hasattr(x, "data_ptr") and hasattr(x, "is_pinned")


def _host_ptr(x):
    if _is_pinned_tensor(x):
        return ctypes.c_void_p(x.data_ptr()) if x.numel() else None
    return ctypes.c_void_p(x.ctypes.data) if x.size else None


def validate_csr(rowptr, colidx, stream=None) -> int:
    """Device check of a CSR (``gc_validate_csr``); returns the gc_status code."""
    import torch
    lib = _load()
    n = int(rowptr.numel()) - 1
    rp = _dev_ptr(rowptr, torch.int32, "rowptr", None)
    ci = _dev_ptr(colidx, torch.int32, "colidx", None)
    if stream is None:
        stream = torch.cuda.current_stream(rowptr.device)
    with torch.cuda.device(rowptr.device):
        return int(lib.gc_validate_csr(rp, ci, n, ctypes.c_void_p(stream.cuda_stream)))


def release() -> None:
    _load().gc_release()


def workspace_bytes() -> int:
    return int(_load().gc_workspace_bytes())


def last_launch_count() -> int:
    return int(_load().gc_last_launch_count())


def last_round_stats(cap: int = 1 << 20):
    """(sizes, volumes) per round of the last coloring call: |U_r| and sum of degrees over U_r."""
    sizes = np.zeros(cap, np.int32)
    vols = np.zeros(cap, np.int64)
    m = int(_load().gc_last_round_stats(ctypes.c_void_p(sizes.ctypes.data),
                                        ctypes.c_void_p(vols.ctypes.data), cap))
    if m < 0:
        raise GcError(m, "gc_last_round_stats")
    return sizes[:m].copy(), vols[:m].copy()


def last_phase_ms():
    """[setup, round 1, later rounds, whole call] in ms, for a call made with telemetry=1."""
    ms = (ctypes.c_float * 4)()
    m = int(_load().gc_last_phase_ms(ms, 4))
    if m < 0:
        raise GcError(m, "gc_last_phase_ms")
    return [float(ms[i]) for i in range(m)]


def last_round_ns(cap: int = 1 << 20):
    """Per-round durations (ns) of the last call made with telemetry=1 in the persistent
    launch: entry k-1 is round k's pass (k >= 2); entry 0 is 0."""
    ns = np.zeros(cap, np.int64)
    m = int(_load().gc_last_round_ns(ctypes.c_void_p(ns.ctypes.data), cap))
    if m < 0:
        raise GcError(m, "gc_last_round_ns")
    return ns[:m].copy()


# ---------------------------------------------------------------- learned priority

MLP_PARAMS = 1313
PRIORITY_MODEL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "priority_mlp_rmat_g.json")


def _stream_handle(stream, device):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc, what):
    if rc != GC_OK:
        raise GcError(rc, what, _load().gc_last_cuda_error())


def features(rowptr, colidx, *, out=None, stream=None):
    """float32 [n, 6] per-vertex features of a graph held on the GPU (``gc_features``)."""
    import torch
    lib = _load()
    n = int(rowptr.numel()) - 1
    rp = _dev_ptr(rowptr, torch.int32, "rowptr", None)
    ci = _dev_ptr(colidx, torch.int32, "colidx", None)
    if out is None:
        out = torch.empty((max(n, 0), 6), dtype=torch.float32, device=rowptr.device)
    fo = _dev_ptr(out, torch.float32, "out", max(n, 0) * 6)
    with torch.cuda.device(rowptr.device):
        _check(lib.gc_features(rp, ci, n, fo, _stream_handle(stream, rowptr.device)), "gc_features")
    return out


def mlp_forward(params, x, *, out=None, stream=None):
    """Network scores, float32 [n], of features x (float32 [n, 6]) (``gc_mlp_forward``)."""
    import torch
    lib = _load()
    n = int(x.numel()) // 6
    pp = _dev_ptr(params, torch.float32, "params", MLP_PARAMS)
    xp = _dev_ptr(x, torch.float32, "x", n * 6)
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=x.device)
    yp = _dev_ptr(out, torch.float32, "out", n)
    with torch.cuda.device(x.device):
        _check(lib.gc_mlp_forward(pp, xp, n, yp, _stream_handle(stream, x.device)), "gc_mlp_forward")
    return out


def mlp_grad(params, x, t, scale: float, grad, sse, *, stream=None):
    """Add the gradient of scale * sum (y - t)^2 into grad (float32 [1313]) and the sum of
    squared errors into sse (float32 [1]) (``gc_mlp_grad``)."""
    import torch
    lib = _load()
    n = int(t.numel())
    args = (_dev_ptr(params, torch.float32, "params", MLP_PARAMS), _dev_ptr(x, torch.float32, "x", n * 6),
            _dev_ptr(t, torch.float32, "t", n), n, float(scale),
            _dev_ptr(grad, torch.float32, "grad", MLP_PARAMS), _dev_ptr(sse, torch.float32, "sse", 1))
    with torch.cuda.device(x.device):
        _check(lib.gc_mlp_grad(*args, _stream_handle(stream, x.device)), "gc_mlp_grad")


def adam_step(params, m, v, grad, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8, *, stream=None):
    """One Adam step on params with moments m, v (all float32 [1313]) (``gc_mlp_adam``)."""
    import torch
    lib = _load()
    ptrs = [_dev_ptr(a, torch.float32, name, MLP_PARAMS)
            for a, name in ((params, "params"), (m, "m"), (v, "v"), (grad, "grad"))]
    with torch.cuda.device(params.device):
        _check(lib.gc_mlp_adam(*ptrs, int(step), float(lr), float(beta1), float(beta2), float(eps),
                               _stream_handle(stream, params.device)), "gc_mlp_adam")


class MlpTrainer:
    """Adam training of the priority network on the GPU (``gc_mlp_train_step``).

    Holds the parameters, both moments and the gradient as float32 CUDA tensors;
    ``step(x, t)`` takes one step on the mean squared error of the batch and
    returns its sum of squared errors as a device scalar (no host sync).
    """

    def __init__(self, params, lr: float = 3e-3, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8):
        import torch
        self.params = params.detach().to(torch.float32).contiguous().clone()
        dev = self.params.device
        self.m = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=dev)
        self.v = torch.zeros_like(self.m)
        self.grad = torch.zeros_like(self.m)
        self.sse = torch.zeros(1, dtype=torch.float32, device=dev)
        self.lr, self.beta1, self.beta2, self.eps = lr, beta1, beta2, eps
        self.t = 0

    def step(self, x, t, stream=None):
        import torch
        lib = _load()
        n = int(t.numel())
        self.t += 1
        ptrs = [_dev_ptr(a, torch.float32, name, MLP_PARAMS)
                for a, name in ((self.params, "params"), (self.m, "m"), (self.v, "v"), (self.grad, "grad"))]
        with torch.cuda.device(self.params.device):
            _check(lib.gc_mlp_train_step(*ptrs, _dev_ptr(self.sse, torch.float32, "sse", 1),
                                         _dev_ptr(x, torch.float32, "x", n * 6),
                                         _dev_ptr(t, torch.float32, "t", n), n, self.t, float(self.lr),
                                         float(self.beta1), float(self.beta2), float(self.eps),
                                         _stream_handle(stream, self.params.device)), "gc_mlp_train_step")
        return self.sse


def priority_keys(scores, *, out=None, stream=None):
    """uint32 keys (as int32) in the order of float32 scores (``gc_priority_keys``)."""
    import torch
    lib = _load()
    n = int(scores.numel())
    sp = _dev_ptr(scores, torch.float32, "scores", n)
    if out is None:
        out = torch.empty(n, dtype=torch.int32, device=scores.device)
    kp = _dev_ptr(out, torch.int32, "out", n)
    with torch.cuda.device(scores.device):
        _check(lib.gc_priority_keys(sp, n, kp, _stream_handle(stream, scores.device)), "gc_priority_keys")
    return out


def load_priority_model(path: Optional[str] = None, device=None):
    """The trained network's float32 parameter vector (on ``device`` if given, else a numpy array)."""
    import json
    with open(path or PRIORITY_MODEL) as f:
        doc = json.load(f)
    p = np.asarray(doc["params"], dtype=np.float32)
    if p.shape != (MLP_PARAMS,):
        raise ValueError(f"model has {p.shape} parameters, expected {MLP_PARAMS}")
    if device is None:
        return p
    import torch
    return torch.from_numpy(p).to(device)


def learned_priority(rowptr, colidx, params, *, stream=None):
    """Priority keys of every vertex: keys(network(features)), all on the GPU."""
    f = features(rowptr, colidx, stream=stream)
    return priority_keys(mlp_forward(params, f, stream=stream), stream=stream)


def color_learned(rowptr, colidx, params=None, *, options=None, stream=None, round_sizes=False) -> Result:
    """Color with the learned priority (the trained model when params is None)."""
    if params is None:
        params = load_priority_model(device=rowptr.device)
    keys = learned_priority(rowptr, colidx, params, stream=stream)
    return color(rowptr, colidx, keys, options=options, stream=stream, round_sizes=round_sizes)


# ---------------------------------------------------------------- batched coloring

def pack_batch(graphs):
    """Lay per-graph CSRs end to end in the batched input layout.

    graphs: iterable of (rowptr, colidx) numpy int32 pairs (each graph's own ids).
    Returns (rowptr_cat, colidx_cat, vertex_offsets, edge_offsets) as numpy arrays.
    """
    rps, cis, nv, ne = [], [], [0], [0]
    for rp, ci in graphs:
        rp = np.asarray(rp, dtype=np.int32)
        ci = np.asarray(ci, dtype=np.int32)
        rps.append(rp)
        cis.append(ci)
        nv.append(nv[-1] + rp.shape[0] - 1)
        ne.append(ne[-1] + ci.shape[0])
    rowptr_cat = np.concatenate(rps) if rps else np.zeros(0, np.int32)
    colidx_cat = np.concatenate(cis) if cis else np.zeros(0, np.int32)
    return rowptr_cat, colidx_cat, np.asarray(nv, np.int64), np.asarray(ne, np.int64)


def color_batched(rowptr_cat, colidx_cat, vertex_offsets, edge_offsets, priority=None, *, options=None,
                  stream=None):
    """Color a batch in one call (``gc_color_batched``): plan, one run, status, free.
    Same arguments as ``Batch``; returns (colors, ncolors, rounds) as CUDA tensors."""
    import torch
    lib = _load()
    voff = np.ascontiguousarray(vertex_offsets, dtype=np.int64)
    eoff = np.ascontiguousarray(edge_offsets, dtype=np.int64)
    G = int(voff.shape[0]) - 1
    if G < 0 or eoff.shape[0] != G + 1:
        raise ValueError("vertex_offsets and edge_offsets must both have G+1 entries")
    N, NNZ = int(voff[-1]), int(eoff[-1])
    dev = rowptr_cat.device
    colors = torch.empty(N, dtype=torch.int32, device=dev)
    ncolors = torch.empty(G, dtype=torch.int32, device=dev)
    rounds = torch.empty(G, dtype=torch.int32, device=dev)
    pr = None if priority is None else _dev_ptr(priority, priority.dtype, "priority", N)
    opt = _options(options)
    with torch.cuda.device(dev):
        rc = lib.gc_color_batched(ctypes.c_void_p(voff.ctypes.data), ctypes.c_void_p(eoff.ctypes.data), G,
                                  _dev_ptr(rowptr_cat, torch.int32, "rowptr_cat", N + G),
                                  _dev_ptr(colidx_cat, torch.int32, "colidx_cat", NNZ), pr,
                                  _dev_ptr(colors, torch.int32, "colors", N),
                                  _dev_ptr(ncolors, torch.int32, "ncolors", G),
                                  _dev_ptr(rounds, torch.int32, "rounds", G), _stream_handle(stream, dev),
                                  ctypes.byref(opt) if opt is not None else None)
    if rc != GC_OK:
        raise GcError(rc, "gc_color_batched", lib.gc_last_cuda_error())
    return colors, ncolors, rounds


class Batch:
    """A planned batch of independent graphs colored in one persistent launch
    (``gc_batch_create`` / ``gc_batch_run`` / ``gc_batch_launch_graph``).

    rowptr_cat, colidx_cat: int32 CUDA tensors in the batched layout (see
    ``pack_batch``); vertex_offsets, edge_offsets: host int64 arrays (G+1);
    priority: optional 32-bit CUDA tensor of voff[G] keys.  The plan owns its
    workspace; ``colors`` (voff[G]), ``ncolors`` and ``rounds`` (G) are CUDA
    tensors written by every run.
    """

    def __init__(self, rowptr_cat, colidx_cat, vertex_offsets, edge_offsets, priority=None, *,
                 options=None, stream=None):
        import torch
        lib = _load()
        self._lib = lib
        voff = np.ascontiguousarray(vertex_offsets, dtype=np.int64)
        eoff = np.ascontiguousarray(edge_offsets, dtype=np.int64)
        G = int(voff.shape[0]) - 1
        if G < 0 or eoff.shape[0] != G + 1:
            raise ValueError("vertex_offsets and edge_offsets must both have G+1 entries")
        N, NNZ = int(voff[-1]), int(eoff[-1])
        dev = rowptr_cat.device
        self.device = dev
        self.num_graphs = G
        self.colors = torch.empty(N, dtype=torch.int32, device=dev)
        self.ncolors = torch.empty(G, dtype=torch.int32, device=dev)
        self.rounds = torch.empty(G, dtype=torch.int32, device=dev)
        rp = _dev_ptr(rowptr_cat, torch.int32, "rowptr_cat", N + G)
        ci = _dev_ptr(colidx_cat, torch.int32, "colidx_cat", NNZ)
        pr = None
        if priority is not None:
            if priority.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
                raise ValueError("priority must be a 32-bit integer tensor")
            pr = _dev_ptr(priority, priority.dtype, "priority", N)
        self._keep = (rowptr_cat, colidx_cat, priority)  # the plan reads these on every run
        opt = _options(options)
        handle = ctypes.c_void_p()
        with torch.cuda.device(dev):
            rc = lib.gc_batch_create(rp, ci, ctypes.c_void_p(voff.ctypes.data), ctypes.c_void_p(eoff.ctypes.data),
                                     G, pr, _dev_ptr(self.colors, torch.int32, "colors", N),
                                     _dev_ptr(self.ncolors, torch.int32, "ncolors", G),
                                     _dev_ptr(self.rounds, torch.int32, "rounds", G),
                                     ctypes.byref(opt) if opt is not None else None,
                                     _stream_handle(stream, dev), ctypes.byref(handle))
        if rc != GC_OK:
            raise GcError(rc, "gc_batch_create", lib.gc_last_cuda_error())
        self._h = handle

    def run(self, *, graph: bool = False, stream=None) -> None:
        """Enqueue one coloring of the batch (as a CUDA graph replay when graph=True)."""
        import torch
        fn = self._lib.gc_batch_launch_graph if graph else self._lib.gc_batch_run
        with torch.cuda.device(self.device):
            _check(fn(self._h, _stream_handle(stream, self.device)),
                   "gc_batch_launch_graph" if graph else "gc_batch_run")

    def status(self, stream=None):
        """Wait for the last run; returns (max rounds, max colors) over the batch."""
        import torch
        r, c = ctypes.c_int32(), ctypes.c_int32()
        with torch.cuda.device(self.device):
            _check(self._lib.gc_batch_status(self._h, _stream_handle(stream, self.device), ctypes.byref(r),
                                             ctypes.byref(c)), "gc_batch_status")
        return int(r.value), int(c.value)

    def features(self, *, out=None, stream=None):
        """float32 [voff[G], 6] features of every vertex of the batch (``gc_batch_features``)."""
        import torch
        n = int(self.colors.numel())
        if out is None:
            out = torch.empty((n, 6), dtype=torch.float32, device=self.device)
        fp = _dev_ptr(out, torch.float32, "out", n * 6)
        with torch.cuda.device(self.device):
            _check(self._lib.gc_batch_features(self._h, fp, _stream_handle(stream, self.device)),
                   "gc_batch_features")
        return out

    def learned_priority(self, params=None, *, out=None, stream=None):
        """Keys of the learned priority for every graph of the batch, written into ``out``
        (pass the priority tensor the plan was created with); the trained model when
        params is None."""
        if params is None:
            params = load_priority_model(device=self.device)
        scores = mlp_forward(params, self.features(stream=stream), stream=stream)
        return priority_keys(scores, out=out, stream=stream)

    def round_stats(self, cap: int = 4096, stream=None):
        """(sizes, volumes, state_bits) of the last run over the whole batch
        (``gc_batch_round_stats``): |U_r| and the active entries round r read."""
        import torch
        sizes = np.zeros(cap, np.int32)
        vols = np.zeros(cap, np.int64)
        bits = ctypes.c_int32(0)
        with torch.cuda.device(self.device):
            m = int(self._lib.gc_batch_round_stats(self._h, ctypes.c_void_p(sizes.ctypes.data),
                                                   ctypes.c_void_p(vols.ctypes.data), cap, ctypes.byref(bits),
                                                   _stream_handle(stream, self.device)))
        if m < 0:
            raise GcError(m, "gc_batch_round_stats")
        return sizes[:m].copy(), vols[:m].copy(), int(bits.value)

    @property
    def mode(self) -> int:
        """1: the graphs share one persistent grid; 2: one thread block per graph."""
        return int(self._lib.gc_batch_mode(self._h))

    @property
    def workspace_bytes(self) -> int:
        return int(self._lib.gc_batch_workspace_bytes(self._h))

    @property
    def launch_count(self) -> int:
        return int(self._lib.gc_batch_launch_count(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.gc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- autotuning

TUNE_CANDIDATES = tuple({"small_max_degree": sm, "medium_max_degree": mm, "block_threads": bt}
                        for sm in (8, 16, 32) for mm in (64, 128, 256) for bt in (128, 256))
# batches: one block per graph, or the grid above shared by all graphs
BATCH_TUNE_CANDIDATES = (tuple({"batch_mode": 2, "local_shared_bytes": kb * 1024} for kb in (0, 132, 224))
                         + tuple(dict(c, batch_mode=1) for c in TUNE_CANDIDATES))


def _tune_cache_path() -> str:
    return os.environ.get("GC_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_1205_3809_gb300", "autotune.json")


def _degree_signature(deg: np.ndarray) -> list:
    """Size and shape of a degree sequence: n, sum, max and the share of vertices in
    each log2 degree bucket (two decimals), so graphs of one family share a key."""
    deg = np.asarray(deg, dtype=np.int64)
    if deg.size == 0:
        return [0, 0, 0]
    hist = np.bincount(np.floor(np.log2(deg + 1)).astype(np.int64))
    return [int(deg.size), int(deg.sum()), int(deg.max())] + [round(float(h) / deg.size, 2) for h in hist]


def _device_key(device) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return f"{p.name}/{p.multi_processor_count}SM"


def _cache_io(key, value=None):
    import json
    path = _tune_cache_path()
    data = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
    if value is None:
        return data.get(key)
    data[key] = value
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1)
    os.replace(tmp, path)
    return value


def _options_array(candidates):
    arr = (Options * len(candidates))()
    for i, c in enumerate(candidates):
        for k, v in dict(c).items():
            setattr(arr[i], k, int(v))
    return arr


def autotune(rowptr, colidx, priority=None, *, candidates=TUNE_CANDIDATES, reps: int = 3,
             cache: bool = True, stream=None):
    """Pick the fastest option set for this graph (``gc_tune``); results are cached per
    device and degree signature.  Returns (options dict, [(options, ms), ...])."""
    import json
    import torch
    lib = _load()
    n = int(rowptr.numel()) - 1
    key = json.dumps(["graph", _device_key(rowptr.device), priority is not None,
                      _degree_signature(np.diff(rowptr.cpu().numpy().astype(np.int64)))])
    if cache:
        hit = _cache_io(key)
        if hit is not None:
            return hit["best"], [tuple(t) for t in hit["table"]]
    cands = list(candidates)
    arr = _options_array(cands)
    ms = (ctypes.c_float * len(cands))()
    best = ctypes.c_int32()
    scratch = torch.empty(max(n, 1), dtype=torch.int32, device=rowptr.device)
    pr = None if priority is None else _dev_ptr(priority, priority.dtype, "priority", n)
    with torch.cuda.device(rowptr.device):
        _check(lib.gc_tune(_dev_ptr(rowptr, torch.int32, "rowptr", None), _dev_ptr(colidx, torch.int32, "colidx", None),
                           n, pr, ctypes.c_void_p(scratch.data_ptr()), arr, len(cands), int(reps),
                           _stream_handle(stream, rowptr.device), ms, ctypes.byref(best)), "gc_tune")
    table = [(dict(c), float(ms[i])) for i, c in enumerate(cands)]
    result = dict(cands[best.value])
    if cache:
        _cache_io(key, {"best": result, "table": table})
    return result, table


def autotune_batch(rowptr_cat, colidx_cat, vertex_offsets, edge_offsets, priority=None, *,
                   candidates=BATCH_TUNE_CANDIDATES, reps: int = 2, cache: bool = True, stream=None):
    """Pick the fastest option set for a batch (``gc_batch_tune``); cached per device and
    the batch's degree signature.  Returns (options dict, [(options, ms), ...])."""
    import json
    import torch
    lib = _load()
    voff = np.ascontiguousarray(vertex_offsets, dtype=np.int64)
    eoff = np.ascontiguousarray(edge_offsets, dtype=np.int64)
    G = int(voff.shape[0]) - 1
    N = int(voff[-1])
    rp = rowptr_cat.cpu().numpy().astype(np.int64)
    keep = np.ones(max(rp.shape[0] - 1, 0), dtype=bool)
    keep[(voff[1:] + np.arange(G))[:-1]] = False   # the step from one graph's rowptr to the next
    key = json.dumps(["batch", 2, _device_key(rowptr_cat.device), G, priority is not None,
                      _degree_signature(np.diff(rp)[keep] if rp.size > 1 else np.zeros(0))])
    if cache:
        hit = _cache_io(key)
        if hit is not None:
            return hit["best"], [tuple(t) for t in hit["table"]]
    cands = list(candidates)
    arr = _options_array(cands)
    ms = (ctypes.c_float * len(cands))()
    best = ctypes.c_int32()
    dev = rowptr_cat.device
    colors = torch.empty(max(N, 1), dtype=torch.int32, device=dev)
    nc = torch.empty(max(G, 1), dtype=torch.int32, device=dev)
    rd = torch.empty(max(G, 1), dtype=torch.int32, device=dev)
    pr = None if priority is None else _dev_ptr(priority, priority.dtype, "priority", N)
    with torch.cuda.device(dev):
        _check(lib.gc_batch_tune(_dev_ptr(rowptr_cat, torch.int32, "rowptr_cat", N + G),
                                 _dev_ptr(colidx_cat, torch.int32, "colidx_cat", int(eoff[-1])),
                                 ctypes.c_void_p(voff.ctypes.data), ctypes.c_void_p(eoff.ctypes.data), G, pr,
                                 ctypes.c_void_p(colors.data_ptr()), ctypes.c_void_p(nc.data_ptr()),
                                 ctypes.c_void_p(rd.data_ptr()), arr, len(cands), int(reps),
                                 _stream_handle(stream, dev), ms, ctypes.byref(best)), "gc_batch_tune")
    table = [(dict(c), float(ms[i])) for i, c in enumerate(cands)]
    result = dict(cands[best.value])
    if cache:
        _cache_io(key, {"best": result, "table": table})
    return result, table
