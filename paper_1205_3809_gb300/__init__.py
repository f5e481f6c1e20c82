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
            "gc_last_round_stats", "gc_last_phase_ms", "gc_color_noalloc", "gc_noalloc_capacity_bytes",
            "gc_features", "gc_mlp_param_count", "gc_mlp_forward", "gc_mlp_grad", "gc_mlp_adam",
            "gc_priority_keys", "gc_mlp_train_step")


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
           "-Xcompiler", "-fPIC", "-shared", "-I", _INCLUDE, "--threads", "2", "-o", LIB_PATH + ".tmp",
           os.path.join(_CSRC, "gc.cu"), os.path.join(_CSRC, "gc_mlp.cu")]
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
                ("narrow_color_limit", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]


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
        lib.gc_last_phase_ms.argtypes = [vp, i32]
        for f in (lib.gc_color, lib.gc_color_ex, lib.gc_color_host, lib.gc_validate_csr,
                  lib.gc_last_cuda_error, lib.gc_release, lib.gc_last_round_stats,
                  lib.gc_last_phase_ms):
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
