"""The C ABI library loads and exports every symbol include/gc.h declares (no GPU
needed: nothing here launches work)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "gc.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|size_t|const char\*)\s+(gc_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    import paper_1205_3809_gb300 as m
    try:
        m.build()
    except (FileNotFoundError, subprocess.CalledProcessError) as e:  # no nvcc here
        pytest.skip(f"cannot build libgc.so: {e}")
    return ctypes.CDLL(m.LIB_PATH)


def test_header_declares_expected_entry_points():
    import paper_1205_3809_gb300 as m
    assert set(_declared()) == set(m.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_strerror_without_gpu(lib):
    lib.gc_strerror.restype = ctypes.c_char_p
    assert lib.gc_strerror(0) == b"ok"
    assert b"max_rounds" in lib.gc_strerror(-4)


def test_no_cpu_fallback_in_binding():
    """The binding marshals arguments only: it never imports the oracle."""
    src = open(os.path.join(ROOT, "paper_1205_3809_gb300", "__init__.py")).read()
    assert "oracle" not in src.replace("oracle.", "")
    assert "import oracle" not in src


def test_options_struct_mirrors_header():
    """Options (ctypes) has the fields of gc_options, in the header's order, all int32."""
    import paper_1205_3809_gb300 as m
    text = open(os.path.join(ROOT, "include", "gc.h")).read()
    body = text[text.index("typedef struct gc_options {"):text.index("} gc_options;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"int32_t\s+(\w+)(?:\[(\d+)\])?\s*;", body)
    names = [f for f, _ in fields]
    assert names == [f for f, _ in m.Options._fields_]
    width = sum(int(n) if n else 1 for _, n in fields)
    assert ctypes.sizeof(m.Options) == 4 * width


def test_color_batched_rejects_bad_offsets_before_any_device_call(lib):
    """gc_color_batched (the one-call batch entry point) checks its host offset
    arrays first: NULL offsets, offsets that do not start at 0 or decrease, and a
    loop_mode the batch kernels do not have are GC_ERR_INVALID, with no GPU."""
    import paper_1205_3809_gb300 as m
    i64 = ctypes.c_int64
    f = lib.gc_color_batched
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 7 + \
                 [ctypes.POINTER(m.Options)]

    def call(voff, eoff, g, opt=None):
        va = (i64 * len(voff))(*voff) if voff is not None else None
        ea = (i64 * len(eoff))(*eoff) if eoff is not None else None
        return f(ctypes.cast(va, ctypes.c_void_p) if va else None, ctypes.cast(ea, ctypes.c_void_p) if ea else None,
                 g, None, None, None, None, None, None, None, ctypes.byref(opt) if opt else None)

    assert call(None, None, 1) == m.GC_ERR_INVALID
    assert call([0, 4], None, 1) == m.GC_ERR_INVALID
    assert call([1, 4], [0, 6], 1) == m.GC_ERR_INVALID           # vertex offsets must start at 0
    assert call([0, 4, 3], [0, 6, 8], 2) == m.GC_ERR_INVALID     # decreasing vertex offsets
    assert call([0, 4, 5], [0, 6, 2], 2) == m.GC_ERR_INVALID     # decreasing edge offsets
    assert call([0, 4], [0, 6], -1) == m.GC_ERR_INVALID          # negative graph count
    o = m.Options()
    o.loop_mode = 1
    assert call([0, 4], [0, 6], 1, o) == m.GC_ERR_INVALID
