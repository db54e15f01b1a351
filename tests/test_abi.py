"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/turtle.h declares.

No compute runs here (there may be no GPU); the only device query is the
device count behind TURTLE_E_NODEV.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w \*]*?\b(turtle_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_1305_1861_gb300 as pkg

    pkg.build()
    return pkg.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("turtle_count", "turtle_count_ex", "turtle_result_free", "turtle_strerror", "turtle_count_device",
                 "turtle_ctx_create", "turtle_ctx_destroy", "turtle_extract", "turtle_filter",
                 "turtle_sort_compact"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_build_targets_sm103a_only():
    from paper_1305_1861_gb300 import _nvcc

    assert _nvcc.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_side_helpers(lib):
    import paper_1305_1861_gb300 as pkg

    p = pkg.Params.default()
    assert p.struct_size == ctypes.sizeof(pkg.Params) and p.pattern_bits == 4 and p.n_patterns == 1024
    assert pkg.turtle_strerror(-1) == "invalid argument"
    assert lib.turtle_stage_name(2) == b"filter"


def test_argument_errors_need_no_device(lib):
    import numpy as np

    import paper_1305_1861_gb300 as pkg

    b = np.frombuffer(b"ACGTACGT", dtype=np.uint8)
    with pytest.raises(pkg.TurtleError) as e:
        pkg.turtle_count(b, np.array([0, 8], dtype=np.uint64), 0, 2)
    assert e.value.code == -1
    with pytest.raises(pkg.TurtleError) as e:
        pkg.turtle_count(b, np.array([0, 8], dtype=np.uint64), 65, 2)
    assert e.value.code == -1
    with pytest.raises(pkg.TurtleError) as e:
        pkg.turtle_count(b, np.array([0, 8], dtype=np.uint64), 31, 0)
    assert e.value.code == -1
    with pytest.raises(pkg.TurtleError) as e:
        pkg.turtle_count(b, np.array([5, 3], dtype=np.uint64), 3, 2)
    assert e.value.code == -1


def test_no_device_reports_nodev(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.turtle_ctx_create(0, ctypes.byref(h)) == -8


def test_misaligned_buffers_are_refused_before_any_device_work(lib):
    """Buffers read or written as whole keys must be aligned to the key width; the allocation-free
    sort-and-compact checks this before it touches a device, so fake (never dereferenced) pointer
    values suffice here."""
    nu = ctypes.c_uint64(99)
    fn = lib.turtle_sort_compact_noalloc
    good16, good8, good4 = 0x10000, 0x20000, 0x30000
    # 128-bit keys need a 16-byte-aligned unique buffer; 8-byte alignment is not enough
    assert fn(ctypes.c_void_p(good8), 4, 2, 100, ctypes.c_void_p(good16 + 8), ctypes.c_void_p(good4),
              ctypes.byref(nu), None) == -1
    # keys on 8 bytes, counts on 4 bytes
    assert fn(ctypes.c_void_p(good8 + 4), 4, 1, 62, ctypes.c_void_p(good8), ctypes.c_void_p(good4),
              ctypes.byref(nu), None) == -1
    assert fn(ctypes.c_void_p(good8), 4, 1, 62, ctypes.c_void_p(good8), ctypes.c_void_p(good4 + 2),
              ctypes.byref(nu), None) == -1
    assert nu.value == 99  # refused before any output was written
