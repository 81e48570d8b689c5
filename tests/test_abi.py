"""The C-ABI library loads without a GPU and exports every entry point include/swift_gpu.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_14538_b300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(swift_gpu_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_abi():
    from paper_2505_14538_b300 import _lib
    assert set(declared()) == set(_lib.EXPORTED)


def test_default_params_and_argument_checks_without_gpu(lib):
    from paper_2505_14538_b300 import _lib
    p = _lib.default_params()
    assert abs(p.kernel_gamma - 1.825742) < 1e-6 and abs(p.eta - 1.2348) < 1e-6 and p.max_iter == 30
    L = _lib.load()
    h = ctypes.c_void_p()
    assert L.swift_gpu_create(ctypes.byref(h), ctypes.byref(p), ctypes.c_int64(0)) == _lib.ERR_ARG
    assert L.swift_gpu_create(None, ctypes.byref(p), ctypes.c_int64(10)) == _lib.ERR_ARG
    bad = _lib.default_params()
    bad.max_iter = 0
    assert L.swift_gpu_create(ctypes.byref(h), ctypes.byref(bad), ctypes.c_int64(10)) == _lib.ERR_ARG
    bad = _lib.default_params()
    bad.flags = _lib.FLAG_ADAPTIVE
    bad.leaf_margin = 0.0  # a leaf cap equal to its largest h leaves no room to grow
    assert L.swift_gpu_create(ctypes.byref(h), ctypes.byref(bad), ctypes.c_int64(10)) == _lib.ERR_ARG
    bad.leaf_margin = 0.01
    bad.leaf_max = 4
    assert L.swift_gpu_create(ctypes.byref(h), ctypes.byref(bad), ctypes.c_int64(10)) == _lib.ERR_ARG
    assert L.swift_gpu_destroy(None) == _lib.OK
    assert L.swift_gpu_density(None, None, None, None, None, None, None, None, None) == _lib.ERR_ARG


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2505_14538_b300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "sph_oracle" not in text, fn
