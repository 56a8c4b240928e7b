"""The C ABI: libtc.so builds for sm_103a, loads without a GPU, and exports
every function include/tc.h declares (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tc_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1211_2293_gb300 import build

    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib_path):
    from paper_1211_2293_gb300 import tc

    assert sorted(tc.EXPORTS) == _declared()
    tc.load(lib_path)


def test_config_struct_matches_header():
    from paper_1211_2293_gb300 import tc

    src = open(os.path.join(ROOT, "include", "tc.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} tc_config;", src, flags=re.S).group(1)
    fields = re.findall(r"int32_t\s+(\w+);", body)
    assert fields == [f for f, _ in tc.tc_config._fields_]


def test_no_oracle_in_product_path():
    pkg = os.path.join(ROOT, "paper_1211_2293_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "tc_oracle" not in txt, f


def test_direct_static_binding_rejects_bad_arguments_before_the_call(monkeypatch):
    """The binding checks element types, shapes and devices before the C ABI
    sees a pointer: a float32 acc, short outputs, an int32 idx or CPU
    tensors would otherwise make the kernels read or write outside the
    caller's buffers.  The library is never loaded for a rejected call."""
    import torch

    from paper_1211_2293_gb300 import tc

    def no_load(*a, **k):
        raise AssertionError("the library was reached")

    monkeypatch.setattr(tc, "load", no_load)
    n, ns = 10, 4
    good = dict(pos=torch.zeros((n, 3)), mass=torch.ones(n), idx=torch.zeros(ns, dtype=torch.int64),
                acc=torch.zeros((ns, 3), dtype=torch.float64), pot=torch.zeros(ns, dtype=torch.float64))
    cases = [
        ("acc", torch.zeros((ns, 3), dtype=torch.float32), TypeError),
        ("acc", torch.zeros((ns - 1, 3), dtype=torch.float64), ValueError),
        ("pot", torch.zeros(ns - 1, dtype=torch.float64), ValueError),
        ("pot", torch.zeros(ns, dtype=torch.float32), TypeError),
        ("idx", torch.zeros(ns, dtype=torch.int32), TypeError),
        ("pos", torch.zeros((n, 4)), ValueError),
        ("pos", torch.zeros((n, 3), dtype=torch.float64), TypeError),
        ("mass", torch.ones((n, 1)), ValueError),
        ("acc", torch.zeros((3, ns), dtype=torch.float64).t(), ValueError),  # not contiguous
        ("pos", np.zeros((n, 3), np.float32), TypeError),
    ]
    for name, bad, exc in cases:
        kw = dict(good)
        kw[name] = bad
        with pytest.raises(exc):
            tc.tc_direct_static(kw["pos"], kw["mass"], kw["idx"], 0.01, 1.0, kw["acc"], kw["pot"])
    # right types and shapes, but host tensors: refused as not on a CUDA device
    with pytest.raises(ValueError, match="CUDA"):
        tc.tc_direct_static(good["pos"], good["mass"], good["idx"], 0.01, 1.0, good["acc"], good["pot"])
