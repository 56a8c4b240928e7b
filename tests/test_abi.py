"""The C ABI: libtc.so builds for sm_103a, loads without a GPU, and exports
every function include/tc.h declares (no compute calls here)."""
import ctypes
import os
import re

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
