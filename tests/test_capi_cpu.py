"""The C-ABI library builds, loads without a GPU and exports every function
include/rsc.h declares; argument checks that need no device work on CPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1806_04374_gb300 import build
    path = build.build()
    import paper_1806_04374_gb300 as rsc
    return rsc.load_library(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rsc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rsc_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    import paper_1806_04374_gb300 as rsc
    assert set(names) == set(rsc.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_host_only_calls(lib):
    import paper_1806_04374_gb300 as rsc
    assert rsc.rsc_version() >> 16 == 1
    assert rsc.rsc_status_string(rsc.RSC_ERR_INVALID) == "invalid argument"
    assert rsc.rsc_dict_destroy(0) == 0
    # null handle / null out-pointer: rejected before any CUDA call
    assert rsc.rsc_encode(0, 0, 10, 3, 0, 0, 0, 0, 0, 0) == rsc.RSC_ERR_INVALID
    assert lib.rsc_dict_create(None, rsc.rsc_dims(4, 6, 8, 8), None, None) == rsc.RSC_ERR_INVALID
    h = ctypes.c_void_p()
    assert lib.rsc_dict_create(None, rsc.rsc_dims(0, 6, 8, 8), None,
                               ctypes.byref(h)) == rsc.RSC_ERR_INVALID
    assert rsc.rsc_encode_host(0, 0, 10, 3, 0, 0, 0, 0, 0, 0) == rsc.RSC_ERR_INVALID
