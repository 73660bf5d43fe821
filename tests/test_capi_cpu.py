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


def test_way_back_and_classifier_reject_bad_arguments(lib):
    """rsc_reconstruct, rsc_synthesize and rsc_classify_images validate their
    arguments before any CUDA call (no GPU needed)."""
    import paper_1806_04374_gb300 as rsc
    inv = rsc.RSC_ERR_INVALID
    vp = ctypes.c_void_p
    # null dictionary / basis handles, bad sizes
    assert lib.rsc_reconstruct(None, 10, 3, None, None, None, None, None) == inv
    assert lib.rsc_reconstruct(None, -1, 3, None, None, None, None, None) == inv
    assert lib.rsc_synthesize(None, None, 10, None, None) == inv
    assert lib.rsc_synthesize(None, None, -1, None, None) == inv
    # classifier: no dictionaries, C = 0, no histogram, bad K
    one = (vp * 1)(None)
    assert lib.rsc_classify_images(None, 1, None, None, None, None, 0, 3, 0, None, None,
                                   None) == inv
    assert lib.rsc_classify_images(one, 0, None, None, None, None, 0, 3, 0, None, None,
                                   None) == inv
    assert lib.rsc_classify_images(one, 1, None, None, None, None, 0, 0, 0, None, None,
                                   None) == inv


def test_workspace_query_argument_checks(lib):
    import paper_1806_04374_gb300 as rsc
    out = ctypes.c_uint64()
    vp = ctypes.c_void_p
    assert lib.rsc_workspace_bytes(vp(None), vp(None), 10, 1, 5, rsc.RSC_F16_RESCORE,
                                   ctypes.byref(out)) == rsc.RSC_ERR_INVALID
    with pytest.raises(rsc.RscError):
        rsc.rsc_workspace_bytes(0, None, 10, 1, 5, rsc.RSC_FP32)
    assert lib.rsc_dict_set_limits(vp(None), 1, 1) == rsc.RSC_ERR_INVALID


def test_binding_constants_match_the_header():
    """Every #define of include/rsc.h (status codes, precisions) has the same
    value in the Python binding."""
    import re
    import paper_1806_04374_gb300 as rsc
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "include", "rsc.h")).read()
    defs = dict(re.findall(r"#define (RSC_[A-Z0-9_]+) \(?(-?\d+)\)?", hdr))
    assert {"RSC_OK", "RSC_FP32", "RSC_F16_RESCORE", "RSC_FP32_PRUNE"} <= set(defs)
    for name, v in defs.items():
        assert getattr(rsc, name) == int(v), name
    assert rsc.PRECISIONS == {"fp32": 0, "f16": 2, "fp32_prune": 3}
