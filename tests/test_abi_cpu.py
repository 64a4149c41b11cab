"""C-ABI library checks that need no GPU: the library loads, exports every
function include/upir.h declares, and its host-only calls behave."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "upir.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(upir_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for must in ("upir_init", "upir_finalize", "upir_data_map", "upir_data_unmap", "upir_spmd_region",
                 "upir_loop", "upir_sync", "upir_region_submit", "upir_batch_create", "upir_ctx_wait"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_2209_10643_b300 as U
    out = subprocess.run(["nm", "-D", "--defined-only", U.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(upir_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(U.lib, n)
        assert n in U.EXPORTED  # the binding declares a signature for each


def test_status_strings_are_static_and_distinct():
    import paper_2209_10643_b300 as U
    codes = [U.UPIR_OK, U.UPIR_EINVAL, U.UPIR_ENOTMAPPED, U.UPIR_EBUSY, U.UPIR_ENOMEM,
             U.UPIR_ECUDA, U.UPIR_ETIMEDOUT, U.UPIR_EUNSUPPORTED]
    texts = [U.status_string(c) for c in codes]
    assert len(set(texts)) == len(texts)
    assert U.status_string(12345) == "unknown upir_status"


def test_null_handles_are_rejected_without_a_gpu():
    import paper_2209_10643_b300 as U
    assert U.lib.upir_finalize(None) == U.UPIR_OK
    assert U.lib.upir_region_submit(None, 0) == U.UPIR_EINVAL
    assert U.lib.upir_loop(None, None) == U.UPIR_EINVAL
    assert U.lib.upir_sync(None, 0) == U.UPIR_EINVAL
    assert U.lib.upir_ctx_wait(None) == U.UPIR_EINVAL
    assert U.lib.upir_init(None, 0, None, None) == U.UPIR_EINVAL
    assert U.lib.upir_data_unmap(None, None) == U.UPIR_EINVAL


def test_init_without_a_device_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2209_10643_b300 as U
    h = ctypes.c_void_p()
    st = U.lib.upir_init(ctypes.byref(h), 0, None, None)
    assert st in (U.UPIR_ECUDA, U.UPIR_EINVAL) and not h.value
    with pytest.raises(U.UpirError):
        U.upir_init(0)
