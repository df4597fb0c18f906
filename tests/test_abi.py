"""The C-ABI library loads and exports every entry point of include/mrf.h;
host-side argument checks work without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mrf():
    from paper_2309_04581_gb300 import build
    build.build()
    import paper_2309_04581_gb300.mrf as m
    return m


def _declared():
    src = open(os.path.join(ROOT, "include", "mrf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mrf_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree(mrf):
    assert _declared() == sorted(mrf.EXPORTS)


def test_library_exports_every_declared_symbol(mrf):
    lib = mrf.lib()
    for name in _declared():
        assert hasattr(lib, name), name
    assert lib.mrf_version().decode().count(".") == 2


def test_null_arguments_are_rejected_without_a_gpu(mrf):
    lib = mrf.lib()
    assert lib.mrf_context_create(0, None) == mrf.MRF_ERR_INVALID_ARG
    assert b"NULL" in lib.mrf_last_error()
    out = C.c_void_p()
    assert lib.mrf_field_create(None, None, C.byref(out)) == mrf.MRF_ERR_INVALID_ARG
    assert lib.mrf_bvh_build(None, None, 0, None, None, 0, C.byref(out)) == mrf.MRF_ERR_INVALID_ARG
    assert lib.mrf_render(None, None, None, None, 1, None, None, None, None) == mrf.MRF_ERR_INVALID_ARG
    assert lib.mrf_bvh_refit(None, None, 3, None) == mrf.MRF_ERR_INVALID_ARG
    assert lib.mrf_materials_set(None, None, 0) == mrf.MRF_ERR_INVALID_ARG
    # destroy functions accept NULL
    lib.mrf_context_destroy(None)
    lib.mrf_field_destroy(None)
    lib.mrf_bvh_destroy(None)


def test_context_create_reports_missing_device(mrf):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = mrf.lib()
    h = C.c_void_p()
    st = lib.mrf_context_create(0, C.byref(h))
    assert st in (mrf.MRF_ERR_CUDA, mrf.MRF_ERR_INVALID_ARG)
    assert h.value is None
    assert lib.mrf_last_error()
