"""CPU checks of the C ABI: the library builds and loads, exports every entry
point include/mf.h declares, the ctypes layouts match the C structs, and
argument validation that happens before any CUDA call reports errors."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mf.h")


@pytest.fixture(scope="module")
def mflib():
    from paper_2309_00019_gb300 import _build, mf
    _build.build()
    return mf


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:mf_status|void|const char\*)\s+(mf_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_entry_points():
    fns = header_functions()
    for name in ["mf_plan", "mf_set_psd", "mf_load_bank", "mf_filter", "mf_get_triggers", "mf_destroy",
                 "mf_last_error", "mf_coincide", "mf_nbhd_union", "mf_strain_to_fd", "mf_decimate"]:
        assert name in fns


def test_library_exports_every_declared_symbol(mflib):
    lib = C.CDLL(mflib.LIB_PATH)
    for name in header_functions():
        assert hasattr(lib, name), name
    # the binding covers every declared function
    assert set(header_functions()) <= set(mflib.SIGNATURES) | {"mf_plan"}


def test_struct_layouts(mflib):
    assert C.sizeof(mflib.mf_trigger) == 24
    assert C.sizeof(mflib.mf_coinc) == 40
    assert C.sizeof(mflib.mf_plan_desc) == 96
    assert C.sizeof(mflib.mf_coinc_desc) == 48
    assert C.sizeof(mflib.mf_batch_desc) == 88
    assert C.sizeof(mflib.mf_batch_trigger) == 32 == mflib.BATCH_TRIGGER_NP.itemsize


@pytest.mark.parametrize("field,value", [("n", 3000), ("n", 1 << 11), ("n", 1 << 21), ("n_det", 0), ("fs", 0.0),
                                         ("snr_thr", 0.0), ("window", 0), ("valid_end", 0), ("max_triggers", 0),
                                         ("f_high", 10.0)])
def test_plan_rejects_invalid_descriptions(mflib, field, value):
    lib = mflib.load()
    d = mflib.mf_plan_desc(fs=512.0, n=4096, n_det=1, f_low=20.0, f_high=256.0, dtype=0, snr_thr=5.0, window=512,
                           valid_begin=0, valid_end=4096, max_triggers=100, cuda_stream=None)
    setattr(d, field, value)
    h = C.c_void_p()
    st = lib.mf_plan(C.byref(h), C.byref(d))
    assert st == mflib.MF_EINVAL
    assert h.value is None
    assert lib.mf_last_error(None).decode().startswith("mf_plan")


def test_null_arguments_are_rejected_without_a_device(mflib):
    lib = mflib.load()
    assert lib.mf_plan(None, None) == mflib.MF_EINVAL
    assert lib.mf_set_psd(None, None, 0) == mflib.MF_EINVAL
    assert lib.mf_filter(None, None, 0, None, 0) == mflib.MF_EINVAL
    lib.mf_destroy(None)  # no-op


def test_batch_rejects_invalid_descriptions(mflib):
    lib = mflib.load()
    lens = (C.c_double * 2)(4.0, 16.0)
    ok = dict(fs=2048.0, n_det=2, n_samples=1 << 20, f_low=25.0, f_high=1024.0, snr_thr=5.0, window=2048, n_class=2,
              class_len=lens, max_triggers=1000, cuda_stream=None)
    for field, value in [("n_det", 0), ("n_det", 9), ("n_class", 0), ("n_class", 9), ("window", 0), ("fs", 0.0),
                         ("snr_thr", 0.0), ("max_triggers", 0)]:
        d = mflib.mf_batch_desc(**{**ok, field: value})
        h = C.c_void_p()
        assert lib.mf_batch_create(C.byref(h), C.byref(d)) == mflib.MF_EINVAL
        assert h.value is None
    bad = (C.c_double * 2)(16.0, 4.0)  # not increasing
    d = mflib.mf_batch_desc(**{**ok, "class_len": bad})
    h = C.c_void_p()
    assert lib.mf_batch_create(C.byref(h), C.byref(d)) == mflib.MF_EINVAL
    assert lib.mf_batch_run(None, None, 0, 0) == mflib.MF_EINVAL
    lib.mf_batch_destroy(None)
