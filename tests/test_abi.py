"""The C-ABI library builds, loads and exports what include/fdas.h declares.

These run without a GPU: they check the build, the exported symbols, the
struct layouts the binding relies on, and the argument validation that every
entry point performs before touching CUDA.
"""
import ctypes
import importlib
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    import paper_2211_13517_gb300 as pkg
    pkg.build()
    from paper_2211_13517_gb300 import capi as c
    c.lib()
    return c


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fdas_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(capi):
    declared = _declared_symbols()
    assert "fdas_search" in declared and "fdas_plan_create" in declared
    lib = ctypes.CDLL(capi.LIB)
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding covers every one of them under the same name
    assert set(capi.EXPORTED) == declared


def test_struct_layouts(capi):
    assert ctypes.sizeof(capi.fdas_candidate) == 20
    assert ctypes.sizeof(capi.fdas_series) == 24
    assert ctypes.sizeof(capi.fdas_opts) == 64
    assert ctypes.sizeof(capi.fdas_plan_info) == 192
    assert capi.CANDIDATE_DTYPE.itemsize == 20
    assert ctypes.sizeof(capi.fdas_seed) == capi.SEED_DTYPE.itemsize == 24
    assert ctypes.sizeof(capi.fdas_refined) == capi.REFINED_DTYPE.itemsize == 40


def test_dedisp_info_layout_and_validation(capi):
    assert ctypes.sizeof(capi.fdas_dedisp_info) == 80
    bad = [
        ((0, 1000, 1400.0, 1.0, 64e-6, 0.0, 1.0, 4, 500), "n_chan"),
        ((16, 1000, 1400.0, 1.0, 64e-6, 0.0, 1.0, 0, 500), "n_dm"),
        ((16, 1000, 1400.0, 1.0, 64e-6, 0.0, 1.0, 4, 1001), "n_out"),
        ((16, 1000, 1400.0, 100.0, 64e-6, 0.0, 1.0, 4, 500), "lowest channel"),
        ((16, 1000, 1400.0, 1.0, 0.0, 0.0, 1.0, 4, 500), "tsamp"),
        ((16, 1000, 1400.0, 1.0, 64e-6, -1.0, 1.0, 4, 500), "dm_lo"),
    ]
    for args, frag in bad:
        with pytest.raises(capi.FdasError) as ei:
            capi.fdas_dedisp_plan_create(*args)
        assert ei.value.status == capi.FDAS_ERR_ARG and frag in str(ei.value), (args, str(ei.value))
    lib = capi.lib()
    assert lib.fdas_dedisperse(None, None, None, None) == capi.FDAS_ERR_ARG
    assert lib.fdas_dedisp_delays(None, None) == capi.FDAS_ERR_ARG
    lib.fdas_dedisp_plan_destroy(None)


def test_defaults_and_version(capi):
    o = capi.fdas_opts_default()
    assert o.precision == capi.FDAS_FP32 and o.threshold_sigma == 6.0
    assert o.norm_block == 2048 and o.max_candidates == 1 << 20
    assert "sm_103a" in capi.fdas_version()


@pytest.mark.parametrize("args,frag", [
    ((1000, 64e-6, 16.0, 2.0, 2048, 4), "n_samples"),
    ((1 << 25, 64e-6, 16.0, 2.0, 2048, 4), "n_samples"),
    ((1 << 17, 64e-6, 16.0, 3.0, 2048, 4), "integer"),
    ((1 << 17, 64e-6, 16.0, 2.0, 2048, 3), "n_harm"),
    ((1 << 17, 64e-6, 16.0, 2.0, 1000, 4), "seg_len"),
    ((1 << 17, 64e-6, 16.0, 2.0, 32768, 4), "seg_len"),
    ((1 << 17, 64e-6, 1000.0, 1.0, 1024, 4), "seg_len must exceed"),
    ((1 << 17, 0.0, 16.0, 2.0, 2048, 4), "tsamp"),
    ((1 << 17, 64e-6, 16.0, -1.0, 2048, 4), "z_step"),
])
def test_plan_argument_validation(capi, args, frag):
    with pytest.raises(capi.FdasError) as ei:
        capi.fdas_plan_create(*args)
    assert ei.value.status == capi.FDAS_ERR_ARG
    assert frag in str(ei.value)


def test_opts_validation(capi):
    o = capi.fdas_opts_default()
    o.norm_block = 1000
    with pytest.raises(capi.FdasError) as ei:
        capi.fdas_plan_create(1 << 17, 64e-6, 16.0, 2.0, 2048, 4, o)
    assert ei.value.status == capi.FDAS_ERR_ARG
    o = capi.fdas_opts_default()
    o.precision = 7
    with pytest.raises(capi.FdasError):
        capi.fdas_plan_create(1 << 17, 64e-6, 16.0, 2.0, 2048, 4, o)
    o = capi.fdas_opts_default()
    o.interbin = 2
    with pytest.raises(capi.FdasError) as ei:
        capi.fdas_plan_create(1 << 17, 64e-6, 16.0, 2.0, 2048, 4, o)
    assert ei.value.status == capi.FDAS_ERR_ARG and "interbin" in str(ei.value)
    # the split tensor-core correlation is for FP32 storage, without interbinning
    o = capi.fdas_opts_default()
    o.correlator = capi.FDAS_CORR_TENSOR_SPLIT
    o.precision = capi.FDAS_BF16
    with pytest.raises(capi.FdasError) as ei:
        capi.fdas_plan_create(1 << 17, 64e-6, 16.0, 2.0, 2048, 4, o)
    assert ei.value.status == capi.FDAS_ERR_ARG and "FP32" in str(ei.value)
    o.precision = capi.FDAS_FP32
    o.interbin = 1
    with pytest.raises(capi.FdasError) as ei:
        capi.fdas_plan_create(1 << 17, 64e-6, 16.0, 2.0, 2048, 4, o)
    assert ei.value.status == capi.FDAS_ERR_ARG and "interbinning" in str(ei.value)
    # the half-bin plane of a 2^24-sample series has 2^24 columns: refused
    o = capi.fdas_opts_default()
    o.interbin = 1
    with pytest.raises(capi.FdasError) as ei:
        capi.fdas_plan_create(1 << 24, 64e-6, 16.0, 2.0, 2048, 4, o)
    assert ei.value.status == capi.FDAS_ERR_ARG and "2^23" in str(ei.value)
    # the template order of the tensor-core chunks takes the three enumerators
    for bad in (-1, 3):
        o = capi.fdas_opts_default()
        o.template_order = bad
        with pytest.raises(capi.FdasError) as ei:
            capi.fdas_plan_create(1 << 17, 64e-6, 16.0, 2.0, 2048, 4, o)
        assert ei.value.status == capi.FDAS_ERR_ARG and "template_order" in str(ei.value)


def test_null_arguments_rejected(capi):
    lib = capi.lib()
    assert lib.fdas_search(None, None, 0, None, 0, None, None) == capi.FDAS_ERR_ARG
    assert lib.fdas_plan_get_info(None, None) == capi.FDAS_ERR_ARG
    assert "NULL" in capi.fdas_last_error() or "plan" in capi.fdas_last_error()
    lib.fdas_plan_destroy(None)   # ignored
    assert lib.fdas_selftest_wait_timeout(None, 1000, None) == capi.FDAS_ERR_ARG
    assert lib.fdas_refine(None, None, None, 0, 0, None, None) == capi.FDAS_ERR_ARG
    assert lib.fdas_correlation_plane(None, None, None, None) == capi.FDAS_ERR_ARG


def test_binding_constants_match_the_header(capi):
    """Every enumerator of include/fdas.h has the same value in the binding."""
    import re
    src = open(os.path.join(ROOT, "include", "fdas.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    found = 0
    for body in re.findall(r"enum\s*\{([^}]*)\}", src):
        for name, val in re.findall(r"(FDAS_[A-Z0-9_]+)\s*=\s*(\d+)", body):
            assert hasattr(capi, name), name
            assert getattr(capi, name) == int(val), (name, getattr(capi, name), val)
            found += 1
    assert found >= 20


def test_fault_injection_reaches_argument_checks_without_a_gpu(capi, monkeypatch):
    """FDAS_FAULT=bad_args makes fdas_plan_create refuse valid arguments
    before any CUDA call; an unknown FDAS_FAULT value is refused by name."""
    good = (1 << 17, 64e-6, 16.0, 2.0, 2048, 4)
    monkeypatch.setenv("FDAS_FAULT", "bad_args")
    with pytest.raises(capi.FdasError) as ei:
        capi.fdas_plan_create(*good)
    assert ei.value.status == capi.FDAS_ERR_ARG and "injected" in str(ei.value)
    for bad in ("alloc:0", "allocate", "nonsense"):
        monkeypatch.setenv("FDAS_FAULT", bad)
        with pytest.raises(capi.FdasError) as ei:
            capi.fdas_plan_create(*good)
        assert ei.value.status == capi.FDAS_ERR_ARG and bad in str(ei.value)
    # a plan that passes validation then needs the device (none here)
    monkeypatch.setenv("FDAS_FAULT", "")
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if not have_gpu:
        with pytest.raises(capi.FdasError) as ei:
            capi.fdas_plan_create(*good)
        assert ei.value.status == capi.FDAS_ERR_CUDA


def test_store_full_status_is_returned_not_raised(capi):
    assert capi.FDAS_ERR_CAND_STORE_FULL == 8
    assert capi.FDAS_ERR_CAND_STORE_FULL in capi.COUNT_STATUSES
    assert capi.STATUS_NAMES[8] == "FDAS_ERR_CAND_STORE_FULL"


def test_checked_build_exports_the_same_symbols(capi):
    """The checked build (-DFDAS_CHECK_BOUNDS) links, exports every declared
    symbol and says so; the ordinary build says it is not."""
    path = importlib.import_module("paper_2211_13517_gb300.build").build(checked=True)
    assert os.path.basename(path) == "libfdas_checked.so" and path != capi.LIB
    chk = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared_symbols()) if not hasattr(chk, n)]
    assert not missing, missing
    chk.fdas_checked_build.restype = ctypes.c_int32
    chk.fdas_version.restype = ctypes.c_char_p
    assert chk.fdas_checked_build() == 1 and b"checked" in chk.fdas_version()
    plain = ctypes.CDLL(capi.LIB)
    plain.fdas_checked_build.restype = ctypes.c_int32
    assert plain.fdas_checked_build() == 0
    assert capi.STATUS_NAMES[capi.FDAS_ERR_BOUNDS] == "FDAS_ERR_BOUNDS"


def test_checked_faults_need_the_checked_build(capi, monkeypatch):
    """FDAS_FAULT=canary / bounds are refused by the ordinary build before any
    CUDA call (FDAS_ERR_UNSUPPORTED, naming the checked build)."""
    if capi.fdas_checked_build():
        pytest.skip("the checked build takes these faults")
    good = (1 << 17, 64e-6, 16.0, 2.0, 2048, 4)
    for fault in ("canary", "bounds"):
        monkeypatch.setenv("FDAS_FAULT", fault)
        with pytest.raises(capi.FdasError) as ei:
            capi.fdas_plan_create(*good)
        assert ei.value.status == capi.FDAS_ERR_UNSUPPORTED
        assert "checked build" in str(ei.value) and fault in str(ei.value)
