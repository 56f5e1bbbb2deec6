"""The C ABI library builds, loads without a GPU and exports every function that
include/pp.h declares; the ctypes binding declares the same set.  No compute call runs."""
import ctypes
import os
import re

from paper_2502_10640_gb300 import build, capi

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "pp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_documented_entry_points():
    names = declared_functions()
    for required in ("pp_create", "pp_set_option", "pp_load_particles", "pp_compute_fields",
                     "pp_step", "pp_diagnostics", "pp_get_particles", "pp_get_state",
                     "pp_set_state", "pp_destroy", "pp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    bound = {name for name, _, _ in capi.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_host_only_calls():
    assert "sm_103a" in capi.pp_version()
    assert capi.pp_pairs_per_step(65536) == 65536.0 ** 2
    try:
        capi.pp_create(0, 1.0, 1e-15, 0.0)
    except capi.PPError as e:
        assert e.status == capi.PP_ERR_ARG
        assert "N must be" in str(e)
    else:
        raise AssertionError("N = 0 accepted")


def test_binding_constants_match_the_header():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    values = dict(re.findall(r"\b(PP_[A-Z0-9_]+)\s*=\s*(-?\d+)", text))
    assert {"PP_MEM_HOST", "PP_MEM_DEVICE", "PP_MEM_HOST_MAPPED", "PP_ACC_KAHAN",
            "PP_POS_AUTO", "PP_ERR_STATE"} <= set(values)
    for name, value in values.items():
        assert getattr(capi, name) == int(value), name
    defines = dict(re.findall(r"#define\s+(PP_[A-Z0-9_]+)\s+(\d+)", text))
    assert {"PP_FRAME_LEN", "PP_FIELDS_NOALLOC_MAX_N"} <= set(defines)
    for name, value in defines.items():
        assert getattr(capi, name) == int(value), name
