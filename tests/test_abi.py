"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/hdda.h declares.  No compute call is made (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hdda.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hdda_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2404_10272_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["hdda_pack_dense", "hdda_build_vdb", "hdda_traverse_dense",
                     "hdda_traverse_hdda", "hdda_composite", "hdda_last_error", "hdda_grid_free"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in hdda.h but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (hdda_[a-z_0-9]+)$", out, flags=re.M))
    assert exported == set(declared_functions()), exported ^ set(declared_functions())


def test_version_and_error_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.hdda_version.restype = ctypes.c_char_p
    lib.hdda_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.hdda_version()
    assert lib.hdda_last_error() == b""


def test_binding_names_match_header():
    from paper_2404_10272_gb300 import hdda
    assert sorted(hdda.EXPORTED) == declared_functions()



def test_region_check_switch_is_host_only(libpath):
    """The region-check switch is a host-side setting (no CUDA call): off by
    default in a fresh process, read back as set."""
    import sys
    code = ("import ctypes, sys; lib = ctypes.CDLL(sys.argv[1]); "
            "print(lib.hdda_region_checks())")
    out = subprocess.run([sys.executable, "-c", code, libpath], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "0", out.stderr
    lib = ctypes.CDLL(libpath)
    before = lib.hdda_region_checks()
    try:
        assert lib.hdda_set_region_checks(1) == 0 and lib.hdda_region_checks() == 1
        assert lib.hdda_set_region_checks(0) == 0 and lib.hdda_region_checks() == 0
    finally:
        lib.hdda_set_region_checks(before)


def test_sampler_form_switch_is_host_only(libpath):
    """The sampler-form switch is a host-side setting: separate (0) by default
    in a fresh process, read back as set, and any other value is refused."""
    import sys
    code = ("import ctypes, sys; lib = ctypes.CDLL(sys.argv[1]); "
            "print(lib.hdda_sampler_form())")
    out = subprocess.run([sys.executable, "-c", code, libpath], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "0", out.stderr
    lib = ctypes.CDLL(libpath)
    before = lib.hdda_sampler_form()
    try:
        assert lib.hdda_set_sampler_form(1) == 0 and lib.hdda_sampler_form() == 1
        assert lib.hdda_set_sampler_form(0) == 0 and lib.hdda_sampler_form() == 0
        assert lib.hdda_set_sampler_form(2) == 1 and lib.hdda_sampler_form() == 0
        assert lib.hdda_set_sampler_form(-1) == 1 and lib.hdda_sampler_form() == 0
    finally:
        lib.hdda_set_sampler_form(before)


def test_argument_errors_are_status_codes_before_any_device_call(libpath):
    """Invalid arguments come back as HDDA_ERR_INVALID_ARG with a message,
    checked before the library touches a device (so this runs without one)."""
    lib = ctypes.CDLL(libpath)
    lib.hdda_last_error.restype = ctypes.c_char_p
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    invalid = 1
    null = vp(None)
    # stream-ordered sampler without a status word
    assert lib.hdda_traverse_async(null, null, i64(0), null, null, null, null, null, null,
                                   i64(0), null, null) == invalid
    assert b"dev_status" in lib.hdda_last_error()
    # render-only path and fused sampler + compositor without a grid
    assert lib.hdda_render(null, null, i64(0), null, null, null, 0, null, null, null) == invalid
    assert b"grid" in lib.hdda_last_error()
    assert lib.hdda_traverse_composite(null, null, i64(0), null, null, null, null, null, null,
                                       i64(0), null, 0, null, null, null) == invalid
    assert b"grid" in lib.hdda_last_error()
    # compositor with a negative ray count and with too many blobs
    assert lib.hdda_composite(null, null, i64(-1), null, null, null, null, 0, null, null) == invalid
    assert lib.hdda_composite(null, null, i64(1), null, null, null, null, 100000, null,
                              null) == invalid
    assert b"n_gauss" in lib.hdda_last_error()
