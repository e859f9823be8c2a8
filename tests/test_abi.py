"""The C-ABI library builds, loads without a GPU, and exports every entry point the header declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"SFGMRES_API\s+[\w\s\*]+?\b(sfgmres_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2506_18408_gb300 import build as b

    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("sfgmres_create", "sfgmres_solve", "sfgmres_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_binding_mirrors_header():
    from paper_2506_18408_gb300 import sfgmres as py

    assert set(py.EXPORTED) == _declared()
    for name in py.EXPORTED:
        assert callable(getattr(py, name))


def test_version_and_error_calls_need_no_gpu(lib):
    lib.sfgmres_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.sfgmres_version()
    lib.sfgmres_last_error.restype = ctypes.c_char_p
    lib.sfgmres_last_error.argtypes = [ctypes.c_void_p]
    assert isinstance(lib.sfgmres_last_error(None), bytes)
    lib.sfgmres_destroy.argtypes = [ctypes.c_void_p]
    assert lib.sfgmres_destroy(None) == 0


def test_create_rejects_bad_arguments_without_touching_the_device(lib):
    lib.sfgmres_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                   ctypes.c_int32, ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.sfgmres_create(ctypes.byref(h), 0, 0, None, None, None, 1, 1, None) == -1
    assert lib.sfgmres_create(None, 4, 4, None, None, None, 1, 1, None) == -1


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2506_18408_gb300")
    for dp, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dp, fn)).read()
                assert "oracle" not in re.findall(r"(?:import|from)\s+(\w+)", text), fn


def test_binding_constants_match_the_header():
    """Every SFGMRES_OPT_* key and status code the header defines has the same value in the binding, and every
    option key has a name in Solver.set/get."""
    from paper_2506_18408_gb300 import sfgmres as py

    text = open(os.path.join(ROOT, "include", "sfgmres.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+SFGMRES_(\w+)\s+\(?(-?\d+)\)?", text)}
    opts = {k[4:]: v for k, v in defs.items() if k.startswith("OPT_")}
    assert len(opts) >= 14
    for name, value in opts.items():
        assert getattr(py, "OPT_" + name) == value, name
    assert sorted(py.Solver._KEYS.values()) == sorted(opts.values())
    for name in ("OK", "NOT_CONVERGED", "BREAKDOWN", "ERR_INVALID_ARG", "ERR_CUDA", "ERR_OOM", "ERR_NAN"):
        assert getattr(py, name) == defs[name], name
