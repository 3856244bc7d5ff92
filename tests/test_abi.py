"""The C-ABI library loads, exports every symbol include/smg.h declares, and rejects invalid
arguments on the host before launching anything (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def smg():
    from paper_1212_6680_gb300 import build

    build.build()
    from paper_1212_6680_gb300 import smg as m

    return m


def declared_functions():
    text = open(os.path.join(ROOT, "include", "smg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)))


def test_header_declarations_are_exported(smg):
    names = declared_functions()
    assert "krylov_solve" in names and "smg_setup" in names and "lobpcg_solve" in names
    for n in names:
        assert hasattr(smg.lib(), n), n
    assert set(names) == set(smg.EXPORTS)


def test_binding_constants_match_the_header(smg):
    """The Python binding passes status codes, variants, precisions and option ids as plain
    integers: each must be the value include/smg.h gives it."""
    text = open(os.path.join(ROOT, "include", "smg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"\b(SMG_\w+)\s*=\s*(-?\d+)", text)}
    assert "SMG_OPT_WIDE_MIN_ROWS" in consts and "SMG_ERR_HOST" in consts
    for name, value in consts.items():
        assert getattr(smg, name) == value, name


def test_library_is_built_for_sm_103a():
    from paper_1212_6680_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def call_setup(smg, *args):
    h = ctypes.c_void_p(123)
    rc = smg.lib().smg_setup(*args, ctypes.byref(h))
    return rc, h.value


@pytest.mark.parametrize("args", [(0, 4, 4, 1, 1), (4, 0, 4, 1, 1), (4, 4, 0, 1, 1), (4, 4, 4, 0, 1),
                                  (4, 4, 4, 1, -1), (2049, 4, 4, 1, 1), (4, 513, 4, 1, 1), (4, 4, 5000, 1, 1)])
def test_setup_rejects_bad_arguments(smg, args):
    rc, h = call_setup(smg, *args)
    assert rc == smg.SMG_ERR_ARG
    assert not h
    assert smg.smg_last_error()


def test_null_handle_and_null_pointers_are_rejected(smg):
    L = smg.lib()
    it = ctypes.c_int(7)
    rr = ctypes.c_double(1.0)
    assert L.krylov_solve(None, 0, None, None, 1e-8, 10, ctypes.byref(it), ctypes.byref(rr), None) == smg.SMG_ERR_ARG
    assert L.smg_apply(None, None, None, None) == smg.SMG_ERR_ARG
    assert L.smg_set_precision(None, 1) == smg.SMG_ERR_ARG
    assert L.lobpcg_solve(None, 1, None, None, 1e-8, 10, None, None) == smg.SMG_ERR_ARG
    assert L.smg_destroy(None) == smg.SMG_OK
    with pytest.raises(smg.SMGError):
        smg.smg_apply(0, 0, 0, stream=0)
