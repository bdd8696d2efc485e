"""The C ABI library builds, loads and exports every symbol include/ahf.h
declares; the Python binding's structs match the C layouts (no GPU needed)."""
import ctypes
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(ahf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_0904_3662_gb300 import build_lib
    lib_path = build_lib.build()
    lib = ctypes.CDLL(lib_path)
    declared = _declared()
    assert "ahf_unbind_batch" in declared and "ahf_profile_batch" in declared
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    lib.ahf_version.restype = ctypes.c_int
    assert lib.ahf_version() >= 100


def test_binding_lists_every_symbol():
    from paper_0904_3662_gb300 import ahf
    assert sorted(ahf.EXPORTS) == _declared()


def test_struct_layouts():
    from paper_0904_3662_gb300 import ahf
    assert ctypes.sizeof(ahf._Params) == 6 * 8 + 4 * 4
    assert ctypes.sizeof(ahf._Particles) == 7 * 8 + 8 + 8 + 2 * 4 + 8
    assert ahf.HALO_DTYPE.itemsize == 48
    assert ahf.RESULT_DTYPE.itemsize == 88
    assert ahf.RESULT_DTYPE.fields["m_vir"][1] == 48


def test_create_without_gpu_reports_error():
    import torch
    if torch.cuda.is_available():
        return
    from paper_0904_3662_gb300 import ahf
    try:
        ahf.Context(0)
    except ahf.AHFError as e:
        assert e.code == ahf.ERR_INVALID
    else:
        raise AssertionError("context creation without a GPU must fail")


def test_serve_create_checks_arguments_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        return
    from paper_0904_3662_gb300 import ahf
    prm = ahf.Params()
    # a cap below one full-size request is refused before any device call
    try:
        ahf.Serve(prm, hbm_cap_bytes=1 << 20)
    except ahf.AHFError as e:
        assert e.code == ahf.ERR_INVALID and "slots" in str(e)
    else:
        raise AssertionError("a tiny cap must be refused")
    bad = ahf.Params(max_iter=0)
    try:
        ahf.Serve(bad)
    except ahf.AHFError as e:
        assert e.code == ahf.ERR_INVALID and "max_iter" in str(e)
    else:
        raise AssertionError("max_iter 0 must be refused")
    try:
        ahf.Serve(prm)
    except ahf.AHFError as e:
        assert e.code == ahf.ERR_INVALID
    else:
        raise AssertionError("serving without a GPU must fail")
