"""The C ABI: the library loads without a GPU and exports every function include/ozdmrg.h
declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ozdmrg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s*([A-Za-z_]\w*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ozaki_gemm", "heff_apply", "davidson_step", "dmrg_sweep", "ozaki_gemm_noalloc"):
        assert required in names
    assert len(names) >= 40


def test_library_exports_every_declared_symbol():
    from paper_2510_04795_gb300 import _native
    lib = ctypes.CDLL(_native.lib_path())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
