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


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    # no CPU fallback: without the compiled library every entry point raises
    import pytest
    from paper_2510_04795_gb300 import _native
    import paper_2510_04795_gb300 as oz
    monkeypatch.setattr(_native, "_lib", None)
    monkeypatch.setattr(_native, "_LIBPATH", str(tmp_path / "libozdmrg.so"))
    with pytest.raises(_native.OzError):
        _native.load()
    with pytest.raises(_native.OzError):
        oz.Context(0)


def test_python_binding_only_marshals():
    # the package imports no oracle module and no numerical fallback
    import ast
    pkg = os.path.join(ROOT, "paper_2510_04795_gb300")
    for f in ("__init__.py", "_native.py", "selector.py"):
        tree = ast.parse(open(os.path.join(pkg, f)).read())
        mods = set()
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                mods.update(a.name.split(".")[0] for a in node.names)
            elif isinstance(node, ast.ImportFrom) and node.module:
                mods.add(node.module.split(".")[0])
        assert "oracle" not in mods, f
