"""CPU checks of the library boundary: it builds, loads, and exports every declared symbol.

No compute call is made here (there is no GPU on the CPU test runner).
"""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "birkhoff.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", src)
    keep = [n for n in names if n.startswith(("bk_", "birkhoff_", "kkt_", "precond_", "krylov_",
                                              "newton_"))]
    return sorted(set(keep))


def test_header_declares_the_boundary_calls():
    names = _declared()
    for n in ["birkhoff_apply", "birkhoff_apply_T", "kkt_apply", "precond_apply", "krylov_solve",
              "newton_solve", "bk_plan_create", "bk_problem_create"]:
        assert n in names


def test_library_builds_and_exports_every_symbol():
    from paper_2509_01855_gb300 import build, _lib
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(_lib.EXPORTS) == _declared()
    L = _lib.lib()
    assert L.bk_version().decode().startswith("birkhoff-gb300")


def test_binding_struct_layouts_match_the_library():
    """The ctypes mirrors of the option and info structs have the compiled sizes (a field added
    on one side only would shift every field after it)."""
    from paper_2509_01855_gb300 import _lib
    L = _lib.lib()
    for which, cls in enumerate([_lib.KrylovOpts, _lib.KrylovInfo, _lib.NewtonOpts, _lib.NewtonInfo]):
        assert L.bk_abi_struct_size(which) == ctypes.sizeof(cls), cls.__name__
    assert L.bk_abi_struct_size(99) == 0


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2509_01855_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    import pytest
    with pytest.raises(ImportError):
        _lib.lib()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2509_01855_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
