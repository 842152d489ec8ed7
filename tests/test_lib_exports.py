"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/dgmg.h declares (no compute calls: this runs on CPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dgmg_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["dgmg_create", "dgmg_destroy", "dgmg_apply", "dgmg_smooth", "dgmg_vcycle", "dgmg_solve",
                 "dgmg_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_00998_gb300 import dgmg
    lib = ctypes.CDLL(dgmg.LIB_PATH)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    assert b"sm_103a" in dgmg.load().dgmg_version()
    # every declared function has a binding signature
    assert not (_declared() - set(dgmg._SIGS)), _declared() - set(dgmg._SIGS)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2510_00998_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", src).replace("the oracle", ""), f
