"""The ctypes structures of the binding have the layout of the C structs of
include/dgmg.h: a C program compiled against the header prints sizeof and
every field's offsetof, and each must equal the ctypes figure (a field added,
dropped or reordered on one side fails here, on the CPU)."""
import ctypes
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "dgmg_mesh": "Mesh", "dgmg_opts": "Opts", "dgmg_info_t": "Info", "dgmg_stats": "Stats",
    "dgmg_server_info_t": "ServerInfo", "dgmg_batch_info_t": "BatchInfo",
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    from paper_2510_00998_gb300 import dgmg
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dgmg.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in getattr(dgmg, pyname)._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    p = subprocess.run([cc, "-std=c11", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert p.returncode == 0, p.stderr         # a ctypes field the C struct lacks fails to compile
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_header(c_layout, cname):
    from paper_2510_00998_gb300 import dgmg
    py = getattr(dgmg, STRUCTS[cname])
    assert ctypes.sizeof(py) == c_layout[(cname, "sizeof")]
    for fname, _ in py._fields_:
        assert getattr(py, fname).offset == c_layout[(cname, fname)], fname


def _prototypes():
    import re
    src = open(os.path.join(ROOT, "include", "dgmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(dgmg_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        args = " ".join(m.group(2).split())
        protos[m.group(1)] = [] if args in ("", "void") else [a.strip() for a in args.split(",")]
    return protos


def _kind_c(arg):
    if "*" in arg:
        return "ptr"
    # size_t and uint64_t are one 64-bit unsigned kind (as are their ctypes
    # types on a 64-bit host)
    for t, k in (("size_t", "u64"), ("uint64_t", "u64"), ("int64_t", "i64"), ("double", "dbl"), ("int", "int")):
        if arg.startswith(t) or f" {t} " in f" {arg} ":
            return k
    raise AssertionError(arg)


def _kind_py(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
        return "ptr"
    assert ctypes.sizeof(ctypes.c_size_t) == 8
    return {ctypes.c_size_t: "u64", ctypes.c_uint64: "u64", ctypes.c_int64: "i64", ctypes.c_double: "dbl",
            ctypes.c_int: "int"}[t]


def test_binding_signatures_match_header():
    """Every prototype's argument count and kinds (pointer, int, double,
    64-bit integers) equal the binding's argtypes."""
    from paper_2510_00998_gb300 import dgmg
    protos = _prototypes()
    assert set(protos) == set(dgmg._SIGS), set(protos) ^ set(dgmg._SIGS)
    for name, args in protos.items():
        got = [_kind_py(t) for t in dgmg._SIGS[name][1]]
        want = [_kind_c(a) for a in args]
        assert got == want, (name, got, want)
