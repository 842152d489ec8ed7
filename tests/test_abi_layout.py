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
