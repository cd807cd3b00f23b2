"""The Python binding mirrors include/panache.h exactly (no GPU needed).

The ctypes structures must have the C structures' sizes and field offsets,
and the binding's constants the header's values: a mismatch would pass
wrong arguments through every call.  The layouts are read from a small C
program compiled against the header with the host compiler.
"""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2607_17481_b300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "panache.h")

PAIRS = [(native.Config, "panache_config"), (native.Motif, "panache_motif"), (native.Request, "panache_request"),
         (native.Stats, "panache_stats"), (native.ServerStats, "panache_server_stats")]


def _c_field(name):
    return name[:-1] if name.endswith("_") and not name.startswith("_") else name   # lambda_ -> lambda


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("layout")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "panache.h"', 'int main(void) {']
    for cls, cname in PAIRS:
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {_c_field(f[0])}));')
    lines += ['return 0;', '}']
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    out = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        cname, field, value = line.split()
        out[(cname, field)] = int(value)
    return out


@pytest.mark.parametrize("cls,cname", PAIRS, ids=[p[1] for p in PAIRS])
def test_struct_layout_matches_header(c_layout, cls, cname):
    assert ctypes.sizeof(cls) == c_layout[(cname, "sizeof")], cname
    for f in cls._fields_:
        assert getattr(cls, f[0]).offset == c_layout[(cname, f[0])], (cname, f[0])


def test_constants_match_header():
    hdr = open(HEADER).read()
    defs = dict(re.findall(r"^#define PANACHE_([A-Z0-9_]+)\s+\(?(-?(?:0x[0-9a-fA-F]+|\d+))\)?", hdr, flags=re.M))
    assert "FLAG_HALF_FEATURES" in defs
    checked = 0
    for name, value in defs.items():
        if hasattr(native, name):
            assert getattr(native, name) == int(value, 0), name
            checked += 1
        assert not name.startswith("FLAG_") or hasattr(native, name), f"flag {name} missing from the binding"
    assert checked >= 15
