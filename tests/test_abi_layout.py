"""The Python bindings' descriptor structs against the C headers' layouts: a small C program
compiled against include/ibfsa.h (and oracle/ibfsa_oracle.h) prints sizeof and offsetof of every
field of ibfsa_grid_desc and ibfsa_plate_desc (and orc_desc), which must equal the ctypes
Structures' (a field added on one side only would shift everything after it)."""
import os
import shutil
import subprocess

import pytest

from paper_1905_00182_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_layout(struct, fields, header="ibfsa.h", incdir=None, outdir=None):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    outdir = outdir or B.BUILD
    os.makedirs(outdir, exist_ok=True)
    src = os.path.join(outdir, f"layout_{struct}.c")
    exe = os.path.join(outdir, f"layout_{struct}")
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{header}"',
             "int main(void) {", f'  printf("size %zu\\n", sizeof({struct}));']
    for f in fields:
        lines.append(f'  printf("{f} %zu\\n", offsetof({struct}, {f}));')
    lines += ["  return 0;", "}"]
    with open(src, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    subprocess.run([cc, "-I", incdir or os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (ln.split() for ln in out.splitlines())}


@pytest.mark.parametrize("which", ["grid", "plate"])
def test_descriptor_layout_matches_the_header(which):
    from paper_1905_00182_gb300 import ibfsa
    S, name = (ibfsa.GridDesc, "ibfsa_grid_desc") if which == "grid" else \
        (ibfsa.PlateDesc, "ibfsa_plate_desc")
    fields = [f for f, _ in S._fields_]
    c = _c_layout(name, fields)
    assert c["size"] == ctypes_sizeof(S)
    for f in fields:
        assert c[f] == getattr(S, f).offset, f


def test_oracle_descriptor_layout_matches_its_header():
    from oracle import oracle as O
    fields = [f for f, _ in O.OrcDesc._fields_]
    c = _c_layout("orc_desc", fields, header="ibfsa_oracle.h",
                  incdir=os.path.join(ROOT, "oracle"),
                  outdir=os.path.join(ROOT, "oracle", "_build"))
    assert c["size"] == ctypes_sizeof(O.OrcDesc)
    for f in fields:
        assert c[f] == getattr(O.OrcDesc, f).offset, f


def ctypes_sizeof(S):
    import ctypes
    return ctypes.sizeof(S)
