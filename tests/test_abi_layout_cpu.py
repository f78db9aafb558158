"""The Python binding's ctypes mirrors of the C-ABI structs (CPU): every field
at the offset and with the size the C compiler gives it for include/frg.h, so
that parameters and statistics cross the boundary unchanged."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_1510_07799_gb300 import frg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {
    "frg_params": frg._Params,
    "frg_flow_stats": frg._Stats,
    "frg_tune": frg._Tune,
    "frg_obs": frg._Obs,
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "frg.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s %s %%zu %%zu\\n", offsetof(%s, %s), sizeof(((%s *)0)->%s));'
                         % (name, field, name, field, name, field))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    size, fields = {}, {}
    for line in out:
        parts = line.split()
        if len(parts) == 3 and parts[1] == "size":
            size[parts[0]] = int(parts[2])
        elif len(parts) == 4:
            fields[(parts[0], parts[1])] = (int(parts[2]), int(parts[3]))
    return size, fields


def test_ctypes_structs_match_the_header(tmp_path):
    size, fields = _c_layout(tmp_path)
    for name, cls in STRUCTS.items():
        assert C.sizeof(cls) == size[name], name
        for field, ctype in cls._fields_:
            off, sz = fields[(name, field)]
            assert getattr(cls, field).offset == off, (name, field)
            assert C.sizeof(ctype) == sz, (name, field)
