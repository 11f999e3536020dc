"""The ctypes mirrors of the ABI's structs (native.py) against the header
itself: a small C program, compiled with gcc against include/ges.h, prints
the size of every struct and the offset of every field the binding names.
A field the header does not have fails the compile; a type, order or padding
difference shows up as a different offset, field size or struct size.  CPU only."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2504_17545_gb300 import native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [N.ges_scene_desc, N.ges_camera, N.ges_render_opts, N.ges_grads, N.ges_tgrads, N.ges_stats,
           N.ges_batch_info, N.ges_profile]


def _c_layout(tmp_path):
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ges.h"', "int main(void) {"]
    for S in STRUCTS:
        n = S.__name__
        lines.append(f'  printf("{n} sizeof %zu\\n", sizeof({n}));')
        for f, _ in S._fields_:
            lines.append(f'  printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
            lines.append(f'  printf("{n} {f}.size %zu\\n", sizeof((({n} *)0)->{f}));')
    lines += ["  return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {(a, b): int(c) for a, b, c in (l.split() for l in out.strip().splitlines())}


def test_ctypes_structs_match_the_header(tmp_path):
    c = _c_layout(tmp_path)
    for S in STRUCTS:
        n = S.__name__
        assert C.sizeof(S) == c[(n, "sizeof")], (n, C.sizeof(S), c[(n, "sizeof")])
        for f, _ in S._fields_:
            assert getattr(S, f).offset == c[(n, f)], (n, f, getattr(S, f).offset, c[(n, f)])
            assert getattr(S, f).size == c[(n, f + ".size")], (n, f, getattr(S, f).size, c[(n, f + ".size")])
