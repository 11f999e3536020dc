"""The ctypes mirrors of the ABI's structs and signatures (native.py) against the header
itself: a small C program, compiled with gcc against include/ges.h, prints
the size of every struct and the offset of every field the binding names.
A field the header does not have fails the compile; a type, order or padding
difference shows up as a different offset, field size or struct size.  The
function table is checked against the header's declarations: the same names,
argument counts, and pointer / integer / float class of every argument and
return value.  CPU only."""
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


def _header_decls():
    """name -> (return type, [parameter declarations]) of every GES_API
    function in include/ges.h, comments removed."""
    import re
    text = open(os.path.join(ROOT, "include", "ges.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    out = {}
    for m in re.finditer(r"GES_API\s+([\w\s\*]+?)\s*\b(ges_\w+)\s*\(([^)]*)\)\s*;", text):
        ret, name, params = m.group(1).strip(), m.group(2), m.group(3).strip()
        plist = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
        out[name] = (ret, plist)
    return out


def _kind_c(decl):
    """Coarse class of a C parameter or return type: pointer or scalar kind."""
    if "*" in decl:
        return "ptr"
    for t, k in (("int64_t", "i64"), ("int32_t", "i32"), ("double", "f64"), ("float", "f32")):
        if t in decl.split():
            return k
    if decl.split()[0].startswith("ges_"):       # enums (ges_status, ges_dtype, ...)
        return "i32"
    raise AssertionError(f"unclassified C type: {decl}")


def _kind_ctypes(t):
    if t in (C.c_void_p, C.c_char_p) or (isinstance(t, type) and issubclass(t, C._Pointer)):
        return "ptr"
    return {C.c_int32: "i32", C.c_int: "i32", C.c_int64: "i64", C.c_float: "f32", C.c_double: "f64"}[t]


def test_binding_signatures_match_the_header():
    decls = _header_decls()
    assert set(decls) == set(N._SIGS), (set(decls) ^ set(N._SIGS))
    for name, (ret, params) in decls.items():
        cret, cargs = N._SIGS[name]
        assert _kind_c(ret) == _kind_ctypes(cret), (name, ret, cret)
        assert len(params) == len(cargs), (name, params, cargs)
        for p, a in zip(params, cargs):
            assert _kind_c(p) == _kind_ctypes(a), (name, p, a)
