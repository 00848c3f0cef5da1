"""The ctypes binding agrees with include/sdx.h: every prototype's argument and return types,
and the memory layout of the two structs the binding mirrors (no GPU needed: nothing here
launches a kernel).  A mismatch here would pass wrong values through the C ABI silently."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from tests._lib import ensure_built

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sdx.h")

OPAQUE = {"sdx_hier_t", "sdx_batch_t", "sdx_net_t", "sdx_p0_t"}
SCALARS = {"int": ctypes.c_int, "double": ctypes.c_double, "float": ctypes.c_float,
           "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64}


def _prototypes():
    """{name: (return type, [parameter types])} from the header, comments removed."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"(int64_t|int|const\s+char\s*\*)\s+(sdx_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
        ret, name, params = m.group(1), m.group(2), m.group(3).strip()
        types = []
        if params and params != "void":
            for p in params.split(","):
                p = " ".join(p.replace("*", " * ").split())
                words = p.split(" ")
                if words[-1] not in ("*",) and re.fullmatch(r"[a-z_][a-z0-9_]*", words[-1]) and len(words) > 1:
                    words = words[:-1]  # drop the parameter name
                types.append(" ".join(w for w in words if w != "const"))
        out[name] = (" ".join(ret.replace("*", " * ").split()), types)
    return out


def _matches(ctype, ct):
    """Whether the ctypes type ct passes a C parameter of (const-stripped) type ctype."""
    if ctype in OPAQUE:
        return ct is ctypes.c_void_p
    if ctype.endswith("*"):
        pointee = ctype[:-1].strip()
        if ct is ctypes.c_void_p:
            return pointee not in OPAQUE  # data pointers may go as void*; handles have a type
        target = getattr(ct, "_type_", None)
        if target is None or not issubclass(ct, ctypes._Pointer):
            return False
        if pointee in OPAQUE:
            return target is ctypes.c_void_p
        if pointee in SCALARS:
            return target is SCALARS[pointee]
        from paper_1604_07994_gb300 import sdx
        return target is getattr(sdx, pointee, None)
    return ct is SCALARS.get(ctype)


def test_every_prototype_is_parsed():
    from paper_1604_07994_gb300 import sdx
    protos = _prototypes()
    assert set(protos) == set(sdx.EXPORTED)


def test_binding_argument_and_return_types_match_the_header():
    ensure_built()
    from paper_1604_07994_gb300 import sdx
    lib = sdx.load()
    rets = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "const char *": ctypes.c_char_p}
    for name, (ret, params) in _prototypes().items():
        fn = getattr(lib, name)
        assert fn.restype is rets[ret], (name, ret, fn.restype)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == len(params), (name, params, fn.argtypes)
        for k, (ctype, ct) in enumerate(zip(params, fn.argtypes)):
            assert _matches(ctype, ct), (name, k, ctype, ct)


def test_a_planted_mismatch_is_caught():
    # the checker itself: a double passed where the header has an int, a handle passed as a
    # data pointer type, an int* passed as int64* all fail
    assert not _matches("int", ctypes.c_double)
    assert not _matches("sdx_hier_t *", ctypes.POINTER(ctypes.c_int))
    assert not _matches("int *", ctypes.POINTER(ctypes.c_int64))
    assert _matches("double *", ctypes.c_void_p)
    assert _matches("sdx_hier_t *", ctypes.POINTER(ctypes.c_void_p))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a C compiler")
def test_struct_layouts_match_the_header(tmp_path):
    from paper_1604_07994_gb300 import sdx
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "sdx.h"', "int main(void) {"]
    for st in (sdx.sdx_desc, sdx.sdx_stats):
        cname = st.__name__
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in st._fields_:
            lines.append(f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for st in (sdx.sdx_desc, sdx.sdx_stats):
        cname = st.__name__
        assert got[(cname, "size")] == ctypes.sizeof(st), cname
        for f, _ in st._fields_:
            assert got[(cname, f)] == getattr(st, f).offset, (cname, f)
