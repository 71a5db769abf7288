"""The Python binding and the C header agree on the ABI: every struct the
binding declares with ctypes has the size, field offsets and field sizes
the C compiler gives the header's struct, every GS_ constant the binding
defines has the header's value, and every prototype's parameters and return
have the ABI classes of the binding's argtypes and restype.  A small C
program built with gcc against include/graphstep.h prints the header's
side; no GPU and no library call is involved."""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


@pytest.fixture(scope="module")
def g():
    import __graft_entry__

    __graft_entry__._builder().build()
    import paper_2501_09398_gb300

    return paper_2501_09398_gb300


def _structs(g):
    return {name: getattr(g, name) for name in dir(g)
            if name.startswith("gs_") and isinstance(getattr(g, name), type)
            and issubclass(getattr(g, name), ctypes.Structure)}


def _constants(g):
    return {name: getattr(g, name) for name in dir(g)
            if name.startswith("GS_") and isinstance(getattr(g, name), int) and not isinstance(getattr(g, name), bool)}


@pytest.fixture(scope="module")
def header_side(g, tmp_path_factory):
    structs, consts = _structs(g), _constants(g)
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "graphstep.h"', "int main(void) {"]
    for name, cls in sorted(structs.items()):
        lines.append(f'    printf("size {name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'    printf("off {name}.{f} %zu\\n", offsetof({name}, {f}));')
            lines.append(f'    printf("fsize {name}.{f} %zu\\n", sizeof((({name} *)0)->{f}));')
    for name in sorted(consts):
        lines.append(f'    printf("const {name} %lld\\n", (long long)({name}));')
    lines += ["    return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", HEADER_DIR, str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        kind, key, val = line.split()
        table[(kind, key)] = int(val)
    return structs, consts, table


def test_struct_sizes_and_offsets_match_the_header(header_side):
    structs, _, table = header_side
    assert len(structs) >= 10
    for name, cls in structs.items():
        assert ctypes.sizeof(cls) == table[("size", name)], name
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == table[("off", f"{name}.{f}")], (name, f)
            assert getattr(cls, f).size == table[("fsize", f"{name}.{f}")], (name, f)


def test_constants_match_the_header(header_side):
    _, consts, table = header_side
    assert len(consts) >= 40
    for name, v in consts.items():
        assert v == table[("const", name)], name


def _c_class(decl: str):
    """ABI class of a C parameter or return type: 'ptr', 'i32' (int, int32_t
    and the gs_ enums), 'i64' (int64_t, uint64_t), 'f32', 'f64', or None
    for void."""
    if "*" in decl:
        return "ptr"
    words = [w for w in decl.replace("const", " ").split()]
    t = words[0] if words else "void"
    if t == "void":
        return None
    if t in ("int", "int32_t") or (t.startswith("gs_") and t not in ("gs_ctx", "gs_multi", "gs_mlp")):
        return "i32"
    if t in ("int64_t", "uint64_t"):
        return "i64"
    return {"float": "f32", "double": "f64"}[t]


def _py_class(t):
    if t is None:
        return None
    if t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer)):
        return "ptr"
    if t is ctypes.c_float:
        return "f32"
    if t is ctypes.c_double:
        return "f64"
    return {4: "i32", 8: "i64"}[ctypes.sizeof(t)]


def test_function_signatures_match_the_header(g):
    # every prototype the header declares: the binding's argtypes have the
    # same number of parameters and the same ABI class for each, and the
    # restype the class of the return type (an int32 passed for an int64_t
    # would leave the register's upper half undefined)
    import re

    with open(os.path.join(HEADER_DIR, "graphstep.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = re.sub(r"#[^\n]*", " ", src)
    flat = " ".join(src.split())
    protos = re.findall(r"([A-Za-z_][\w\s\*]*?)\b(gs_\w+)\s*\(([^()]*)\)\s*;", flat)
    assert len(protos) >= 60
    for ret, name, params in protos:
        fn = getattr(g._lib, name)
        assert fn.argtypes is not None, name
        cparams = [] if params.strip() == "void" else [p.strip() for p in params.split(",")]
        assert len(fn.argtypes) == len(cparams), name
        for i, (p, t) in enumerate(zip(cparams, fn.argtypes)):
            assert _py_class(t) == _c_class(p), (name, i, p, t)
        assert _py_class(fn.restype) == _c_class(ret), (name, ret, fn.restype)
