"""The binding's ctypes signatures against the C prototypes of include/tr.h.

ctypes trusts the argument list it is given: a missing parameter, an int
where the C side takes a double or a 64-bit integer, or a value where it
takes a pointer would pass garbage through the C ABI without any error.
This test parses every prototype of the header and checks, for each entry
point the binding declares, the return type and each parameter's kind
(pointer, 32-bit integer or enum, 64-bit integer, float, double)."""

import ctypes
import os
import re

from paper_2506_09594_gb300 import tr

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "tr.h")
INT32 = {"int", "unsigned", "int32_t", "uint32_t", "tr_status", "tr_dtype", "tr_penalty",
         "tr_prec", "tr_noise", "tr_lr_engine", "tr_engine"}
INT64 = {"int64_t", "uint64_t", "size_t", "long long", "unsigned long long"}


def _prototypes():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"^\s*#[^\n]*", "", src, flags=re.M)      # preprocessor lines
    enums = set(re.findall(r"typedef\s+enum\s*\w*\s*\{[^}]*\}\s*(\w+)\s*;", src))
    protos = {}
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(tr_\w+)\s*\(([^;{()]*)\)\s*;", src):
        ret, name, args = m.group(1).strip(), m.group(2), m.group(3).strip()
        if "typedef" in ret:
            continue
        params = [] if args in ("", "void") else [a.strip() for a in args.split(",")]
        protos[name] = (ret, params)
    return protos, enums


def _c_kind(decl, enums, is_return=False):
    if "*" in decl or "[" in decl:    # an array parameter is a pointer
        return "ptr"
    words = decl.replace("const ", "").split()
    base = " ".join(words if is_return else words[:-1])
    if base == "void":
        return "void"
    if base == "double":
        return "f64"
    if base == "float":
        return "f32"
    if base in INT64:
        return "i64"
    if base in INT32 or base in enums:
        return "i32"
    raise AssertionError("unclassified C type %r in %r" % (base, decl))


def _ct_kind(t):
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "ptr"
    if t is ctypes.c_double:
        return "f64"
    if t is ctypes.c_float:
        return "f32"
    if issubclass(t, ctypes._SimpleCData) and t._type_ in "bBhHiIlLqQnN":
        return {4: "i32", 8: "i64"}[ctypes.sizeof(t)]
    raise AssertionError("unclassified ctypes type %r" % (t,))


def test_every_binding_signature_matches_its_prototype():
    protos, enums = _prototypes()
    assert len(protos) >= 50
    missing = sorted(set(tr._SIGS) - set(protos))
    assert not missing, missing
    for name, (restype, argtypes) in tr._SIGS.items():
        ret, params = protos[name]
        assert _ct_kind(restype) == _c_kind(ret, enums, is_return=True), name
        assert len(argtypes) == len(params), (name, len(argtypes), len(params))
        for i, (a, p) in enumerate(zip(argtypes, params)):
            assert _ct_kind(a) == _c_kind(p, enums), (name, i, p, a)


def test_the_binding_declares_every_prototype():
    protos, _ = _prototypes()
    assert sorted(set(protos) - set(tr._SIGS)) == []
