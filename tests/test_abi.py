"""The C ABI library loads, exports every symbol include/*.h declares, and
rejects bad arguments on the host before touching a GPU (no compute calls)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(deepinv_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def L():
    from paper_1701_03891_gb300 import build, deepinv
    build.build()
    return deepinv.lib()


def test_header_declares_the_boundary():
    d = _declared()
    for n in ("deepinv_measure", "deepinv_forward", "deepinv_backward", "deepinv_net_create"):
        assert n in d


def test_every_declared_symbol_is_exported(L):
    from paper_1701_03891_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (deepinv_\w+)", out))
    missing = _declared() - exported
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1701_03891_gb300 import deepinv
    assert _declared() <= set(deepinv.SIGNATURES)


def test_binding_constants_match_header():
    from paper_1701_03891_gb300 import deepinv
    with open(os.path.join(ROOT, "include", "deepinv.h")) as f:
        h = f.read()
    assert int(re.search(r"#define DEEPINV_NSTAGES (\d+)", h).group(1)) == deepinv.NSTAGES == len(deepinv.STAGES)
    assert int(re.search(r"#define DEEPINV_MAX_HIDDEN (\d+)", h).group(1)) == deepinv.MAX_HIDDEN


def test_version(L):
    assert L.deepinv_version() == 201


def test_launch_count_starts_at_zero_without_launches(L):
    # host-side checks that reject a call launch nothing, so the count does not move
    before = L.deepinv_launch_count()
    assert L.deepinv_measure(None, 4, 8, None, 2, None, 0, None) != 0
    assert L.deepinv_launch_count() == before


def test_null_pointers_rejected_on_host(L):
    from paper_1701_03891_gb300 import deepinv
    rc = L.deepinv_measure(None, 4, 8, None, 2, None, 0, None)
    assert rc == deepinv.EINVAL
    assert b"null" in L.deepinv_last_error()
    assert L.deepinv_forward(None, None, 1, None, None, None) == deepinv.EINVAL
    assert L.deepinv_net_reserve(None, 4, None) == deepinv.EINVAL


def test_bad_descriptions_rejected_on_host(L):
    from paper_1701_03891_gb300 import deepinv
    out = ctypes.c_void_p()
    bad = [
        deepinv.NetDesc(0, 8, 4, 64, 32, 1, 11, 0, 0, 0),      # empty image
        deepinv.NetDesc(8, 8, 65, 64, 32, 1, 11, 0, 0, 0),     # M > N
        deepinv.NetDesc(8, 8, 4, 64, 32, 1, 10, 0, 0, 0),      # even kernel
        deepinv.NetDesc(8, 8, 4, 64, 32, 2, 11, 0, 0, 0),      # l3 != 1
        deepinv.NetDesc(8, 8, 4, 64, 32, 1, 11, 0, 0, 7),      # unknown precision
        deepinv.NetDesc(8, 8, 4, 64, 32, 1, 11, 0, 0, 0, -1),  # negative hidden layer count
        deepinv.NetDesc(8, 8, 4, 64, 32, 1, 11, 0, 0, 0, deepinv.MAX_HIDDEN + 1),   # too many hidden layers
    ]
    for d in bad:
        rc = L.deepinv_net_create(ctypes.byref(d), ctypes.c_void_p(16), None, None, None, ctypes.byref(out))
        assert rc == deepinv.EINVAL, (d.n1, d.M, d.k, d.hidden, rc)
    d = deepinv.NetDesc(8, 8, 4, 16, 32, 1, 11, 0, 0, deepinv.BF16)  # bf16 needs 64/32/1
    rc = L.deepinv_net_create(ctypes.byref(d), ctypes.c_void_p(16), None, None, None, ctypes.byref(out))
    assert rc == deepinv.EUNSUPPORTED


def test_saved_bytes_null_net(L):
    assert L.deepinv_saved_bytes(None, 4) == 0


def _declarations():
    """name -> (return type, [parameter declarations]) of every deepinv_* function in include/*.h."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^([A-Za-z_][\w\s\*]*?)\s*\b(deepinv_\w+)\s*\(([^;{]*?)\)\s*;", src, flags=re.M | re.S):
            ret, name, params = " ".join(m.group(1).split()), m.group(2), " ".join(m.group(3).split())
            out[name] = (ret, [] if params in ("", "void") else [p.strip() for p in params.split(",")])
    return out


def test_binding_signatures_match_header():
    """Each ctypes prototype has the header's return type, parameter count and,
    per parameter, the same scalar type or a pointer where the header has one
    (a mismatch would pass arguments in the wrong registers or widths)."""
    from paper_1701_03891_gb300 import deepinv
    ret_types = {"int": ctypes.c_int, "size_t": ctypes.c_size_t, "const char*": ctypes.c_char_p,
                 "const char *": ctypes.c_char_p, "unsigned long long": ctypes.c_ulonglong}
    scalars = {"int": ctypes.c_int, "float": ctypes.c_float, "double": ctypes.c_double,
               "size_t": ctypes.c_size_t, "uint64_t": ctypes.c_uint64}
    decl = _declarations()
    assert decl.keys() == _declared()
    for name, (ret, params) in decl.items():
        res, args = deepinv.SIGNATURES[name]
        assert len(args) == len(params), (name, len(args), len(params))
        assert res is ret_types[ret], (name, ret)
        for p, a in zip(params, args):
            if "*" in p or "[" in p:
                assert a in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(a, ctypes._Pointer), (name, p, a)
            else:
                ctype = " ".join(p.replace("const ", "").split()[:-1])
                assert a is scalars[ctype], (name, p, a)


def test_struct_layouts_match_header(tmp_path):
    """sizeof and every field's offset of the structs shared with C, compiled
    from include/deepinv.h by gcc, equal the ctypes mirrors'."""
    from paper_1701_03891_gb300 import deepinv
    structs = {"deepinv_net_desc": deepinv.NetDesc, "deepinv_request": deepinv.Request,
               "deepinv_result": deepinv.Result, "deepinv_serve_stats": deepinv.ServeStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "deepinv.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {k: int(v) for k, v in (line.rsplit(" ", 1) for line in out.splitlines())}
    for cname, cls in structs.items():
        assert got[cname] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[cname + "." + f] == getattr(cls, f).offset, (cname, f)


def test_measure_sizes_beyond_2_30_rejected_on_host(L):
    from paper_1701_03891_gb300 import deepinv
    p = ctypes.c_void_p(16)
    for M, N, B in ((1 << 30, (1 << 30) + 1, 1), ((1 << 30) + 1, 1 << 30, 1), (4, 8, (1 << 30) + 1),
                    (2147483647, 2147483647, 1)):
        assert L.deepinv_measure(p, M, N, p, B, p, 0, None) == deepinv.EINVAL, (M, N, B)
        assert L.deepinv_measure_noalloc(p, M, N, p, B, p, None) == deepinv.EINVAL, (M, N, B)
        assert b"bad sizes" in L.deepinv_last_error()
