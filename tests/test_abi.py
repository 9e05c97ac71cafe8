"""The C-ABI library loads and exports every entry point include/hss.h declares
(no GPU needed: loading the library performs no CUDA call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(hss_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hss_create", "hss_factorize", "hss_solve", "hss_logdet", "hss_matvec",
                 "hss_destroy", "hss_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2311_00921_gb300 import hss
    if not os.path.exists(hss.LIB_PATH):
        pytest.skip("library not built (run __graft_entry__.build())")
    lib = ctypes.CDLL(hss.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    # the binding declares a signature for every entry point of the header
    assert set(declared_functions()) <= set(hss.SIGNATURES)
    lib.hss_strerror.restype = ctypes.c_char_p
    assert lib.hss_strerror(-3).startswith(b"matrix not positive definite")


def test_create_rejects_bad_shapes_without_touching_the_device():
    from paper_2311_00921_gb300 import hss
    if not os.path.exists(hss.LIB_PATH):
        pytest.skip("library not built")
    lib = hss.load()
    out = ctypes.c_void_p()
    bad = hss.Shape(1000, 256, 32, 2)          # n != leaf * 2^levels
    buf = (ctypes.c_double * 4)()
    assert lib.hss_create(ctypes.byref(bad), buf, buf, buf, buf, 0, ctypes.byref(out)) == -1
    bad = hss.Shape(512, 256, 300, 1)          # rank > leaf
    assert lib.hss_create(ctypes.byref(bad), buf, buf, buf, buf, 0, ctypes.byref(out)) == -1
    assert lib.hss_create(None, buf, buf, buf, buf, 0, ctypes.byref(out)) == -1


def _c_layout(struct, fields):
    """sizeof and offsetof of a header struct, from a C program compiled here."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    body = "".join(f'  printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    src = (f'#include <stdio.h>\n#include "hss.h"\nint main(void) {{\n'
           f'  printf("%zu\\n", sizeof({struct}));\n{body}  return 0;\n}}\n')
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return [int(v) for v in out]


@pytest.mark.parametrize("struct,cls", [("hss_shape", "Shape"), ("hss_options", "Options"),
                                        ("hss_tuning", "Tuning")])
def test_binding_structs_match_the_header(struct, cls):
    """Every struct the binding passes by pointer has the header's size and field
    offsets (a mismatch would shift every later field silently)."""
    from paper_2311_00921_gb300 import hss
    py = getattr(hss, cls)
    fields = [f[0] for f in py._fields_]
    c = _c_layout(struct, fields)
    assert c[0] == ctypes.sizeof(py), (struct, c[0], ctypes.sizeof(py))
    for f, off in zip(fields, c[1:]):
        assert off == getattr(py, f).offset, (struct, f, off, getattr(py, f).offset)
