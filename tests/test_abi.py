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


def _lib():
    from paper_2311_00921_gb300 import hss
    if not os.path.exists(hss.LIB_PATH):
        pytest.skip("library not built (run __graft_entry__.build())")
    return hss, hss.load()


def test_create_refuses_bad_shapes_before_any_device_call():
    """Argument errors of hss_create come back as HSS_ERR_INVALID_ARG from the
    host-side checks, before the library touches a device."""
    hss, lib = _lib()
    buf = (ctypes.c_double * 8)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    out = ctypes.c_void_p()

    def create(n, leaf, rank, levels, sizes=None, E=p, on_device=0):
        sh = hss.Shape(n, leaf, rank, levels, sizes)
        return lib.hss_create(ctypes.byref(sh), p, p, E, p, on_device, ctypes.byref(out))

    assert lib.hss_create(None, p, p, p, p, 0, ctypes.byref(out)) == -1
    assert create(1025 * 4, 1025, 16, 2) == -1          # leaf above 1024
    assert create(64 * 4, 64, 65, 2) == -1              # rank above leaf
    assert create(512 * 4, 512, 257, 2) == -1           # rank above 256
    assert create(64, 64, 16, 0) == -1                  # no level
    assert create(64 << 25, 64, 16, 25) == -1           # too many levels
    assert create(64 * 4 + 1, 64, 16, 2) == -1          # n is not leaf * 2^L
    assert create(64 * 4, 64, 16, 2, E=None) == -1      # transfers missing
    sizes = (ctypes.c_int32 * 4)(60, 64, 64, 70)        # a leaf order above leaf
    assert create(258, 64, 16, 2, ctypes.cast(sizes, ctypes.POINTER(ctypes.c_int32))) == -1
    sizes = (ctypes.c_int32 * 4)(60, 64, 64, 60)        # orders not summing to n
    assert create(250, 64, 16, 2, ctypes.cast(sizes, ctypes.POINTER(ctypes.c_int32))) == -1
    sizes = (ctypes.c_int32 * 4)(60, 64, 64, 60)        # uneven trees come from the host
    assert create(248, 64, 16, 2, ctypes.cast(sizes, ctypes.POINTER(ctypes.c_int32)),
                  on_device=1) == -1
    assert out.value is None


def test_null_handles_and_error_names():
    hss, lib = _lib()
    d = ctypes.c_double()
    assert lib.hss_factorize(None, None, None) == -1
    assert lib.hss_solve(None, None, None, 1, 1, None) == -1
    assert lib.hss_matvec(None, None, None, 1, 1, None) == -1
    assert lib.hss_logdet(None, ctypes.byref(d)) == -1
    assert lib.hss_sync(None) == -1
    assert lib.hss_trace(None, 1) == -1
    lib.hss_destroy(None)                               # a no-op
    names = [lib.hss_strerror(c) for c in range(0, -9, -1)]
    assert all(names) and len(set(names)) == len(names), names
