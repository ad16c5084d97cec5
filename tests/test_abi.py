"""The C-ABI library builds for sm_103a and exports every function include/sah.h declares.
No compute call is made here (no GPU needed)."""
import ctypes
import os
import subprocess

import pytest

import paper_2211_12751_gb300 as lib


@pytest.fixture(scope="module")
def libpath():
    return lib.build()


def test_header_declares_the_boundary():
    names = lib.declared_functions()
    for required in ("sah_build_index", "sah_rkmips", "sah_rkmips_batch", "sah_free_index",
                     "sah_index_stats", "sah_status_string", "sah_last_error", "sah_default_params"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    so = ctypes.CDLL(libpath)
    missing = [n for n in lib.declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_exports_are_c_symbols(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for n in lib.declared_functions():
        assert n in exported, n


def test_params_struct_matches_defaults(libpath):
    lib._lib = None
    p = lib.default_params()
    assert (p.k_max, p.leaf_size, p.n_tables, p.code_bits) == (50, 20, 128, 16)
    assert abs(p.b - 0.5) < 1e-7 and p.srp is None


def test_status_strings(libpath):
    so = lib.load()
    assert so.sah_status_string(0) == b"ok"
    assert so.sah_status_string(4) == b"result buffer too small"


def _c_layout(struct: str, fields):
    """sizeof and offsetof of a struct of include/sah.h, from a C program compiled with gcc."""
    import shutil
    import tempfile
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lines = [f'  printf("%zu\\n", sizeof({struct}));']
    lines += [f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    src = ("#include <stdio.h>\n#include <stddef.h>\n#include \"sah.h\"\nint main(void) {\n"
           + "\n".join(lines) + "\n  return 0;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(c, "w") as f:
            f.write(src)
        subprocess.run([gcc, "-std=c99", "-I", os.path.join(root, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("struct, cls", [("sah_params", "Params"), ("sah_stats", "Stats")])
def test_ctypes_structs_match_the_header_layout(struct, cls):
    """The binding's ctypes mirrors have the C structs' fields, in order, at the same offsets
    and with the same size, so that no field is read from the wrong place."""
    py = getattr(lib, cls)
    names = [n for n, _ in py._fields_]
    size, offsets = _c_layout(struct, names)
    assert ctypes.sizeof(py) == size
    assert [getattr(py, n).offset for n in names] == offsets
