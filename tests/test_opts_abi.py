"""The binding's ctypes mirror of tucker_opts has the C struct's size and
field offsets (compiled from include/tucker.h with the host C compiler)."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_1804_09494_gb300 import tucker as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELDS = ["prec", "P_bins", "gauss_seidel", "timing", "wait_cap", "ttm_path", "alloc", "free", "alloc_user", "svd", "reserved"]


def test_opts_layout_matches_header():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"tucker.h\"\nint main(void) {\n"
    src += '  printf("%zu\\n", sizeof(tucker_opts));\n'
    for f in FIELDS:
        src += f'  printf("%zu\\n", offsetof(tucker_opts, {f}));\n'
    src += "  return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        with open(os.path.join(d, "m.c"), "w") as fh:
            fh.write(src)
        exe = os.path.join(d, "m")
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), os.path.join(d, "m.c"), "-o", exe], check=True)
        out = [int(x) for x in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(T.Opts)
    for f, off in zip(FIELDS, out[1:]):
        assert getattr(T.Opts, f).offset == off, f
