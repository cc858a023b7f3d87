"""The C-ABI library builds, loads without a GPU, and exports every entry
point include/tucker.h declares (no compute call is made here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tucker.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:tucker_status|void|const char\s*\*)\s*\**\s*([A-Za-z_]\w*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1804_09494_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("tucker_init", "ttm_chain", "factor_update", "core", "hooi_iter", "ttm_chain_backward",
                 "tucker_stats", "tucker_last_error", "tucker_destroy"):
        assert want in names


def test_every_declared_symbol_is_exported(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_exports_are_c_symbols(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    for n in declared_functions():
        assert n in exported, n  # unmangled, i.e. extern "C"


def test_binding_declares_same_names(lib_path):
    from paper_1804_09494_gb300 import tucker
    lib = tucker.load_library(lib_path)
    assert set(declared_functions()) == set(tucker.SIGNATURES)
    assert lib is not None


def test_binding_refuses_cpu_tensors(lib_path):
    import torch
    from paper_1804_09494_gb300 import tucker
    with pytest.raises((RuntimeError, TypeError)):
        tucker.Tucker(torch.zeros(3, 4, dtype=torch.int32), torch.zeros(4), (2, 2, 2), (1, 1, 1))
