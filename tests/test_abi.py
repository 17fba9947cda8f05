"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every function that include/kdefft.h declares; the Python
binding's structure layout matches the header."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1511_07482_gb300 import build
    return build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "kdefft.h")).read()
    return sorted(set(re.findall(r"\b(kdefft_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["kdefft_create", "kdefft_bin", "kdefft_psi", "kdefft_lscv", "kdefft_scv", "kdefft_pi",
              "kdefft_select_H", "kdefft_batch_lscv", "kdefft_counts"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (kdefft_[A-Za-z0-9_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches(lib_path):
    import paper_1511_07482_gb300 as pkg
    lib = pkg.load()
    for n in _declared():
        assert hasattr(lib, n)
    assert set(pkg.EXPORTS) == set(_declared())
    # default options through the C ABI (no GPU needed)
    o = pkg.default_opts()
    assert o.tau == 3.7 and o.P_rule == pkg.P_MINIMAL and o.precision == pkg.FP32
    assert lib.kdefft_strerror(2) == b"matrix not symmetric positive definite"


def test_create_without_gpu_fails_loudly(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1511_07482_gb300 as pkg
    with pytest.raises(pkg.KdefftError):
        pkg.Context(0, stream=0)


def test_opts_struct_size_matches_header(lib_path):
    import paper_1511_07482_gb300 as pkg
    # double + 2 int + 4 int + 4 int = 8 + 40 = 48 bytes
    assert ctypes.sizeof(pkg._lib.Opts) == 48
