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


def _prototypes():
    """name -> (return type, [parameter declarations]) of every function the
    header declares (comments removed, declarations joined across lines)."""
    import re as _re
    src = open(os.path.join(ROOT, "include", "kdefft.h")).read()
    src = _re.sub(r"/\*.*?\*/", "", src, flags=_re.S)
    out = {}
    for m in _re.finditer(r"(int|const char\*)\s+(kdefft_\w+)\s*\(([^)]*)\)\s*;", src):
        params = [p.strip() for p in m.group(3).split(",") if p.strip() and p.strip() != "void"]
        out[m.group(2)] = (m.group(1), params)
    return out


def _kind_of_decl(p):
    if "*" in p or p.split()[0] in ("kdefft_ctx", "kdefft_ds"):
        return "ptr"
    t = p.replace("const ", "").split()[0]
    return {"int": "int", "int64_t": "int64", "double": "double"}[t]


def _kind_of_ctype(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and t.__name__.startswith("LP_"):
        return "ptr"
    return {ctypes.c_int: "int", ctypes.c_int64: "int64", ctypes.c_double: "double"}[t]


def test_binding_signatures_match_the_header(lib_path):
    """Every ctypes prototype the binding sets has the header's number of
    parameters, and each parameter the header's kind (pointer, int, int64,
    double): a mismatch would pass the wrong bytes through the C ABI."""
    import paper_1511_07482_gb300 as pkg
    lib = pkg.load()
    protos = _prototypes()
    assert set(protos) == set(_declared())
    for name, (ret, params) in protos.items():
        f = getattr(lib, name)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == len(params), (name, len(f.argtypes), params)
        for i, (t, p) in enumerate(zip(f.argtypes, params)):
            assert _kind_of_ctype(t) == _kind_of_decl(p), (name, i, p, t)
        assert (f.restype is ctypes.c_char_p) == (ret == "const char*"), name


def test_binding_constants_match_the_header():
    """The status codes and option enums of the binding carry the header's
    values (KDEFFT_X in the header is X in the binding)."""
    import re as _re
    from paper_1511_07482_gb300 import _lib
    src = _re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "kdefft.h")).read(), flags=_re.S)
    consts = {m.group(1): int(m.group(2)) for m in _re.finditer(r"#define KDEFFT_(\w+)\s+(\d+)\s*$", src, _re.M)}
    for body in _re.findall(r"enum\s*\{([^}]*)\}", src):
        for m in _re.finditer(r"KDEFFT_(\w+)\s*=\s*(\d+)", body):
            consts[m.group(1)] = int(m.group(2))
    checked = 0
    for name, value in consts.items():
        if hasattr(_lib, name):
            assert getattr(_lib, name) == value, name
            checked += 1
    assert checked >= 25
    for name in ("OK", "ERR_ARG", "ERR_NOT_SPD", "ERR_OUTSIDE_GRID", "ERR_CUDA", "ERR_TIMEOUT", "P_MINIMAL",
                 "FP32", "FP64", "BIN_SIMPLE", "LSCV", "SCV", "PI", "DT_I32"):
        assert hasattr(_lib, name) and consts[name] == getattr(_lib, name), name
