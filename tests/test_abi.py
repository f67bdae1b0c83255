"""The C ABI library builds, loads and exports every entry point its headers declare, and
rejects bad arguments synchronously (no GPU needed for any of this)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2604_27985_gb300 as g

    return g


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char|int64_t)\s*\*?\s*(\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_plain_and_descriptor_calls():
    names = declared_functions()
    for n in ("spmm_csr", "sddmm_csr", "spmm_csr_ex", "sddmm_csr_ex", "gbsp_csr_validate"):
        assert n in names


def test_every_declared_symbol_is_exported(gb):
    from paper_2604_27985_gb300 import _lib

    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in declared_functions():
        getattr(_lib.lib, n)  # resolvable through ctypes too
    # nothing beyond the declared C ABI leaks out
    extra = [n for n in exported if n not in declared_functions()]
    assert not extra, f"exported but not declared: {extra}"


def test_status_strings(gb):
    from paper_2604_27985_gb300._lib import lib

    for s in range(0, -8, -1):
        assert lib.gbsp_status_string(s)
    assert lib.gbsp_status_string(-99) == b"unknown status"


def test_argument_errors_return_without_launching(gb):
    from paper_2604_27985_gb300 import _lib

    lib = _lib.lib
    P = ctypes.byref
    assert lib.spmm_csr_ex(None, None, None, None, None) == -1
    assert b"null" in lib.gbsp_last_error_message()
    A = _lib.Csr(4, 5, 3, 16, 16, 16, None, _lib.F32)
    B = _lib.Dense(16, 6, 8, 8, None, _lib.F32)  # B rows != A cols
    C = _lib.Dense(16, 4, 8, 8, None, _lib.F32)
    assert lib.spmm_csr_ex(P(A), P(B), P(C), None, None) == -1
    B = _lib.Dense(16, 5, 8, 4, None, _lib.F32)  # ld < cols
    assert lib.spmm_csr_ex(P(A), P(B), P(C), None, None) == -1
    B = _lib.Dense(16, 5, 8, 8, None, _lib.BF16)  # dtype mismatch with A
    assert lib.spmm_csr_ex(P(A), P(B), P(C), None, None) == -4
    B = _lib.Dense(16, 5, 8, 8, None, _lib.F32)
    o = _lib.Opts(1, 0, 3, 0, 0)  # unroll 3 is not offered
    assert lib.spmm_csr_ex(P(A), P(B), P(C), P(o), None) == -1
    o = _lib.Opts(1, 0, 2, 0, 3)  # 3 vectors per lane are not offered
    assert lib.spmm_csr_ex(P(A), P(B), P(C), P(o), None) == -1
    E = _lib.Dense(16, 5, 8, 8, None, _lib.E4M3)  # E4M3 without row scales
    assert lib.spmm_csr_ex(P(A), P(E), P(C), None, None) == -1
    S = _lib.Csr(4, 5, 3, 16, 16, 16, None, _lib.BF16)  # SDDMM values must be FP32
    X = _lib.Dense(16, 4, 8, 8, None, _lib.F32)
    Y = _lib.Dense(16, 5, 8, 8, None, _lib.F32)
    assert lib.sddmm_csr_ex(P(S), P(X), P(Y), 16, None, None) == -4
    S = _lib.Csr(4, 5, 3, 16, 16, 16, None, _lib.F32)
    Y = _lib.Dense(16, 6, 8, 8, None, _lib.F32)
    assert lib.sddmm_csr_ex(P(S), P(X), P(Y), 16, None, None) == -1
    assert lib.gbsp_quantize_bf16(None, None, -1, None) == -1
    assert lib.gbsp_quantize_e4m3_rows(None, None, 2, 4, 2, None, None, None) == -1
    assert lib.gbsp_get_last_error() == -1


def _run_with_fault(fault, code):
    import subprocess
    import sys

    env = dict(os.environ, GBSP_FAULT=fault)
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    return r.stdout.strip()


def test_injected_faults_surface_as_status_codes(gb):
    """GBSP_FAULT makes the library take its error paths before touching a GPU."""
    code = (
        "import ctypes\n"
        "from paper_2604_27985_gb300 import _lib\n"
        "lib = _lib.lib; P = ctypes.byref\n"
        "A = _lib.Csr(4, 5, 3, 16, 16, 16, None, _lib.F32)\n"
        "B = _lib.Dense(16, 5, 8, 8, None, _lib.F32); C = _lib.Dense(16, 4, 8, 8, None, _lib.F32)\n"
        "X = _lib.Dense(16, 4, 8, 8, None, _lib.F32); Y = _lib.Dense(16, 5, 8, 8, None, _lib.F32)\n"
        "bad = ctypes.c_int64(0)\n"
        "print(lib.spmm_csr_ex(P(A), P(B), P(C), None, None), lib.sddmm_csr_ex(P(A), P(X), P(Y), 16, None, None),\n"
        "      lib.gbsp_csr_validate(P(A), None, P(bad)), bad.value)\n")
    assert _run_with_fault("launch", code).split()[:2] == ["-5", "-5"]
    assert _run_with_fault("alloc", code).split()[2] == "-6"
    assert _run_with_fault("validate", code).split()[2:] == ["-2", "-1"]
