"""FP64 CPU oracle for CSR SpMM (Eq. 1) and SDDMM (Eq. 2), plus the BF16 / E4M3 roundings.

TEST INFRASTRUCTURE ONLY: the tests, the benchmark's CPU-baseline leg and the smoke check
import this package; the library never does.  The arithmetic lives in ``oracle.c`` (plain
loops in double precision); this module only marshals numpy arrays into it.  It shares no
code with the CUDA library.

Parity pins: every routine here is checked by ``tests/test_oracle.py`` against brute-force
dense products, numpy / torch library routines, closed forms and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.oracle_spmm_f64.argtypes = [I64, I64, I64, P, P, P, P, P, P, I]
        lib.oracle_sddmm_f64.argtypes = [I64, I64, I64, P, P, P, P, P, P, P, I]
        lib.oracle_bf16_round.argtypes = [I64, P, P]
        lib.oracle_bf16_decode.argtypes = [I64, P, P]
        lib.oracle_e4m3_round.argtypes = [I64, P, P]
        lib.oracle_e4m3_decode.argtypes = [I64, P, P]
        lib.oracle_e4m3_rows.argtypes = [I64, P, I64, P, P, P]
        lib.oracle_e4m3_fold.argtypes = [I64, I64, P, P, P, P, P, I, P, P, P, P]
        lib.oracle_max_threads.restype = I
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else None


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def spmm(rowptr, colidx, vals, B, threads: int = 0):
    """C = A B and the per-output scale sum |a||b| (Eq. 1), all in FP64."""
    lib = _load()
    rowptr, colidx = _c(rowptr, np.int32), _c(colidx, np.int32)
    vals, B = _c(vals, np.float64), _c(B, np.float64)
    M = rowptr.shape[0] - 1
    K, N = B.shape
    C = np.empty((M, N), dtype=np.float64)
    S = np.empty((M, N), dtype=np.float64)
    lib.oracle_spmm_f64(M, K, N, _p(rowptr), _p(colidx), _p(vals), _p(B), _p(C), _p(S), threads)
    return C, S


def sddmm(rowptr, colidx, svals, X, Y, threads: int = 0):
    """out[p] = s_p <X_i, Y_j> on the pattern of S, and its scale (Eq. 2), in FP64."""
    lib = _load()
    rowptr, colidx = _c(rowptr, np.int32), _c(colidx, np.int32)
    svals, X, Y = _c(svals, np.float64), _c(X, np.float64), _c(Y, np.float64)
    M, Kd = X.shape
    N = Y.shape[0]
    nnz = colidx.shape[0]
    out = np.empty(nnz, dtype=np.float64)
    S = np.empty(nnz, dtype=np.float64)
    lib.oracle_sddmm_f64(M, N, Kd, _p(rowptr), _p(colidx), _p(svals), _p(X), _p(Y), _p(out),
                         _p(S), threads)
    return out, S


def bf16_round(x) -> np.ndarray:
    """BF16 bits (uint16) of the round-to-nearest-even conversion of FP32 values."""
    x = _c(x, np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    _load().oracle_bf16_round(x.size, _p(x), _p(out))
    return out


def bf16_decode(h) -> np.ndarray:
    h = _c(h, np.uint16)
    out = np.empty(h.shape, dtype=np.float64)
    _load().oracle_bf16_decode(h.size, _p(h), _p(out))
    return out


def e4m3_round(x) -> np.ndarray:
    """E4M3 codes of the saturating round-to-nearest-even conversion of FP32 values."""
    x = _c(x, np.float32)
    out = np.empty(x.shape, dtype=np.uint8)
    _load().oracle_e4m3_round(x.size, _p(x), _p(out))
    return out


def e4m3_decode(q) -> np.ndarray:
    q = _c(q, np.uint8)
    out = np.empty(q.shape, dtype=np.float64)
    _load().oracle_e4m3_decode(q.size, _p(q), _p(out))
    return out


def e4m3_rows(x, rowptr=None):
    """Per-row scaled E4M3: (codes, FP32 row scales).  Rows are CSR segments when
    ``rowptr`` is given, else the rows of the 2-D array ``x``."""
    x = _c(x, np.float32)
    if rowptr is None:
        nrows, ncols = x.shape
        rp = None
    else:
        rp = _c(rowptr, np.int32)
        nrows, ncols = rp.shape[0] - 1, 0
    q = np.empty(x.shape, dtype=np.uint8)
    s = np.empty(nrows, dtype=np.float32)
    _load().oracle_e4m3_rows(nrows, _p(rp) if rp is not None else None, ncols, _p(x), _p(q), _p(s))
    return q, s


def e4m3_rows_dequant(q, s, rowptr=None) -> np.ndarray:
    """FP64 values s_r * decode(q) of a per-row scaled E4M3 array."""
    v = e4m3_decode(q)
    if rowptr is None:
        return v * np.asarray(s, dtype=np.float64)[:, None]
    lengths = np.diff(np.asarray(rowptr, dtype=np.int64))
    return v * np.repeat(np.asarray(s, dtype=np.float64), lengths)


def e4m3_fold(rowptr, colidx, K, qa, sa, tb, threshold=0):
    """Operands of the E4M3 condensed-tile SpMM: aligned 16 x 8 blocks with at least
    ``threshold`` entries (10 when < 1) are dense; their entries take a~ = fl32(fl32(s_i
    dec(q)) t_k), each row is requantised to E4M3 with the power-of-two scale u_i = 2^e (e
    the smallest >= -126 with max |a~| <= 448 u_i).  Returns (codes, dense, eff, exps):
    per entry the requantised code (the input code outside dense blocks), whether it is
    dense, and the FP64 value the product uses (u_i dec(q') or s_i dec(q) t_k); per row e."""
    lib = _load()
    rp, ci = _c(rowptr, np.int32), _c(colidx, np.int32)
    qa, sa, tb = _c(qa, np.uint8), _c(sa, np.float32), _c(tb, np.float32)
    M, nnz = rp.shape[0] - 1, ci.shape[0]
    codes = np.empty(nnz, np.uint8)
    dense = np.empty(nnz, np.uint8)
    eff = np.empty(nnz, np.float64)
    exps = np.empty(M, np.int32)
    lib.oracle_e4m3_fold(M, int(K), _p(rp), _p(ci), _p(qa), _p(sa), _p(tb), int(threshold), _p(codes), _p(dense),
                         _p(eff), _p(exps))
    return codes, dense.astype(bool), eff, exps


def row_softmax(rowptr, E):
    """Softmax over each row's stored entries: a_ij = exp(E_ij - m_i) / sum_j exp(E_ij - m_i)
    with m_i the row's largest E (the attention normalisation of a GAT layer, which the
    paper names as the SDDMM -> SpMM use case).  Empty rows have no entries."""
    rp = np.asarray(rowptr, dtype=np.int64)
    E = np.asarray(E, dtype=np.float64)
    out = np.empty_like(E)
    for i in range(rp.size - 1):
        a, b = rp[i], rp[i + 1]
        if a == b:
            continue
        w = np.exp(E[a:b] - E[a:b].max())
        out[a:b] = w / w.sum()
    return out


def gat_chain(rowptr, colidx, svals, H, threads: int = 0):
    """Per graph: E = S o (H H^T) on the pattern of S (Eq. 2 with X = Y = H), alpha = the
    softmax of each row's E, then O = alpha H (Eq. 1 with A's values replaced by alpha).
    Returns alpha, O and O's scale (sum_j alpha_ij |H_jn|)."""
    E, _ = sddmm(rowptr, colidx, svals, H, H, threads)
    alpha = row_softmax(rowptr, E)
    O, sO = spmm(rowptr, colidx, alpha, H, threads)
    return alpha, O, sO


def gnn_chain(rowptr, colidx, svals, H, threads: int = 0):
    """Per graph: E = S o (H H^T) on the pattern of S (Eq. 2 with X = Y = H), then
    O = E H (Eq. 1 with A's values replaced by E).  Returns E, O and both scales."""
    E, sE = sddmm(rowptr, colidx, svals, H, H, threads)
    O, sO = spmm(rowptr, colidx, E, H, threads)
    return E, O, sE, sO
