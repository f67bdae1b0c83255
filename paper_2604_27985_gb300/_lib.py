"""ctypes view of the C ABI in include/gbsp.h (argument marshalling only).

The shared library is built in-tree by ``paper_2604_27985_gb300.build``.  There is no
fallback: if libgbsp.so is missing or does not load, importing this module fails.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbsp.so")

GBSP_OK = 0
STATUS = {
    0: "GBSP_OK",
    -1: "GBSP_ERR_INVALID_ARG",
    -2: "GBSP_ERR_INVALID_CSR",
    -3: "GBSP_ERR_ALIGN",
    -4: "GBSP_ERR_UNSUPPORTED",
    -5: "GBSP_ERR_CUDA",
    -6: "GBSP_ERR_OOM",
    -7: "GBSP_ERR_TIMEOUT",
}
F32, BF16, E4M3 = 0, 1, 2
VARIANTS = {"auto": 0, "rowsplit": 1, "merge": 2, "scalar": 3, "entry": 4, "rowgroup": 5}


class GbspError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Csr(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("vals", ctypes.c_void_p),
                ("row_scale", ctypes.c_void_p), ("dtype", ctypes.c_int32)]


class Dense(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("ld", ctypes.c_int64), ("row_scale", ctypes.c_void_p), ("dtype", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("validate", ctypes.c_int32), ("unroll", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("vecs", ctypes.c_int32)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_2604_27985_gb300.build` "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    sig = {
        "spmm_csr": [P, P, P, P, P, I64, I64, I64],
        "sddmm_csr": [P, P, P, P, P, P, I64, I64, I64],
        "spmm_csr_noalloc": [P, P, P, P, P, I64, I64, I64, P],
        "gbsp_gather_probe": [P, I64, I64, I64, P, I64, P, I, I, P],
        "gbsp_plan_sddmm": [P, P, ctypes.POINTER(Dense), ctypes.POINTER(Dense), P, I, P],
        "spmm_csr_ex": [ctypes.POINTER(Csr), ctypes.POINTER(Dense), ctypes.POINTER(Dense), ctypes.POINTER(Opts), P],
        "sddmm_csr_ex": [ctypes.POINTER(Csr), ctypes.POINTER(Dense), ctypes.POINTER(Dense), P,
                         ctypes.POINTER(Opts), P],
        "gbsp_csr_validate": [ctypes.POINTER(Csr), P, ctypes.POINTER(ctypes.c_int64)],
        "gbsp_auto_choice": [ctypes.POINTER(Csr), ctypes.c_int32, I64, I64, P, ctypes.POINTER(ctypes.c_int32),
                             ctypes.POINTER(I64)],
        "gbsp_quantize_bf16": [P, P, I64, P],
        "gbsp_quantize_e4m3_rows": [P, P, I64, I64, I64, P, P, P],
        "gbsp_plan_create": [ctypes.POINTER(Csr), ctypes.c_int32, ctypes.POINTER(Opts), P, ctypes.POINTER(P)],
        "gbsp_plan_execute": [P, ctypes.POINTER(Dense), ctypes.POINTER(Dense), P],
        "gbsp_plan_info": [P, ctypes.POINTER(I64), I],
        "gbsp_plan_check": [P, P],
        "gbsp_plan_test_withhold": [P, ctypes.c_int32],
        "gbsp_gnn_plan_create": [I, ctypes.POINTER(Csr), ctypes.POINTER(Dense), ctypes.POINTER(P),
                                 ctypes.POINTER(Dense), ctypes.c_int32, P, ctypes.POINTER(P)],
        "gbsp_gnn_plan_execute": [P, P],
        "gbsp_gnn_plan_info": [P, ctypes.POINTER(I64), I],
        "gnn_sddmm_spmm_batched": [I, ctypes.POINTER(Csr), ctypes.POINTER(Dense), ctypes.POINTER(P),
                                   ctypes.POINTER(Dense), P],
        "gbsp_gnn_plan_create_ex": [I, ctypes.POINTER(Csr), ctypes.POINTER(Dense), ctypes.POINTER(P),
                                    ctypes.POINTER(Dense), ctypes.c_int32, ctypes.c_int32, P, ctypes.POINTER(P)],
        "gnn_gat_batched": [I, ctypes.POINTER(Csr), ctypes.POINTER(Dense), ctypes.POINTER(P), ctypes.POINTER(Dense),
                            P],
        "gbsp_kbin_plan_create": [ctypes.POINTER(Csr), I64, I64, P, ctypes.POINTER(P)],
        "gbsp_kbin_plan_execute": [P, ctypes.POINTER(Dense), ctypes.POINTER(Dense), P],
        "gbsp_kbin_plan_info": [P, ctypes.POINTER(I64), I],
        "gbsp_sell_plan_create": [ctypes.POINTER(Csr), ctypes.c_int32, ctypes.c_int32, P, ctypes.POINTER(P)],
        "gbsp_sell_plan_execute": [P, ctypes.POINTER(Dense), ctypes.POINTER(Dense), P],
        "gbsp_sell_plan_info": [P, ctypes.POINTER(I64), I],
        "gbsp_hsp_plan_create": [ctypes.POINTER(Csr), P, ctypes.POINTER(P)],
        "gbsp_hsp_plan_execute": [P, ctypes.POINTER(Dense), ctypes.POINTER(Dense), P],
        "gbsp_hsp_plan_info": [P, ctypes.POINTER(I64), I],
        "gbsp_variant_opts": [I, ctypes.POINTER(Opts)],
        "gbsp_sddmm_variant_opts": [I, ctypes.POINTER(Opts)],
        "gbsp_autotune_sddmm": [ctypes.POINTER(Csr), ctypes.POINTER(Dense), ctypes.POINTER(Dense), P, I,
                                ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32), P],
        "gbsp_features": [ctypes.POINTER(Csr), I64, ctypes.c_int32, P, P],
        "gbsp_feature_norm": [P, I, P, P],
        "gbsp_mlp_predict": [P, P, P, I, P, P, P],
        "gbsp_mlp_train": [P, P, P, P, P, P, P, I, I, I, ctypes.c_float, I, P],
        "gbsp_autotune": [ctypes.POINTER(Csr), ctypes.POINTER(Dense), ctypes.POINTER(Dense), I,
                          ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32), P],
        "gbsp_spmm_sddmm_host": [P, P, P, P, P, I64, P, P, P, I64, I64, I64, I64, ctypes.c_int32, ctypes.c_int32,
                                 P],
        "gbsp_batch_plan_create_spmm": [I, ctypes.POINTER(Csr), ctypes.POINTER(Dense), ctypes.POINTER(Dense), P,
                                        ctypes.POINTER(P)],
        "gbsp_batch_plan_create_sddmm": [I, ctypes.POINTER(Csr), ctypes.POINTER(Dense), ctypes.POINTER(Dense),
                                         ctypes.POINTER(P), P, ctypes.POINTER(P)],
        "gbsp_batch_plan_execute": [P, P],
        "spmm_csr_batched": [I, ctypes.POINTER(Csr), ctypes.POINTER(Dense), ctypes.POINTER(Dense), P],
        "sddmm_csr_batched": [I, ctypes.POINTER(Csr), ctypes.POINTER(Dense), ctypes.POINTER(Dense),
                              ctypes.POINTER(P), P],
        "gbsp_get_last_error": [],
        "gbsp_device_sm_count": [],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = I
    lib.gbsp_auto_forget.argtypes = []
    lib.gbsp_auto_forget.restype = None
    lib.gbsp_batch_plan_destroy.argtypes = [P]
    lib.gbsp_batch_plan_destroy.restype = None
    lib.gbsp_sell_plan_destroy.argtypes = [P]
    lib.gbsp_sell_plan_destroy.restype = None
    lib.gbsp_hsp_plan_destroy.argtypes = [P]
    lib.gbsp_hsp_plan_destroy.restype = None
    lib.gbsp_kbin_plan_destroy.argtypes = [P]
    lib.gbsp_kbin_plan_destroy.restype = None
    lib.gbsp_gnn_plan_destroy.argtypes = [P]
    lib.gbsp_gnn_plan_destroy.restype = None
    lib.gbsp_plan_destroy.argtypes = [P]
    lib.gbsp_plan_destroy.restype = None
    lib.gbsp_status_string.argtypes = [I]
    lib.gbsp_status_string.restype = ctypes.c_char_p
    lib.gbsp_launch_count.argtypes = []
    lib.gbsp_launch_count.restype = ctypes.c_int64
    lib.gbsp_last_error_message.argtypes = []
    lib.gbsp_last_error_message.restype = ctypes.c_char_p
    return lib


lib = _load()


def check(status: int) -> None:
    if status != GBSP_OK:
        msg = lib.gbsp_last_error_message().decode(errors="replace")
        raise GbspError(status, msg or lib.gbsp_status_string(status).decode())
