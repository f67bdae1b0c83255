"""GB300-native CSR SpMM and SDDMM.

The compute path is libgbsp.so (hand-written CUDA for sm_103a behind the C ABI of
include/gbsp.h); this package is its thin Python binding.  Importing it fails loudly when
the library is not built: there is no CPU fallback.
"""
from ._lib import GbspError, LIB_PATH  # noqa: F401
from .ops import (  # noqa: F401
    BatchPlan,
    sddmm_csr_batched,
    spmm_csr_batched,
    N_PARAMS,
    N_VARIANTS,
    autotune,
    autotune_sddmm,
    sddmm_variant_options,
    N_SDDMM_VARIANTS,
    feature_norm,
    features,
    gather_probe,
    mlp_predict,
    mlp_train,
    variant_options,
    GnnPlan,
    gnn_sddmm_spmm_batched,
    gnn_gat_batched,
    HspPlan,
    SellPlan,
    KbinPlan,
    TcPlan,
    auto_choice,
    auto_forget,
    csr_validate,
    launch_count,
    quantize_bf16,
    quantize_e4m3_rows,
    sddmm,
    sddmm_csr,
    sm_count,
    spmm,
    spmm_csr,
    spmm_csr_noalloc,
    spmm_sddmm_host,
)
