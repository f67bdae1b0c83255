"""The allocation-free SpMM entry point (spmm_csr_noalloc) against the general one.

spmm_csr_noalloc exists for callers that cannot allocate device memory during a call
(HBM already handed out by another allocator, latency-bound loops, regions recorded into
CUDA graphs); its merge-path carries live in a fixed device array of the library.  This
file is collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev

pytestmark = pytest.mark.gpu
TOL = 1e-5


def test_noalloc_matches_general_entry_point_twice():
    import torch

    import paper_2604_27985_gb300 as gb
    from paper_2604_27985_gb300 import _lib

    # two calls in a row with different matrices and widths: the second must not see
    # anything the first left in the shared scratch
    cases = [(gen.csr_powerlaw(5000, 4000, 0.99, seed=301), 64),
             (gen.csr_from_lengths(np.r_[np.full(700, 2), [3000], np.zeros(40, np.int64)], 3000, seed=302), 128)]
    for A, N in cases:
        B = gen.dense_normal(A.K, N, 303)
        rp, ci, v, Bd = dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B)
        C0 = torch.full((A.M, N), float("nan"), device="cuda")
        st = _lib.lib.spmm_csr_noalloc(rp.data_ptr(), ci.data_ptr(), v.data_ptr(), Bd.data_ptr(), C0.data_ptr(),
                                       A.M, A.K, N, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, _lib.lib.gbsp_last_error_message()
        C1 = gb.spmm(rp, ci, v, Bd, variant="merge")
        torch.cuda.synchronize()
        _, scale = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
        assert_within(C0.cpu().numpy(), C1.cpu().numpy().astype(np.float64), scale, TOL, f"noalloc N={N}")


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_2604_27985_gb300 import _lib

    x = torch.zeros(16, device="cuda")
    i = torch.zeros(16, dtype=torch.int32, device="cuda")
    st = _lib.lib.spmm_csr_noalloc(i.data_ptr(), i.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), 1, 1, 2048,
                                   None)
    assert st == -1 and b"exceeds the maximum" in _lib.lib.gbsp_last_error_message()
