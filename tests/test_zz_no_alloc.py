"""The allocation-free SpMM entry point (spmm_csr_noalloc).

Some callers cannot allocate device memory during a call: a process whose HBM is already
handed out by another allocator (an allocation can fail at call time) or a latency-bound
loop that cannot absorb an allocation.  spmm_csr_noalloc keeps its merge-path carries in a
fixed device array of the library instead of the library's pool.  Its results are checked
against the FP64 oracle and against the general entry point (spmm_csr_ex, merge path),
within the FP32 tolerance, on calls made back to back so that each one runs over what the
previous one left in the shared array.  This file is collected last so that a failure here
leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _noalloc(A, Bd, N, C):
    import torch

    from paper_2604_27985_gb300 import _lib

    rp, ci, v = dev(A.rowptr), dev(A.colidx), dev(A.vals)
    st = _lib.lib.spmm_csr_noalloc(rp.data_ptr(), ci.data_ptr(), v.data_ptr(), Bd.data_ptr(), C.data_ptr(), A.M,
                                   A.K, N, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, _lib.lib.gbsp_last_error_message()
    return rp, ci, v


# Back-to-back calls with different matrices and widths.  N = 1024 is the documented
# maximum: its four 256-column tiles make each warp's carries 4 KB, so the 4 MiB array holds
# 1,008 warps, fewer than the occupancy-sized grid (152 SMs x 8 warps x CTAs per SM), and
# the entry point shrinks the grid to what fits.  N = 1020 leaves the last tile ragged.
CASES = [
    ("powerlaw", 64), ("short_and_one_long", 128), ("uniform_100_per_row", 1024), ("powerlaw_wide", 1020),
    ("uniform_100_per_row", 8),
]


def _matrix(name):
    if name == "powerlaw":
        return gen.csr_powerlaw(5000, 4000, 0.99, seed=301)
    if name == "short_and_one_long":
        return gen.csr_from_lengths(np.r_[np.full(700, 2), [3000], np.zeros(40, np.int64)], 3000, seed=302)
    if name == "uniform_100_per_row":
        return gen.csr_uniform(8000, 5000, 0.98, seed=304)
    return gen.csr_powerlaw(3000, 2000, 0.95, seed=305)


def test_noalloc_matches_oracle_and_general_entry_point_back_to_back():
    import torch

    import paper_2604_27985_gb300 as gb

    for k, (name, N) in enumerate(CASES):
        A = _matrix(name)
        B = gen.dense_normal(A.K, N, 303 + k)
        Bd = dev(B)
        C0 = torch.full((A.M, N), float("nan"), device="cuda")
        rp, ci, v = _noalloc(A, Bd, N, C0)
        C1 = gb.spmm(rp, ci, v, Bd, variant="merge")
        torch.cuda.synchronize()
        ref, scale = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
        got = C0.cpu().numpy()
        assert_within(got, ref, scale, TOL, f"noalloc vs oracle, {name} N={N}")
        assert_within(got, C1.cpu().numpy().astype(np.float64), scale, TOL, f"noalloc vs merge path, {name} N={N}")


def test_noalloc_integers_bit_exact_at_maximum_width():
    """Integer values and B: every partial sum is exact in FP32, so the capped grid's
    carries must add up to the oracle's result bit for bit."""
    import torch

    A = gen.csr_powerlaw(4000, 3000, 0.97, seed=306)
    vals = gen.vals_int(A.nnz, 307)
    B = gen.dense_int(A.K, 1024, 308)
    A = A.with_vals(vals.astype(np.float32))
    C = torch.empty((A.M, 1024), device="cuda")
    _noalloc(A, dev(B), 1024, C)
    torch.cuda.synchronize()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.cpu().numpy().astype(np.float64), want)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_2604_27985_gb300 import _lib

    x = torch.zeros(16, device="cuda")
    i = torch.zeros(16, dtype=torch.int32, device="cuda")
    st = _lib.lib.spmm_csr_noalloc(i.data_ptr(), i.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), 1, 1, 1028,
                                   None)
    assert st == -1 and b"exceeds the maximum" in _lib.lib.gbsp_last_error_message()
