"""The host-resident, chunk-streamed SpMM / SDDMM (gbsp_spmm_sddmm_host) gives the same bits
as the device entry points (same row-split kernels, same per-row order) and matches the
oracle, for any number of chunks and buffer slots."""
import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


@pytest.mark.parametrize("chunks,slots", [(1, 2), (3, 2), (8, 3), (50, 4)])
def test_host_pipeline_matches_device(gb, chunks, slots):
    import torch

    A = gen.csr_powerlaw(6000, 5000, 0.99, seed=701)
    B, X, Y = gen.dense_normal(A.K, 64, 702), gen.dense_normal(A.M, 32, 703), gen.dense_normal(A.K, 32, 704)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hp = [pin(a) for a in (A.rowptr, A.colidx, A.vals, B, X, Y)]
    C = torch.full((A.M, 64), np.nan).pin_memory()
    out = torch.full((A.nnz,), np.nan).pin_memory()
    gb.spmm_sddmm_host(hp[0], hp[1], hp[2], B=hp[3], C=C, X=hp[4], Y=hp[5], out=out, chunks=chunks, slots=slots)
    torch.cuda.synchronize()
    Cd = gb.spmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B), variant="rowsplit").cpu().numpy()
    od = gb.sddmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(X), dev(Y), variant="rowsplit").cpu().numpy()
    assert np.array_equal(C.numpy(), Cd)
    assert np.array_equal(out.numpy(), od)
    ref, sc = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C.numpy(), ref, sc, 1e-5, "host spmm")


def test_host_pipeline_single_op_and_empty_rows(gb):
    import torch

    lengths = np.r_[np.zeros(30, np.int64), np.full(500, 40), np.zeros(20, np.int64)]
    A = gen.csr_from_lengths(lengths, 900, seed=705)
    X, Y = gen.dense_normal(A.M, 16, 706), gen.dense_normal(A.K, 16, 707)
    out = np.full(A.nnz, np.nan, dtype=np.float32)
    gb.spmm_sddmm_host(A.rowptr, A.colidx, A.vals, X=X, Y=Y, out=out, ncols=A.K, chunks=4)
    torch.cuda.synchronize()
    ref, sc = oracle.sddmm(A.rowptr, A.colidx, A.vals, X, Y)
    assert_within(out, ref, sc, 1e-5, "host sddmm only")
    B = gen.dense_normal(A.K, 8, 708)
    C = np.full((A.M, 8), np.nan, dtype=np.float32)
    gb.spmm_sddmm_host(A.rowptr, A.colidx, A.vals, B=B, C=C, chunks=7, slots=2)
    torch.cuda.synchronize()
    ref, sc = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref, sc, 1e-5, "host spmm only")
