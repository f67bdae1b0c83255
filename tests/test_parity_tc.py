"""GPU parity of the condensed-tile tensor-core SpMM plan (BF16 operands, FP32 accumulation).

Dense 16 x 8 blocks run on tcgen05, the residual on the CSR kernels; the result is C = A B
(Eq. 1).  Integer-valued inputs (exact in BF16, partial sums below 2^24) must match the
oracle bit for bit whatever the split; random inputs are held to the FP32 tolerance
against the oracle on the BF16-rounded operands and to 1e-2 against the FP32 originals.
"""
import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev, sub_csr

pytestmark = pytest.mark.gpu
TOL32, TOL_BF16 = 1e-5, 1e-2


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


def bf16(x):
    import torch

    return dev(oracle.bf16_round(x).view(np.int16)).view(torch.bfloat16)


def plan_of(gb, A, vals, threshold=0):
    return gb.TcPlan(dev(A.rowptr), dev(A.colidx), bf16(vals), A.K, threshold)


@pytest.mark.parametrize("threshold", [0, 1, 40, 129])
@pytest.mark.parametrize("N", [128, 256])
def test_tc_integers_bit_exact(gb, threshold, N):
    """threshold 1: every occupied block on the tensor cores; 129: none; 0 (default 14) and
    40: the clustered blocks on the tensor cores, the scattered rest on the CSR kernels."""
    A = gen.csr_clustered(1024, 1024, 0.9, seed=401)
    vals = gen.vals_int(A.nnz, 402)
    B = gen.dense_int(A.K, N, 403)
    plan = plan_of(gb, A, vals, threshold)
    info = plan.info()
    assert info["dense_nnz"] + info["residual_nnz"] == A.nnz
    if threshold == 129:
        assert info["dense_windows"] == 0
    else:
        assert info["dense_windows"] > 0
    C = plan.execute(bf16(B)).cpu().numpy()
    plan.check()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.astype(np.float64), want)


@pytest.mark.parametrize("shape", [(2000, 2003, 384), (1000, 1000, 136), (64, 4096, 512), (1001, 64, 64)])
def test_tc_ragged_shapes(gb, shape):
    """M not a multiple of 16, K not a multiple of 8, N not a multiple of 128."""
    M, K, N = shape
    lengths = np.random.default_rng(404).integers(0, min(K, 300), M)
    A = gen.csr_from_lengths(lengths, K, seed=405)
    vals = gen.vals_int(A.nnz, 406)
    B = gen.dense_int(K, N, 407)
    plan = plan_of(gb, A, vals, threshold=2)
    C = plan.execute(bf16(B)).cpu().numpy()
    plan.check()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.astype(np.float64), want)


def test_tc_random_values(gb):
    A = gen.csr_clustered(2048, 2048, 0.9, seed=408)
    B = gen.dense_normal(A.K, 256, 409)
    plan = plan_of(gb, A, A.vals)
    assert plan.info()["dense_windows"] > 0
    C = plan.execute(bf16(B)).cpu().numpy()
    plan.check()
    da = oracle.bf16_decode(oracle.bf16_round(A.vals))
    db = oracle.bf16_decode(oracle.bf16_round(B))
    ref, sc = oracle.spmm(A.rowptr, A.colidx, da, db)
    assert_within(C, ref, sc, TOL32, "tc dequantised")
    ref0, sc0 = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref0, sc0, TOL_BF16, "tc vs fp32")


def test_tc_repeated_execute_and_padded_ld(gb):
    import torch

    A = gen.csr_clustered(1024, 1024, 0.9, seed=410)
    vals = gen.vals_int(A.nnz, 411)
    plan = plan_of(gb, A, vals)
    want = None
    for seed in (412, 413):
        Bf = gen.dense_int(A.K, 264, seed)
        Bv = bf16(Bf)[:, :256]  # ld = 264
        Cfull = torch.full((A.M, 260), 5.0, device="cuda")
        C = plan.execute(Bv, out=Cfull[:, :256])
        want, _ = oracle.spmm(A.rowptr, A.colidx, vals, Bf[:, :256])
        assert np.array_equal(C.cpu().numpy().astype(np.float64), want)
        assert torch.all(Cfull[:, 256:] == 5.0)
    plan.check()


def test_tc_rejects_unsorted_columns(gb):
    A = gen.csr_uniform(64, 64, 0.5, seed=414)
    ci = A.colidx.copy()
    ci[A.rowptr[3]:A.rowptr[4]] = ci[A.rowptr[3]:A.rowptr[4]][::-1]
    with pytest.raises(gb.GbspError, match="UNSUPPORTED"):
        gb.TcPlan(dev(A.rowptr), dev(ci), bf16(A.vals), A.K)


def test_tc_full_size_clustered_sampled_rows(gb):
    """The precision configuration: 16,384^2 at 90%, clustered (16 x 8 blocks at 40% fill
    hold half the nonzeros), N = 256, BF16 — checked on 400 sampled rows."""
    A = gen.csr_clustered(16384, 16384, 0.9, seed=2002)
    B = gen.dense_normal(A.K, 256, 2003)
    plan = plan_of(gb, A, A.vals)
    info = plan.info()
    assert info["dense_nnz"] >= A.meta["block_nnz"]
    C = plan.execute(bf16(B)).cpu().numpy()
    plan.check()
    rows = np.sort(np.random.default_rng(11).choice(A.M, 400, replace=False))
    rp, ci, v, _ = sub_csr(A.rowptr, A.colidx, A.vals, rows)
    da = oracle.bf16_decode(oracle.bf16_round(v))
    db = oracle.bf16_decode(oracle.bf16_round(B))
    ref, sc = oracle.spmm(rp, ci, da, db)
    assert_within(C[rows], ref, sc, TOL32, "tc full size dequantised")
    ref0, sc0 = oracle.spmm(rp, ci, v, B)
    assert_within(C[rows], ref0, sc0, TOL_BF16, "tc full size vs fp32")


def test_tc_bounded_wait_reports_timeout(gb):
    """A stage that never arrives makes the window's MMA warp give up after about a second:
    the kernel returns, gbsp_plan_check reports GBSP_ERR_TIMEOUT, and the next execution on
    the same context is exact again."""
    import time

    A = gen.csr_clustered(512, 512, 0.9, seed=420)
    vals = gen.vals_int(A.nnz, 421)
    B = gen.dense_int(A.K, 128, 422)
    plan = plan_of(gb, A, vals)
    plan.test_withhold(0)
    t0 = time.time()
    plan.execute(bf16(B))
    with pytest.raises(gb.GbspError, match="TIMEOUT"):
        plan.check()
    assert time.time() - t0 < 30
    plan.test_withhold(-1)
    C = plan.execute(bf16(B)).cpu().numpy()
    plan.check()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.astype(np.float64), want)
