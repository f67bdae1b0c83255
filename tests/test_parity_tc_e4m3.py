"""GPU parity of the condensed-tile tensor-core plan on per-row-scaled FP8-E4M3 operands
(tcgen05 kind::f8f6f4, FP32 accumulation).

A holds codes q_ik with row scales s_i, B codes with row scales t_k; C = A B (Eq. 1) on the
dequantised values.  The plan folds t into the dense-block values and requantises each
window row with a power-of-two scale u_r; the oracle states that step (oracle.e4m3_fold,
pinned by a hand-worked example in tests/test_oracle_fold.py), so the expected result is the
FP64 oracle on exactly the operands the tensor cores multiply.  At the precision
configuration the plan is also held to the E4M3 tolerance, 4e-2 of sum |a||b|, against the
FP64 product of the original FP32 values.  Integer inputs with unit scales
pass the requantisation unchanged and must match the oracle bit for bit.
"""
import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev, sub_csr

pytestmark = pytest.mark.gpu
TOL32 = 1e-5
TOL_REQUANT = 2.0 ** -4  # one more E4M3 rounding of each dense-block value: |delta| <= 2^-4 |a~|


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


def effective_values(rowptr, colidx, K, qa, sa, tb, threshold):
    """Per stored entry, the FP64 value the plan multiplies with decode(qb), and whether the
    entry lies in a dense block: the oracle's statement of the fold (oracle.e4m3_fold)."""
    _, dense, eff, _ = oracle.e4m3_fold(rowptr, colidx, K, qa, sa, tb, threshold)
    return eff, dense


def e4m3_plan(gb, A, qa, sa, threshold=0):
    return gb.TcPlan(dev(A.rowptr), dev(A.colidx), dev(qa), A.K, threshold, row_scale=dev(sa))


@pytest.mark.parametrize("threshold", [0, 1, 129])
@pytest.mark.parametrize("N", [96, 128, 256, 512])
def test_tc_e4m3_integers_bit_exact(gb, threshold, N):
    """Integers in [-8, 8] with unit scales: exact in E4M3 before and after the power-of-two
    requantisation, partial sums far below 2^24."""
    A = gen.csr_clustered(1024, 1024, 0.9, seed=431)
    vals = gen.vals_int(A.nnz, 432)
    B = gen.dense_int(A.K, N, 433)
    plan = e4m3_plan(gb, A, oracle.e4m3_round(vals), np.ones(A.M, np.float32), threshold)
    info = plan.info()
    assert info["dense_nnz"] + info["residual_nnz"] == A.nnz
    assert (info["dense_windows"] == 0) == (threshold == 129)
    assert info["dense_blocks"] % 16 == 0
    C = plan.execute(dev(oracle.e4m3_round(B)), row_scale=dev(np.ones(A.K, np.float32))).cpu().numpy()
    plan.check()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.astype(np.float64), want)


@pytest.mark.parametrize("shape", [(2000, 2003, 384), (1000, 1000, 144), (64, 4096, 512), (1001, 64, 64)])
def test_tc_e4m3_ragged_shapes(gb, shape):
    M, K, N = shape
    lengths = np.random.default_rng(434).integers(0, min(K, 300), M)
    A = gen.csr_from_lengths(lengths, K, seed=435)
    vals = gen.vals_int(A.nnz, 436)
    B = gen.dense_int(K, N, 437)
    plan = e4m3_plan(gb, A, oracle.e4m3_round(vals), np.ones(M, np.float32), threshold=2)
    C = plan.execute(dev(oracle.e4m3_round(B)), row_scale=dev(np.ones(K, np.float32))).cpu().numpy()
    plan.check()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.astype(np.float64), want)


@pytest.mark.parametrize("threshold", [0, 1])
@pytest.mark.parametrize("N", [128, 256, 160])
def test_tc_e4m3_random_values(gb, threshold, N):
    """Per-row-scaled E4M3 of normal values (scales far from 1): the plan against the oracle
    on its effective operands (FP32 tolerance) and on the dequantised inputs (the
    requantisation bound)."""
    A = gen.csr_clustered(2048, 2048, 0.9, seed=438)
    B = gen.dense_normal(A.K, N, 439) * 3.0
    qa, sa = oracle.e4m3_rows(A.vals, A.rowptr)
    qb, tb = oracle.e4m3_rows(B)
    plan = e4m3_plan(gb, A, qa, sa, threshold)
    assert plan.info()["dense_windows"] > 0
    C = plan.execute(dev(qb), row_scale=dev(tb)).cpu().numpy()
    plan.check()
    eff, dense = effective_values(A.rowptr, A.colidx, A.K, qa, sa, tb, threshold)
    assert dense.any() and (threshold == 1) == dense.all()
    ref, sc = oracle.spmm(A.rowptr, A.colidx, eff, oracle.e4m3_decode(qb))
    assert_within(C, ref, sc, TOL32, "tc e4m3 effective operands")
    ref0, sc0 = oracle.spmm(A.rowptr, A.colidx, oracle.e4m3_rows_dequant(qa, sa, A.rowptr),
                            oracle.e4m3_rows_dequant(qb, tb))
    assert_within(C, ref0, sc0, TOL_REQUANT, "tc e4m3 dequantised inputs")


def test_tc_e4m3_repeated_execute_new_scales(gb):
    """The fold runs at every execution: a second B with other row scales (and a padded
    leading dimension) gives its own product."""
    import torch

    A = gen.csr_clustered(1024, 1024, 0.9, seed=440)
    qa, sa = oracle.e4m3_rows(A.vals, A.rowptr)
    plan = e4m3_plan(gb, A, qa, sa)
    for seed, amp in ((441, 1.0), (442, 1e-3)):
        B = gen.dense_normal(A.K, 272, seed) * amp
        qb, tb = oracle.e4m3_rows(B)
        Bv = dev(qb)[:, :256]  # ld = 272
        Cfull = torch.full((A.M, 260), 5.0, device="cuda")
        C = plan.execute(Bv, out=Cfull[:, :256], row_scale=dev(tb)).cpu().numpy()
        eff, _ = effective_values(A.rowptr, A.colidx, A.K, qa, sa, tb, 0)
        ref, sc = oracle.spmm(A.rowptr, A.colidx, eff, oracle.e4m3_decode(qb[:, :256]))
        assert_within(C, ref, sc, TOL32, f"tc e4m3 repeat amp={amp}")
        assert torch.all(Cfull[:, 256:] == 5.0)
    plan.check()


def test_tc_e4m3_argument_errors(gb):
    import torch

    A = gen.csr_clustered(256, 256, 0.9, seed=443)
    qa, sa = oracle.e4m3_rows(A.vals, A.rowptr)
    with pytest.raises(gb.GbspError, match="INVALID_ARG"):
        gb.TcPlan(dev(A.rowptr), dev(A.colidx), dev(qa), A.K)  # no row scales
    plan = e4m3_plan(gb, A, qa, sa)
    qb, tb = oracle.e4m3_rows(gen.dense_normal(A.K, 128, 444))
    with pytest.raises(gb.GbspError, match="INVALID_ARG"):
        plan.execute(dev(qb))  # B without row scales
    with pytest.raises(gb.GbspError, match="UNSUPPORTED"):
        plan.execute(torch.zeros((A.K, 128), dtype=torch.bfloat16, device="cuda"))
    with pytest.raises(gb.GbspError, match="UNSUPPORTED"):
        plan.execute(dev(qb)[:, :120], row_scale=dev(tb))  # N not a multiple of 16


def test_tc_e4m3_full_size_clustered_sampled_windows(gb):
    """The precision configuration in E4M3: 16,384^2 at 90%, clustered, N = 256 — checked
    on 25 sampled 16-row windows (the requantisation is per window row)."""
    A = gen.csr_clustered(16384, 16384, 0.9, seed=2002)
    B = gen.dense_normal(A.K, 256, 2003)
    qa, sa = oracle.e4m3_rows(A.vals, A.rowptr)
    qb, tb = oracle.e4m3_rows(B)
    plan = e4m3_plan(gb, A, qa, sa)
    assert plan.info()["dense_nnz"] >= A.meta["block_nnz"]
    C = plan.execute(dev(qb), row_scale=dev(tb)).cpu().numpy()
    plan.check()
    wins = np.sort(np.random.default_rng(12).choice(A.M // 16, 25, replace=False))
    rows = (wins[:, None] * 16 + np.arange(16)).ravel()
    rp, ci, q, idx = sub_csr(A.rowptr, A.colidx, qa, rows)
    s = sa[rows]
    eff, _ = effective_values(rp, ci, A.K, q, s, tb, 0)
    ref, sc = oracle.spmm(rp, ci, eff, oracle.e4m3_decode(qb))
    assert_within(C[rows], ref, sc, TOL32, "tc e4m3 full size effective operands")
    ref0, sc0 = oracle.spmm(rp, ci, oracle.e4m3_rows_dequant(q, s, rp), oracle.e4m3_rows_dequant(qb, tb))
    assert_within(C[rows], ref0, sc0, TOL_REQUANT, "tc e4m3 full size dequantised inputs")


def test_tc_e4m3_bounded_wait_reports_timeout(gb):
    """The FP8 window kernel's waits are bounded too: a withheld stage ends in
    GBSP_ERR_TIMEOUT, and the next execution is exact."""
    import time

    A = gen.csr_clustered(512, 512, 0.9, seed=445)
    vals = gen.vals_int(A.nnz, 446)
    B = gen.dense_int(A.K, 128, 447)
    plan = e4m3_plan(gb, A, oracle.e4m3_round(vals), np.ones(A.M, np.float32))
    qb, ones = dev(oracle.e4m3_round(B)), dev(np.ones(A.K, np.float32))
    plan.test_withhold(0)
    t0 = time.time()
    plan.execute(qb, row_scale=ones)
    with pytest.raises(gb.GbspError, match="TIMEOUT"):
        plan.check()
    assert time.time() - t0 < 30
    plan.test_withhold(-1)
    C = plan.execute(qb, row_scale=ones).cpu().numpy()
    plan.check()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(C.astype(np.float64), want)
