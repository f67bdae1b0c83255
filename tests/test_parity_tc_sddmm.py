"""GPU parity of the condensed-tile SDDMM on a tensor-core plan's pattern (Eq. 2).

out[p] = s_p <X_i, Y_j> for every stored entry, in the matrix's CSR order: residual entries
through the row-split CSR kernel at their own positions, the dense 16 x 8 blocks from
tcgen05 products of the blocks' Y rows with the window's X rows.  BF16 and E4M3 operands
are exact in the products (FP32 accumulation), so random inputs are held to the FP32
tolerance against the FP64 oracle on the dequantised operands, and integer inputs must
match bit for bit.
"""
import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev, sub_csr

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


def bf16(x):
    import torch

    return dev(oracle.bf16_round(x).view(np.int16)).view(torch.bfloat16)


def bf16_plan(gb, A, threshold=0):
    return gb.TcPlan(dev(A.rowptr), dev(A.colidx), bf16(A.vals), A.K, threshold)


@pytest.mark.parametrize("tiles", [1, 0, -1])
@pytest.mark.parametrize("threshold", [0, 1, 129])
@pytest.mark.parametrize("Kd", [64, 128, 256, 512])
def test_tc_sddmm_bf16_integers_bit_exact(gb, tiles, threshold, Kd):
    A = gen.csr_clustered(1024, 1024, 0.9, seed=451)
    svals = gen.vals_int(A.nnz, 452)
    X, Y = gen.dense_int(A.M, Kd, 453, -4, 4), gen.dense_int(A.K, Kd, 454, -4, 4)
    plan = bf16_plan(gb, A, threshold)
    assert (plan.info()["dense_windows"] == 0) == (threshold == 129)
    out = plan.sddmm(dev(svals), bf16(X), bf16(Y), tiles=tiles).cpu().numpy()
    plan.check()
    want, _ = oracle.sddmm(A.rowptr, A.colidx, svals, X, Y)
    assert np.array_equal(out.astype(np.float64), want)


@pytest.mark.parametrize("threshold", [0, 1])
@pytest.mark.parametrize("Kd", [128, 256, 512])
def test_tc_sddmm_e4m3_integers_bit_exact(gb, threshold, Kd):
    """Integers in [-8, 8] with unit row scales are exact in E4M3."""
    A = gen.csr_clustered(1024, 1024, 0.9, seed=455)
    svals = gen.vals_int(A.nnz, 456)
    X, Y = gen.dense_int(A.M, Kd, 457), gen.dense_int(A.K, Kd, 458)
    plan = bf16_plan(gb, A, threshold)
    out = plan.sddmm(dev(svals), dev(oracle.e4m3_round(X)), dev(oracle.e4m3_round(Y)),
                     x_scale=dev(np.ones(A.M, np.float32)), y_scale=dev(np.ones(A.K, np.float32)),
                     tiles=1).cpu().numpy()
    plan.check()
    want, _ = oracle.sddmm(A.rowptr, A.colidx, svals, X, Y)
    assert np.array_equal(out.astype(np.float64), want)


@pytest.mark.parametrize("shape", [(2000, 2003, 256), (1001, 64, 64), (64, 4096, 128), (700, 900, 192)])
def test_tc_sddmm_ragged_shapes(gb, shape):
    """M not a multiple of 16 (X rows past M read as zeros), K not a multiple of 8."""
    M, K, Kd = shape
    lengths = np.random.default_rng(459).integers(0, min(K, 300), M)
    A = gen.csr_from_lengths(lengths, K, seed=460)
    svals = gen.vals_int(A.nnz, 461)
    X, Y = gen.dense_int(M, Kd, 462, -4, 4), gen.dense_int(K, Kd, 463, -4, 4)
    plan = bf16_plan(gb, A, threshold=2)
    assert plan.info()["dense_windows"] > 0
    out = plan.sddmm(dev(svals), bf16(X), bf16(Y), tiles=1).cpu().numpy()
    plan.check()
    want, _ = oracle.sddmm(A.rowptr, A.colidx, svals, X, Y)
    assert np.array_equal(out.astype(np.float64), want)


@pytest.mark.parametrize("dtype", ["bf16", "e4m3"])
@pytest.mark.parametrize("threshold", [0, 1])
def test_tc_sddmm_random_values(gb, dtype, threshold):
    A = gen.csr_clustered(2048, 2048, 0.9, seed=464)
    Kd = 256
    X, Y = gen.dense_normal(A.M, Kd, 465), gen.dense_normal(A.K, Kd, 466) * 2.0
    plan = bf16_plan(gb, A, threshold)
    if dtype == "bf16":
        out = plan.sddmm(dev(A.vals), bf16(X), bf16(Y), tiles=1).cpu().numpy()
        dx, dy = oracle.bf16_decode(oracle.bf16_round(X)), oracle.bf16_decode(oracle.bf16_round(Y))
    else:
        qx, u = oracle.e4m3_rows(X)
        qy, v = oracle.e4m3_rows(Y)
        out = plan.sddmm(dev(A.vals), dev(qx), dev(qy), x_scale=dev(u), y_scale=dev(v), tiles=1).cpu().numpy()
        dx, dy = oracle.e4m3_rows_dequant(qx, u), oracle.e4m3_rows_dequant(qy, v)
    plan.check()
    ref, sc = oracle.sddmm(A.rowptr, A.colidx, A.vals, dx, dy)
    assert_within(out, ref, sc, TOL32, f"tc sddmm {dtype}")


def test_tc_sddmm_padded_ld_and_repeat(gb):
    """Leading dimensions above Kd; a second execution with other inputs."""
    A = gen.csr_clustered(1024, 1024, 0.9, seed=467)
    plan = bf16_plan(gb, A)
    for seed in (468, 469):
        X = gen.dense_int(A.M, 136, seed, -4, 4)
        Y = gen.dense_int(A.K, 136, seed + 1, -4, 4)
        svals = gen.vals_int(A.nnz, seed + 2)
        out = plan.sddmm(dev(svals), bf16(X)[:, :128], bf16(Y)[:, :128], tiles=1).cpu().numpy()
        want, _ = oracle.sddmm(A.rowptr, A.colidx, svals, X[:, :128], Y[:, :128])
        assert np.array_equal(out.astype(np.float64), want)
    plan.check()


def test_tc_sddmm_argument_errors(gb):
    import torch

    A = gen.csr_clustered(256, 256, 0.9, seed=470)
    plan = bf16_plan(gb, A)
    s = dev(A.vals)
    with pytest.raises(gb.GbspError, match="UNSUPPORTED"):  # FP32 X / Y
        plan.sddmm(s, dev(gen.dense_normal(A.M, 64, 1)), dev(gen.dense_normal(A.K, 64, 2)))
    with pytest.raises(gb.GbspError, match="UNSUPPORTED"):  # Kd = 32 on the tiles
        plan.sddmm(s, bf16(gen.dense_normal(A.M, 32, 1)), bf16(gen.dense_normal(A.K, 32, 2)), tiles=1)
    with pytest.raises(gb.GbspError, match="INVALID_ARG"):  # E4M3 without row scales
        plan.sddmm(s, torch.zeros((A.M, 128), dtype=torch.uint8, device="cuda"),
                   torch.zeros((A.K, 128), dtype=torch.uint8, device="cuda"))
    with pytest.raises(gb.GbspError, match="INVALID_ARG"):  # shape
        plan.sddmm(s, bf16(gen.dense_normal(A.M + 1, 64, 1)), bf16(gen.dense_normal(A.K, 64, 2)))


def test_tc_sddmm_full_size_clustered_sampled_rows(gb):
    """The precision configuration: 16,384^2 at 90% clustered, Kd = 256, BF16 — 400 sampled
    rows against the oracle."""
    A = gen.csr_clustered(16384, 16384, 0.9, seed=2002)
    X, Y = gen.dense_normal(A.M, 256, 2004), gen.dense_normal(A.K, 256, 2005)
    plan = bf16_plan(gb, A)
    out = plan.sddmm(dev(A.vals), bf16(X), bf16(Y)).cpu().numpy()
    plan.check()
    rows = np.sort(np.random.default_rng(13).choice(A.M, 400, replace=False))
    rp, ci, v, idx = sub_csr(A.rowptr, A.colidx, A.vals, rows)
    dx, dy = oracle.bf16_decode(oracle.bf16_round(X)), oracle.bf16_decode(oracle.bf16_round(Y))
    ref, sc = oracle.sddmm(rp, ci, v, dx[rows], dy)
    assert_within(out[idx], ref, sc, TOL32, "tc sddmm full size")


def test_tc_sddmm_auto_choice(gb):
    """tiles=-1 takes the tiles when dense blocks average at least 24 entries (clustered: 51
    per block) and the CSR kernels otherwise (uniform at 90%: about 16); both give the
    oracle's integers exactly."""
    cases = [(gen.csr_clustered(1024, 1024, 0.9, seed=471), 2), (gen.csr_uniform(1024, 1024, 0.9, seed=472), 1)]
    for A, launches in cases:
        plan = bf16_plan(gb, A)
        info = plan.info()
        assert (info["dense_nnz"] >= 24 * info["dense_blocks"]) == (launches == 2)
        svals = gen.vals_int(A.nnz, 473)
        X, Y = gen.dense_int(A.M, 64, 474, -4, 4), gen.dense_int(A.K, 64, 475, -4, 4)
        x, y, sv = bf16(X), bf16(Y), dev(svals)
        l0 = gb.launch_count()
        out = plan.sddmm(sv, x, y).cpu().numpy()
        assert gb.launch_count() - l0 == launches  # residual + tiles, or one CSR launch
        plan.check()
        want, _ = oracle.sddmm(A.rowptr, A.colidx, svals, X, Y)
        assert np.array_equal(out.astype(np.float64), want)
