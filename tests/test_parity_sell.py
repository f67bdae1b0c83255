"""GPU parity of the SELL-C-sigma SpMM plan (Eq. 1 through sliced, padded, column-major
storage with rows sorted by length within windows of sigma rows).

Integer inputs must match the FP64 oracle bit for bit (every partial sum is exact), random
FP32 inputs within 1e-5 of sum |a||b|; the plan's slot count is checked against the
padding computed on the host from the same sort.
"""
import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev

pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


def mixed_lengths(M, seed):
    rng = np.random.default_rng(seed)
    kind = rng.random(M)
    lengths = rng.integers(1, 12, M)
    lengths[kind < 0.2] = 0
    lengths[kind > 0.97] = rng.integers(40, 400, M)[kind > 0.97]
    return lengths.astype(np.int64)


def rows_per_block(N):
    """Rows a 256-thread block takes: 8 warps x (32 / lanes per row), with the library's
    lane layout of N FP32 columns (2 vectors per lane from 16 vectors on, lanes the power of
    two covering the row, at most 32)."""
    nvec = N // 4
    vpl = 2 if nvec >= 16 else 1
    lpn = min(32, 1 << int(np.ceil(np.log2(-(-nvec // vpl)))))
    return 8 * (32 // lpn)


def expected_slots(lengths, C, sigma):
    M = len(lengths)
    sigma = M if sigma <= 0 or sigma > M else sigma
    order = np.concatenate([w0 + np.argsort(-lengths[w0:w0 + sigma], kind="stable") for w0 in range(0, M, sigma)])
    L = lengths[order]
    return sum(int(L[s:s + C].max()) * C for s in range(0, M, C))


@pytest.mark.parametrize("C,sigma", [(64, 0), (64, 256), (128, 0), (256, 512), (32, 64)])
@pytest.mark.parametrize("N", [16, 64, 128, 200])
def test_sell_integers_bit_exact(gb, C, sigma, N):
    lengths = mixed_lengths(3001, C + N)
    A = gen.csr_from_lengths(lengths, 2500, seed=701)
    vals = gen.vals_int(A.nnz, 702)
    B = gen.dense_int(A.K, N, 703)
    plan = gb.SellPlan(dev(A.rowptr), dev(A.colidx), dev(vals), A.K, C=C, sigma=sigma)
    info = plan.info()
    assert info["slots"] == expected_slots(lengths, C, sigma) and info["nnz"] == A.nnz
    if C % rows_per_block(N):
        with pytest.raises(gb.GbspError, match="UNSUPPORTED"):
            plan.execute(dev(B))
        return
    Cout = plan.execute(dev(B)).cpu().numpy()
    want, _ = oracle.spmm(A.rowptr, A.colidx, vals, B)
    assert np.array_equal(Cout.astype(np.float64), want)


@pytest.mark.parametrize("make", [lambda: gen.csr_powerlaw(8000, 8000, 0.995, seed=704),
                                  lambda: gen.csr_uniform(10000, 9000, 0.999, seed=705)])
def test_sell_random_fp32(gb, make):
    A = make()
    B = gen.dense_normal(A.K, 64, 706)
    plan = gb.SellPlan(dev(A.rowptr), dev(A.colidx), dev(A.vals), A.K)
    C = plan.execute(dev(B)).cpu().numpy()
    ref, sc = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref, sc, TOL32, "sell fp32")


def test_sell_unsorted_repeated_padded_ld_and_errors(gb):
    import torch

    rp = np.array([0, 3, 3, 7, 8], np.int32)
    ci = np.array([5, 1, 5, 0, 0, 7, 2, 3], np.int32)  # unsorted, a repeated column
    vals = gen.vals_int(8, 707)
    B = gen.dense_int(8, 16, 708)
    plan = gb.SellPlan(dev(rp), dev(ci), dev(vals), 8, C=64)
    Bp = torch.zeros((8, 24), device="cuda")
    Bp[:, :16] = dev(B)
    Cp = torch.full((4, 20), 3.0, device="cuda")
    plan.execute(Bp[:, :16], out=Cp[:, :16])
    want, _ = oracle.spmm(rp, ci, vals, B)
    assert np.array_equal(Cp[:, :16].cpu().numpy().astype(np.float64), want)
    assert torch.all(Cp[:, 16:] == 3.0)
    with pytest.raises(gb.GbspError, match="ALIGN"):
        plan.execute(dev(gen.dense_int(8, 18, 709)))
    with pytest.raises(gb.GbspError, match="INVALID_ARG"):
        gb.SellPlan(dev(rp), dev(ci), dev(vals), 8, C=12)
    bad = np.array([0, 3, 3, 7, 8], np.int32)
    with pytest.raises(gb.GbspError, match="INVALID_CSR"):
        gb.SellPlan(dev(bad), dev(np.array([5, 1, 5, 0, 0, 9, 2, 3], np.int32)), dev(vals), 8)


def test_sell_empty_matrix(gb):
    import torch

    z = torch.zeros(5, dtype=torch.int32, device="cuda")
    plan = gb.SellPlan(z, z[:0], torch.zeros(0, device="cuda"), 7)
    C = plan.execute(torch.ones((7, 16), device="cuda")).cpu().numpy()
    assert np.all(C == 0) and plan.info()["slots"] == 0
