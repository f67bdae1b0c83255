"""GPU parity of the grouped SpMM / SDDMM over many problems of uneven size (one persistent
launch replayed from a CUDA graph), FP32 and BF16 dense operands."""
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


def _problems(seed, G=9):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(G):
        M, K = int(rng.integers(1, 3000)), int(rng.integers(1, 2500))
        kind = k % 3
        A = (gen.csr_uniform(M, K, 0.98, seed=seed + k) if kind == 0 else
             gen.csr_powerlaw(M, K, 0.97, seed=seed + k) if kind == 1 else
             gen.csr_from_lengths(np.r_[np.zeros(M // 3, np.int64), rng.integers(0, min(40, K) + 1, M - M // 3)], K,
                                  seed=seed + k))
        out.append(A)
    return out


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_spmm_batched(gb, dtype):
    import torch

    mats = _problems(801)
    widths = [8, 16, 32, 64, 96, 128, 200, 256, 24]
    probs, host = [], []
    for A, N in zip(mats, widths):
        B = gen.dense_normal(A.K, N, 802 + N)
        if dtype == "bf16":
            vb, Bb = oracle.bf16_round(A.vals), oracle.bf16_round(B)
            v = dev(vb.view(np.int16)).view(torch.bfloat16)
            Bd = dev(Bb.view(np.int16)).view(torch.bfloat16)
            host.append((A, oracle.bf16_decode(vb), oracle.bf16_decode(Bb)))
        else:
            v, Bd = dev(A.vals), dev(B)
            host.append((A, A.vals, B))
        probs.append((dev(A.rowptr), dev(A.colidx), v, Bd, torch.full((A.M, N), np.nan, device="cuda")))
    plan = gb.BatchPlan(probs)
    plan.execute()
    plan.execute()  # replay
    torch.cuda.synchronize()
    for (A, va, Bh), pr in zip(host, probs):
        ref, sc = oracle.spmm(A.rowptr, A.colidx, va, Bh)
        assert_within(pr[4].cpu().numpy(), ref, sc, 1e-5, f"batched spmm {dtype} {A.M}x{A.K}")


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_sddmm_batched(gb, dtype):
    import torch

    mats = _problems(811)
    widths = [4, 8, 16, 32, 64, 128, 256, 40, 8] if dtype == "f32" else [8, 16, 32, 64, 128, 256, 512, 48, 8]
    probs, host = [], []
    for A, Kd in zip(mats, widths):
        X, Y = gen.dense_normal(A.M, Kd, 812 + Kd), gen.dense_normal(A.K, Kd, 813 + Kd)
        if dtype == "bf16":
            xb, yb = oracle.bf16_round(X), oracle.bf16_round(Y)
            Xd = dev(xb.view(np.int16)).view(torch.bfloat16)
            Yd = dev(yb.view(np.int16)).view(torch.bfloat16)
            host.append((A, oracle.bf16_decode(xb), oracle.bf16_decode(yb)))
        else:
            Xd, Yd = dev(X), dev(Y)
            host.append((A, X, Y))
        probs.append((dev(A.rowptr), dev(A.colidx), dev(A.vals), Xd, Yd,
                      torch.full((max(A.nnz, 1),), np.nan, device="cuda")))
    gb.sddmm_csr_batched(probs)
    for (A, Xh, Yh), pr in zip(host, probs):
        ref, sc = oracle.sddmm(A.rowptr, A.colidx, A.vals, Xh, Yh)
        assert_within(pr[5].cpu().numpy()[:A.nnz], ref, sc, 1e-5, f"batched sddmm {dtype} {A.M}x{A.K}")


def test_batched_integers_bit_exact(gb):
    import torch

    mats = _problems(821, G=5)
    probs, host = [], []
    for k, A in enumerate(mats):
        vals = gen.vals_int(A.nnz, 822 + k)
        B = gen.dense_int(A.K, 64, 823 + k)
        probs.append((dev(A.rowptr), dev(A.colidx), dev(vals), dev(B), torch.empty((A.M, 64), device="cuda")))
        host.append((A, vals, B))
    gb.spmm_csr_batched(probs)
    for (A, vals, B), pr in zip(host, probs):
        assert np.array_equal(pr[4].cpu().numpy().astype(np.float64), oracle.spmm(A.rowptr, A.colidx, vals, B)[0])
