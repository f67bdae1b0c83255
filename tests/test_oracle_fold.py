"""Pins of the oracle's E4M3 condensed-tile operands (oracle.e4m3_fold), without a GPU.

The fold is the library's reading of how B's per-row scales t_k, which lie along the
contraction of Eq. 1, reach FP8 tensor-core tiles: dense 16 x 8 blocks take a~ = (s_i q) t_k
in FP32, and each row is requantised to E4M3 with a power-of-two scale.  It is pinned by a
hand-worked example whose codes were derived on paper (tests/golden/e4m3_fold_worked.txt:
a boundary row maximum, two ties to even, a block just below the threshold, a second
window), by the identity of unit scales, by the rounding bound of E4M3, by the exact
dequantisation of residual entries and by a brute-force block count.
"""
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "e4m3_fold_worked.txt")


def _golden():
    d = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            d[key] = vals
    return d


def test_fold_worked_example():
    g = _golden()
    rp = np.array(g["rowptr"], np.int32)
    ci = np.array(g["colidx"], np.int32)
    q = np.array([int(x, 16) for x in g["codes_in"]], np.uint8)
    sa = np.array(g["row_scale"], np.float32)
    tb = np.array(g["b_scale"], np.float32)
    codes, dense, eff, exps = oracle.e4m3_fold(rp, ci, int(g["K"][0]), q, sa, tb, int(g["threshold"][0]))
    assert [f"{c:02X}" for c in codes] == [c.upper() for c in g["codes_out"]]
    assert dense.astype(int).tolist() == [int(x) for x in g["dense"]]
    assert eff.tolist() == [float(x) for x in g["eff"]]
    assert exps.tolist() == [int(x) for x in g["exp"]]
    # the input values decode as the fixture states (checks the fixture's own codes)
    assert oracle.e4m3_decode(q).tolist() == [1.0, -6.0, 448.0, 2.0, 0.875, -3.25, 1.0, 0.5, -1.75]


def _random_codes(n, seed):
    q = np.random.default_rng(seed).integers(0, 256, n).astype(np.uint8)
    return np.where((q & 0x7F) == 0x7F, q ^ 0x01, q).astype(np.uint8)  # no NaN codes


@pytest.mark.parametrize("threshold", [0, 1, 12])
def test_fold_unit_scales_keep_values(threshold):
    """s = t = 1: a~ is an E4M3 value and u a power of two no smaller than needed, so the
    requantisation is exact and every entry keeps its value; a row whose maximum is 448
    (code 0x7E) keeps e = 0 and its codes bit for bit."""
    A = gen.csr_clustered(256, 256, 0.9, seed=91)
    q = _random_codes(A.nnz, 92)
    ones_m, ones_k = np.ones(A.M, np.float32), np.ones(A.K, np.float32)
    codes, dense, eff, exps = oracle.e4m3_fold(A.rowptr, A.colidx, A.K, q, ones_m, ones_k, threshold)
    assert np.array_equal(eff, oracle.e4m3_decode(q))
    assert dense.any() and (threshold == 1) == dense.all()
    q2 = q.copy()
    rows = np.repeat(np.arange(A.M), np.diff(A.rowptr))
    first = A.rowptr[:-1][np.diff(A.rowptr) > 0]
    q2[first[dense[first]]] = 0x7E
    codes2, dense2, eff2, exps2 = oracle.e4m3_fold(A.rowptr, A.colidx, A.K, q2, ones_m, ones_k, threshold)
    full = np.isin(rows, rows[first[dense[first]]])
    assert np.all(exps2[rows[first[dense[first]]]] == 0)
    assert np.array_equal(codes2[full], q2[full])


def test_fold_rounding_bound_and_scale_choice():
    """Random scales: every dense entry is within one E4M3 rounding of s q t (relative 2^-4
    in the normal range, half the subnormal step 2^-9 u below it, plus the two FP32
    roundings of the fold), |u q'| <= 448 u, and u is the smallest power of two that holds
    the row's largest |a~| (so that value lies above 224 u)."""
    A = gen.csr_clustered(512, 512, 0.9, seed=93)
    rng = np.random.default_rng(94)
    q = _random_codes(A.nnz, 95)
    sa = np.exp(rng.uniform(-20, 20, A.M)).astype(np.float32)
    tb = np.exp(rng.uniform(-20, 20, A.K)).astype(np.float32)
    codes, dense, eff, exps = oracle.e4m3_fold(A.rowptr, A.colidx, A.K, q, sa, tb, 0)
    rows = np.repeat(np.arange(A.M), np.diff(A.rowptr))
    exact = sa[rows].astype(np.float64) * oracle.e4m3_decode(q) * tb[A.colidx].astype(np.float64)
    u = np.ldexp(1.0, exps[rows])
    d = dense
    assert d.sum() > 1000
    err = np.abs(eff[d] - exact[d])
    small = np.abs(exact[d]) < u[d] * 2.0 ** -6
    bound = np.where(small, u[d] * 2.0 ** -10, np.abs(exact[d]) * 2.0 ** -4) + np.abs(exact[d]) * 2.0 ** -22
    assert np.all(err <= bound)
    assert np.all(np.abs(eff[d]) <= 448 * u[d])
    for i in np.unique(rows[d]):
        sel = d & (rows == i)
        amax = np.abs(exact[sel]).max()
        assert amax <= 448 * 2.0 ** exps[i] * (1 + 2.0 ** -22)
        assert exps[i] == -126 or amax > 224 * 2.0 ** exps[i] * (1 - 2.0 ** -22)
    # residual entries are the dequantised product, exact in FP64
    assert np.array_equal(eff[~d], exact[~d])
    assert np.array_equal(codes[~d], q[~d])


def test_fold_dense_blocks_by_brute_force_count():
    """An entry is dense exactly when its aligned 16-row x 8-column block holds at least
    `threshold` stored entries (10 by default), counted here entry by entry."""
    lengths = np.random.default_rng(96).integers(0, 9, 100)
    A = gen.csr_from_lengths(lengths, 40, seed=97)
    q = _random_codes(A.nnz, 98)
    rows = np.repeat(np.arange(A.M), lengths)
    for thr in (0, 2, 5, 10, 11):
        counts = {}
        for i, k in zip(rows, A.colidx):
            counts[(i // 16, k // 8)] = counts.get((i // 16, k // 8), 0) + 1
        want = [counts[(i // 16, k // 8)] >= (thr if thr >= 1 else 10) for i, k in zip(rows, A.colidx)]
        _, dense, _, _ = oracle.e4m3_fold(A.rowptr, A.colidx, A.K, q, np.ones(A.M, np.float32),
                                          np.ones(A.K, np.float32), thr)
        assert dense.tolist() == want
