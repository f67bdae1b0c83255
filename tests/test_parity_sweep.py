"""The scale / sparsity sweep at its full sizes (FP32): 65,536^2 at 90% and 99% and
1,048,576^2 at 99.99%, uniform and power-law rows, SpMM N in {32, 64, 128} and SDDMM Kd in
{32, 128}, in the launch configurations the library picks by default and the merge path.
Each case checks a sample of whole rows against the FP64 oracle (|err| <= 1e-5 * scale)."""
import numpy as np
import pytest

import gen
import oracle
from _util import assert_within, dev, sub_csr

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
TOL = 1e-5


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


_mats = {}


def mat(key):
    if key not in _mats:
        _mats.clear()  # one large matrix at a time
        n, s, kind, seed = key
        _mats[key] = (gen.csr_uniform(n, n, s, seed=seed) if kind == "uniform"
                      else gen.csr_powerlaw(n, n, s, seed=seed))
    return _mats[key]


CASES = [
    ((65536, 0.99, "powerlaw", 1101), 32, 32),
    ((65536, 0.99, "powerlaw", 1101), 128, 128),
    ((1048576, 0.9999, "uniform", 1102), 128, 128),
    ((1048576, 0.9999, "powerlaw", 1103), 64, 32),
    ((65536, 0.9, "uniform", 1104), 64, 32),
    ((65536, 0.9, "powerlaw", 1105), 32, 128),
]


def _rows(A, k, seed):
    lens = A.row_lengths()
    r = np.random.default_rng(seed).choice(A.M, k, replace=False)
    r = np.concatenate([r, [int(np.argmax(lens)), 0, A.M - 1]])  # include the longest row
    return np.unique(r)


@pytest.mark.parametrize("key,N,Kd", CASES, ids=[f"{c[0][0]}-{c[0][1]}-{c[0][2]}-N{c[1]}-Kd{c[2]}" for c in CASES])
def test_sweep_cell(gb, key, N, Kd):
    A = mat(key)
    assert A.nnz == gen.nnz_for(key[0], key[0], key[1])
    rp, ci, v = dev(A.rowptr), dev(A.colidx), dev(A.vals)
    B = gen.dense_normal(A.K, N, key[3] + 1)
    rows = _rows(A, 200, key[3] + 2)
    srp, sci, sv, idx = sub_csr(A.rowptr, A.colidx, A.vals, rows)
    ref, sc = oracle.spmm(srp, sci, sv, B)
    Bd = dev(B)
    for variant in ("auto", "merge"):
        C = gb.spmm(rp, ci, v, Bd, variant=variant)
        assert_within(C[dev(rows.astype(np.int64))].cpu().numpy(), ref, sc, TOL, f"spmm {variant}")
        del C
    X, Y = gen.dense_normal(A.M, Kd, key[3] + 3), gen.dense_normal(A.K, Kd, key[3] + 4)
    ref, sc = oracle.sddmm(srp, sci, sv, X[rows], Y)
    for variant in ("auto", "merge"):
        out = gb.sddmm(rp, ci, v, dev(X), dev(Y), variant=variant)
        assert_within(out[dev(idx.astype(np.int64))].cpu().numpy(), ref, sc, TOL, f"sddmm {variant}")
