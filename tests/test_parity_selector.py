"""GPU parity of the selection kernels: features, feature standardisation, MLP inference and
MLP training (Adam) against the FP64 selector oracle, and the autotuner's bookkeeping."""
import numpy as np
import pytest

import gen
import oracle
from _util import dev
from oracle import selector as osel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_2604_27985_gb300 as g

    return g


MATS = [
    lambda: gen.csr_uniform(3000, 2500, 0.99, seed=601),
    lambda: gen.csr_powerlaw(5000, 5000, 0.995, seed=602),
    lambda: gen.csr_banded(4096, 4096, 0.99, seed=603, band_frac=0.02),
    lambda: gen.csr_blocked(4096, 4096, 0.99, seed=604, b=16),
    lambda: gen.csr_clustered(2048, 2048, 0.9, seed=605),
    lambda: gen.csr_from_lengths(np.r_[np.zeros(10, np.int64), np.full(90, 7)], 300, seed=606),
]


@pytest.mark.parametrize("k", range(len(MATS)))
@pytest.mark.parametrize("N,dtype", [(64, 0), (256, 1)])
def test_features(gb, k, N, dtype):
    A = MATS[k]()
    f = gb.features(dev(A.rowptr), dev(A.colidx), A.K, N, dtype).cpu().numpy()
    want = osel.features(A.rowptr, A.colidx, A.M, A.K, N, dtype).astype(np.float32)
    np.testing.assert_allclose(f, want, rtol=3e-7, atol=0)


def test_feature_norm_and_predict(gb):
    rng = np.random.default_rng(607)
    feats = (rng.standard_normal((300, 16)) * rng.uniform(0.5, 4, 16) + rng.uniform(-3, 3, 16)).astype(np.float32)
    feats[:, 15] = 1.0  # a constant feature gets standard deviation 1
    norm = gb.feature_norm(dev(feats)).cpu().numpy()
    np.testing.assert_allclose(norm, osel.feature_norm(feats), rtol=1e-5, atol=1e-6)
    w = (rng.standard_normal(osel.N_PARAMS) * 0.2).astype(np.float32)
    out, choice = gb.mlp_predict(dev(w), dev(norm), dev(feats))
    y, _ = osel.forward(w.astype(np.float64), osel.standardise(feats, norm))
    np.testing.assert_allclose(out.cpu().numpy(), y, rtol=1e-4, atol=1e-4)
    c = choice.cpu().numpy()
    # the chosen output is the smallest (ties broken towards the lower index)
    o = out.cpu().numpy()
    assert np.array_equal(c, np.argmin(o, axis=1))


def test_mlp_train_steps(gb):
    rng = np.random.default_rng(608)
    n = 200
    feats = rng.standard_normal((n, 16)).astype(np.float32)
    targets = np.abs(rng.standard_normal((n, 24))).astype(np.float32)
    mask = (rng.random((n, 24)) > 0.1).astype(np.float32)
    w0 = (rng.standard_normal(osel.N_PARAMS) * 0.15).astype(np.float32)
    norm = osel.feature_norm(feats).astype(np.float32)
    order = rng.permutation(n).astype(np.int32)
    import torch

    W = dev(w0)
    adam = torch.zeros(2 * osel.N_PARAMS, device="cuda")
    gb.mlp_train(W, adam, dev(norm), dev(feats), dev(targets), dev(mask), dev(order), steps=4, batch=48, lr=1e-3)
    w_o, adam_o = osel.train(w0, np.zeros(2 * osel.N_PARAMS), norm, feats, targets, mask, order, 4, 48, 1e-3)
    np.testing.assert_allclose(W.cpu().numpy(), w_o, rtol=0, atol=2e-6)
    np.testing.assert_allclose(adam.cpu().numpy()[:osel.N_PARAMS], adam_o[:osel.N_PARAMS], rtol=1e-3, atol=1e-7)
    # resuming from step 4 continues the same trajectory
    rolled = np.roll(order, -((4 * 48) % n))
    gb.mlp_train(W, adam, dev(norm), dev(feats), dev(targets), dev(mask), dev(rolled), steps=2, batch=48, lr=1e-3,
                 t0=4)
    w_o2, _ = osel.train(w_o, adam_o, norm, feats, targets, mask, rolled, 2, 48, 1e-3, t0=4)
    np.testing.assert_allclose(W.cpu().numpy(), w_o2, rtol=0, atol=4e-6)


def test_mlp_training_reduces_loss(gb):
    """Many steps on a learnable target (a fixed random MLP's outputs) lower the loss."""
    import torch

    rng = np.random.default_rng(609)
    n = 512
    feats = rng.standard_normal((n, 16)).astype(np.float32)
    teacher = (rng.standard_normal(osel.N_PARAMS) * 0.3)
    norm = osel.feature_norm(feats)
    targets = osel.forward(teacher, osel.standardise(feats, norm))[0].astype(np.float32)
    mask = np.ones((n, 24), np.float32)
    W = dev((rng.standard_normal(osel.N_PARAMS) * 0.1).astype(np.float32))
    adam = torch.zeros(2 * osel.N_PARAMS, device="cuda")
    order = dev(rng.permutation(n).astype(np.int32))
    normd = dev(norm.astype(np.float32))
    l0 = osel.loss(W.cpu().numpy().astype(np.float64), osel.standardise(feats, norm), targets, mask)
    gb.mlp_train(W, adam, normd, dev(feats), dev(targets), dev(mask), order, steps=800, batch=64, lr=3e-3)
    l1 = osel.loss(W.cpu().numpy().astype(np.float64), osel.standardise(feats, norm), targets, mask)
    assert l1 < 0.2 * l0


def test_autotune_bookkeeping(gb):
    import torch

    A = gen.csr_powerlaw(4000, 3000, 0.99, seed=610)
    B = gen.dense_normal(A.K, 64, 611)
    C = torch.empty((A.M, 64), device="cuda")
    times, best = gb.autotune(dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B), C, reps=2)
    assert len(times) == 24 and all(np.isfinite(times)) and all(t > 0 for t in times)
    assert best == int(np.argmin(times))
    ref, sc = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    from _util import assert_within

    assert_within(C.cpu().numpy(), ref, sc, 1e-5, "last autotuned variant")
    for v in (0, 9, 18, 22, 23):
        kw = gb.variant_options(v)
        out = gb.spmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B), **kw).cpu().numpy()
        assert_within(out, ref, sc, 1e-5, f"variant {v}")
