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

    assert_within(C.cpu().numpy(), ref, sc, 1e-5, "last autotuned variant (the hyper-sparse plan)")
    for v in (0, 9, 18, 22):
        kw = gb.variant_options(v)
        out = gb.spmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B), **kw).cpu().numpy()
        assert_within(out, ref, sc, 1e-5, f"variant {v}")
    assert gb.variant_options(22)["variant"] == "rowgroup" and gb.variant_options(23) == {"variant": "hsp_plan"}
    assert gb.variant_options(21) == {"variant": "sell_plan"}
    # BF16: the SELL-C-sigma and hyper-sparse plans (FP32 only) do not apply
    times16, best16 = gb.autotune(dev(A.rowptr), dev(A.colidx), gb.quantize_bf16(dev(A.vals)),
                                  gb.quantize_bf16(dev(B)), C, reps=1)
    assert np.isinf(times16[21]) and np.isinf(times16[23]) and best16 == int(np.argmin(times16))
    assert all(np.isfinite(np.delete(times16, [21, 23])))


def test_autotune_sddmm_bookkeeping(gb):
    import torch

    A = gen.csr_powerlaw(4000, 3000, 0.99, seed=612)
    X, Y = gen.dense_normal(A.M, 64, 613), gen.dense_normal(A.K, 64, 614)
    out = torch.empty(A.nnz, device="cuda")
    times, best = gb.autotune_sddmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(X), dev(Y), out, reps=2)
    assert len(times) == 24 and all(np.isfinite(times[:9])) and all(np.isinf(times[9:]))
    assert best == int(np.argmin(times))
    ref, sc = oracle.sddmm(A.rowptr, A.colidx, A.vals, X, Y)
    from _util import assert_within

    assert_within(out.cpu().numpy(), ref, sc, 1e-5, "last autotuned SDDMM variant")
    for v in range(gb.N_SDDMM_VARIANTS):
        o = gb.sddmm(dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(X), dev(Y),
                     **gb.sddmm_variant_options(v)).cpu().numpy()
        assert_within(o, ref, sc, 1e-5, f"sddmm variant {v}")


def _untrained(op, **kw):
    from paper_2604_27985_gb300 import selector as sel

    s = sel.Selector(seed=3, op=op, **kw)
    rng = np.random.default_rng(615)
    s.norm = dev(np.r_[rng.standard_normal(16), np.ones(16)].astype(np.float32))
    return s


def test_selector_fallback_outside_training_range(gb):
    """A matrix whose features lie outside the training range goes to the autotuner; its
    best is kept per pattern (the second call does not autotune again) and the result is the
    oracle's."""
    from _util import assert_within

    s = _untrained("spmm", margin=0.0, gap=0.0)
    s.fmin, s.fmax = np.full(16, -1e-3), np.full(16, 1e-3)  # nothing real fits
    A = gen.csr_powerlaw(3000, 3000, 0.995, seed=616)
    B = gen.dense_normal(A.K, 64, 617)
    rp, ci, v, Bd = dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B)
    choice, reason = s.decide(rp, ci, A.K, 64, tune=lambda: gb.autotune(rp, ci, v, Bd,
                                                                          gb.spmm(rp, ci, v, Bd))[1])
    assert reason == "range" and 0 <= choice < 24
    ref, sc = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    for _ in range(2):
        C = s.spmm(rp, ci, v, Bd).cpu().numpy()
        assert_within(C, ref, sc, 1e-5, "fallback choice")
    assert s.counts["autotuned"] == 1 and s.counts["range"] == 3


def test_selector_fallback_when_top_two_are_close(gb):
    from _util import assert_within

    s = _untrained("spmm", margin=1e9, gap=1e9)  # every prediction counts as ambiguous
    s.fmin, s.fmax = np.zeros(16), np.ones(16)
    A = gen.csr_uniform(4000, 4000, 0.999, seed=618)
    B = gen.dense_normal(A.K, 32, 619)
    rp, ci, v, Bd = dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B)
    v_sel = s.choose(rp, ci, A.K, 32)
    assert s.counts["gap"] == 1 and s.counts["autotuned"] == 1
    C = s.run_spmm(v_sel, rp, ci, v, Bd, gb.spmm(rp, ci, v, Bd)).cpu().numpy()
    ref, sc = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    assert_within(C, ref, sc, 1e-5, "gap fallback choice")
    # without the fallback the model's own choice stands (over the applicable variants)
    s2 = _untrained("spmm", margin=1e9, gap=0.0)
    s2.fmin, s2.fmax = np.zeros(16), np.ones(16)
    f = gb.features(rp, ci, A.K, 32)
    out, _ = gb.mlp_predict(s2.weights, s2.norm, f.reshape(1, -1))
    assert s2.choose(rp, ci, A.K, 32) == int(np.argmin(out.cpu().numpy()[0]))
    assert s2.counts["autotuned"] == 0


def test_selector_runs_the_plan_variants(gb):
    from _util import assert_within

    s = _untrained("spmm")
    A = gen.csr_uniform(20000, 20000, 0.9999, seed=620)
    B = gen.dense_normal(A.K, 64, 621)
    rp, ci, v, Bd = dev(A.rowptr), dev(A.colidx), dev(A.vals), dev(B)
    ref, sc = oracle.spmm(A.rowptr, A.colidx, A.vals, B)
    for variant in (23, 21):
        for _ in range(2):  # built once, then reused
            C = s.run_spmm(variant, rp, ci, v, Bd, gb.spmm(rp, ci, v, Bd)).cpu().numpy()
            assert_within(C, ref, sc, 1e-5, f"plan variant {variant} through the selector")
    assert len(s._plans) == 2


def test_sddmm_selector_with_fallback(gb):
    from _util import assert_within

    s = _untrained("sddmm", margin=0.0, gap=0.0)
    s.fmin, s.fmax = np.full(16, -1e-3), np.full(16, 1e-3)
    A = gen.csr_powerlaw(3000, 3000, 0.99, seed=622)
    X, Y = gen.dense_normal(A.M, 128, 623), gen.dense_normal(A.K, 128, 624)
    rp, ci, v = dev(A.rowptr), dev(A.colidx), dev(A.vals)
    out = s.sddmm(rp, ci, v, dev(X), dev(Y)).cpu().numpy()
    assert s.counts["range"] == 1 and s.counts["autotuned"] == 1
    ref, sc = oracle.sddmm(A.rowptr, A.colidx, A.vals, X, Y)
    assert_within(out, ref, sc, 1e-5, "sddmm selector")
    # the model alone picks among the 9 SDDMM variants only
    s2 = _untrained("sddmm", margin=1e9, gap=0.0)
    assert 0 <= s2.choose(rp, ci, A.K, 128) < gb.N_SDDMM_VARIANTS
