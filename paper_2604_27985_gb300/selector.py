"""Learned choice of the SpMM (or SDDMM) variant: features -> MLP -> the variant with the
smallest predicted time, trained on the exhaustive autotuner's timings, with the autotuner
itself as the fallback where the model should not be trusted.

Everything numerical runs in the library's kernels (gbsp_features, gbsp_autotune,
gbsp_autotune_sddmm, gbsp_feature_norm, gbsp_mlp_train, gbsp_mlp_predict); this module keeps
the weight tensors, turns timings into targets (log of each variant's time over the best
one, masked where a variant did not run), decides when to fall back, caches the fallback's
result per pattern, and saves / loads a trained model (raw FP32 weights + JSON header).

Fallback (the exhaustive autotuner on the caller's matrix, result kept per pattern):
  * "range": a feature lies outside the training set's range by more than `margin` times
    that range (a matrix unlike any the model was trained on, e.g. more rows);
  * "gap": the two smallest predicted log-times differ by less than `gap` (the model cannot
    tell the top two apart; its typical error is larger than that).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

from . import ops
from ._lib import BF16, F32

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_MODEL = os.path.join(HERE, "selector_gb300")
DEFAULT_SDDMM_MODEL = os.path.join(HERE, "selector_sddmm_gb300")


def targets_from_times(times):
    """(targets, mask): log(t_v / t_best) per variant; mask 0 where a variant did not run."""
    t = np.asarray(times, dtype=np.float64)
    ok = np.isfinite(t) & (t > 0)
    best = t[ok].min(axis=-1, keepdims=True) if t.ndim == 1 else np.where(ok, t, np.inf).min(axis=-1, keepdims=True)
    tgt = np.where(ok, np.log(np.where(ok, t, 1.0) / best), 0.0)
    return tgt.astype(np.float32), ok.astype(np.float32)


def regret(times, choices):
    """t_chosen / t_best - 1 per matrix (times n x 24, choices n)."""
    t = np.asarray(times, dtype=np.float64)
    best = np.where(np.isfinite(t), t, np.inf).min(axis=1)
    chosen = t[np.arange(len(t)), np.asarray(choices)]
    return chosen / best - 1.0


def label(rowptr, colidx, vals, ncols, N, dtype, reps=3, stream=None, op="spmm"):
    """Features (device float32[16]) and the 24 variant times (ms) of one matrix, with
    zero-filled dense operands of width N in the given dtype (SpMM: B; SDDMM: X and Y)."""
    dev = rowptr.device
    dt = torch.bfloat16 if dtype == BF16 else torch.float32
    M = rowptr.numel() - 1
    feats = ops.features(rowptr, colidx, ncols, N, dtype, stream=stream)
    if op == "sddmm":
        X = torch.zeros((M, N), dtype=dt, device=dev)
        Y = torch.zeros((ncols, N), dtype=dt, device=dev)
        out = torch.empty(colidx.numel(), dtype=torch.float32, device=dev)
        times, _ = ops.autotune_sddmm(rowptr, colidx, vals, X, Y, out, reps=reps, stream=stream)
    else:
        B = torch.zeros((ncols, N), dtype=dt, device=dev)
        C = torch.empty((M, N), dtype=torch.float32, device=dev)
        v = ops.quantize_bf16(vals) if dtype == BF16 else vals
        times, _ = ops.autotune(rowptr, colidx, v, B, C, reps=reps, stream=stream)
    return feats, times


def applicable(op, dtype):
    """Variant indices the model may choose for this op and dtype: SDDMM has 9; the SELL-C-
    sigma and hyper-sparse plans (SpMM variants 21 and 23) take FP32 only."""
    if op == "sddmm":
        return np.arange(ops.N_SDDMM_VARIANTS)
    return np.arange(ops.N_VARIANTS) if dtype == F32 else np.setdiff1d(np.arange(ops.N_VARIANTS), [21, 23])


class Selector:
    """The 16 -> 64 -> 64 -> 24 MLP, its feature standardisation and training range, on the
    device, for one op ("spmm" or "sddmm")."""

    def __init__(self, weights=None, norm=None, seed=0, device="cuda", op="spmm", margin=0.1, gap=0.02):
        self.device = torch.device(device)
        self.op = op
        if weights is None:
            rng = np.random.default_rng(seed)
            parts = []
            for fan_out, fan_in in ((64, 16), (64, 64), (24, 64)):
                parts.append(rng.standard_normal(fan_out * fan_in) * math.sqrt(2.0 / fan_in))
                parts.append(np.zeros(fan_out))
            weights = np.concatenate(parts).astype(np.float32)
        self.weights = torch.as_tensor(np.asarray(weights, np.float32), device=self.device).contiguous()
        assert self.weights.numel() == ops.N_PARAMS
        self.norm = None if norm is None else torch.as_tensor(np.asarray(norm, np.float32), device=self.device)
        self.adam = torch.zeros(2 * ops.N_PARAMS, device=self.device)
        self.steps_done = 0
        self.fmin = self.fmax = None  # training range of every feature (host float64[16])
        self.margin, self.gap = float(margin), float(gap)
        self.meta = {"seed": seed, "op": op}
        self._fallback = {}  # pattern key -> autotuned variant
        self._plans = {}  # pattern key -> HspPlan (variant 23)
        self.counts = {"choices": 0, "range": 0, "gap": 0, "autotuned": 0}

    # ---- training ------------------------------------------------------------------------

    def fit(self, feats, times, steps=3000, batch=64, lr=1e-3, seed=0):
        """Adam on the masked squared error of log(t_v / t_best); records the features'
        training range for the fallback."""
        f_host = np.asarray(feats, np.float32)
        feats = torch.as_tensor(f_host, device=self.device).contiguous()
        tgt, mask = targets_from_times(times)
        n = feats.shape[0]
        if self.norm is None:
            self.norm = ops.feature_norm(feats)
        self.fmin, self.fmax = f_host.min(axis=0).astype(np.float64), f_host.max(axis=0).astype(np.float64)
        order = np.concatenate([np.random.default_rng([seed, e]).permutation(n)
                                for e in range((steps * batch) // n + 1)]).astype(np.int32)
        order_d = torch.as_tensor(order, device=self.device)
        ops.mlp_train(self.weights, self.adam, self.norm, feats, torch.as_tensor(tgt, device=self.device),
                      torch.as_tensor(mask, device=self.device), order_d, steps, batch, lr, self.steps_done)
        self.steps_done += steps
        self.meta.update({"steps": self.steps_done, "batch": batch, "lr": lr, "train_samples": int(n)})
        return self

    def predict(self, feats):
        feats = torch.as_tensor(np.asarray(feats, np.float32), device=self.device).reshape(-1, ops.N_FEATURES)
        out, choice = ops.mlp_predict(self.weights, self.norm, feats.contiguous())
        return out, choice

    # ---- choice with fallback --------------------------------------------------------------

    def out_of_range(self, f) -> bool:
        """True when a feature lies outside the training range widened by margin x range."""
        if self.fmin is None:
            return False
        f = np.asarray(f, np.float64)
        span = np.maximum(self.fmax - self.fmin, 1e-6)
        return bool(np.any(f < self.fmin - self.margin * span) or np.any(f > self.fmax + self.margin * span))

    def model_choice(self, f_dev, dtype):
        """(variant, gap, predictions) of the MLP alone, over the applicable variants."""
        out, _ = ops.mlp_predict(self.weights, self.norm, f_dev.reshape(1, -1))
        pred = out.cpu().numpy()[0].astype(np.float64)
        idx = applicable(self.op, dtype)
        order = idx[np.argsort(pred[idx], kind="stable")]
        gap = float(pred[order[1]] - pred[order[0]]) if order.size > 1 else math.inf
        return int(order[0]), gap, pred

    def decide(self, rowptr, colidx, ncols, N, dtype=F32, tune=None, fallback=True):
        """(variant, reason): the MLP's choice (reason None), or, when a fallback trigger
        fires ("range" or "gap") and ``tune`` is given, the autotuner's best on this
        pattern (kept per pattern and width, so it runs once).  ``tune()`` runs the
        autotuner and returns its best index."""
        self.counts["choices"] += 1
        f = ops.features(rowptr, colidx, ncols, N, dtype)
        v, gap, _ = self.model_choice(f, dtype)
        if not fallback or tune is None:
            return v, None
        reason = "range" if self.out_of_range(f.cpu().numpy()) else "gap" if gap < self.gap else None
        if reason is None:
            return v, None
        self.counts[reason] += 1
        key = (rowptr.data_ptr(), colidx.data_ptr(), rowptr.numel(), int(ncols), colidx.numel(), int(N), int(dtype))
        if key not in self._fallback:
            self._fallback[key] = int(tune())
            self.counts["autotuned"] += 1
        return self._fallback[key], reason

    def choose(self, rowptr, colidx, ncols, N, dtype=F32, fallback=True) -> int:
        """Variant index for one matrix and width.  The fallback autotunes on zero-valued
        operands of this pattern and width (the timings do not depend on the values)."""
        def tune():
            M, nnz = rowptr.numel() - 1, colidx.numel()
            dt = torch.bfloat16 if dtype == BF16 else torch.float32
            vals = torch.zeros(nnz, dtype=torch.float32 if self.op == "sddmm" else dt, device=rowptr.device)
            if self.op == "sddmm":
                X = torch.zeros((M, N), dtype=dt, device=rowptr.device)
                Y = torch.zeros((ncols, N), dtype=dt, device=rowptr.device)
                out = torch.empty(nnz, dtype=torch.float32, device=rowptr.device)
                return ops.autotune_sddmm(rowptr, colidx, vals, X, Y, out)[1]
            B = torch.zeros((ncols, N), dtype=dt, device=rowptr.device)
            C = torch.empty((M, N), dtype=torch.float32, device=rowptr.device)
            return ops.autotune(rowptr, colidx, vals, B, C)[1]

        return self.decide(rowptr, colidx, ncols, N, dtype, tune=tune, fallback=fallback)[0]

    def spmm(self, rowptr, colidx, vals, B, out=None, fallback=True, **kw):
        """C = A B with the chosen variant (the fallback autotunes on these operands)."""
        assert self.op == "spmm"
        dtype = BF16 if vals.dtype == torch.bfloat16 else F32
        if out is None:
            out = torch.empty((rowptr.numel() - 1, B.shape[1]), dtype=torch.float32, device=B.device)
        v, _ = self.decide(rowptr, colidx, B.shape[0], B.shape[1], dtype,
                           tune=lambda: ops.autotune(rowptr, colidx, vals, B, out)[1], fallback=fallback)
        return self.run_spmm(v, rowptr, colidx, vals, B, out, **kw)

    def run_spmm(self, v, rowptr, colidx, vals, B, out, stream=None):
        """Runs SpMM variant v (21 / 23: the SELL-C-sigma / hyper-sparse plan, built once per
        pattern; a SELL plan copies the values, so it is rebuilt if they are to change)."""
        opts = ops.variant_options(v)
        if opts["variant"] in (ops.HSP_PLAN, ops.SELL_PLAN):
            key = (opts["variant"], rowptr.data_ptr(), colidx.data_ptr(), vals.data_ptr(), rowptr.numel(),
                   colidx.numel())
            if key not in self._plans:
                make = ops.HspPlan if opts["variant"] == ops.HSP_PLAN else ops.SellPlan
                self._plans[key] = make(rowptr, colidx, vals, B.shape[0], stream=stream)
            return self._plans[key].execute(B, out=out, stream=stream)
        return ops.spmm(rowptr, colidx, vals, B, out=out, stream=stream, **opts)

    def sddmm(self, rowptr, colidx, svals, X, Y, out=None, fallback=True, **kw):
        """out = S o (X Y^T) with the chosen SDDMM variant."""
        assert self.op == "sddmm"
        dtype = BF16 if X.dtype == torch.bfloat16 else F32
        if out is None:
            out = torch.empty(colidx.numel(), dtype=torch.float32, device=X.device)
        v, _ = self.decide(rowptr, colidx, Y.shape[0], X.shape[1], dtype,
                           tune=lambda: ops.autotune_sddmm(rowptr, colidx, svals, X, Y, out)[1], fallback=fallback)
        return ops.sddmm(rowptr, colidx, svals, X, Y, out=out, **ops.sddmm_variant_options(v), **kw)

    # ---- persistence -------------------------------------------------------------------------

    def save(self, path=None, **extra):
        path = path or (DEFAULT_SDDMM_MODEL if self.op == "sddmm" else DEFAULT_MODEL)
        w = self.weights.cpu().numpy().astype("<f4")
        nm = self.norm.cpu().numpy().astype("<f4")
        with open(path + ".bin", "wb") as f:
            f.write(w.tobytes())
            f.write(nm.tobytes())
        variants = ([ops.sddmm_variant_options(i) for i in range(ops.N_SDDMM_VARIANTS)] if self.op == "sddmm"
                    else [ops.variant_options(i) for i in range(ops.N_VARIANTS)])
        head = {"format": "gbsp-selector-2", "op": self.op, "params": int(w.size), "norm": int(nm.size),
                "layers": [16, 64, 64, 24], "variants": variants,
                "feature_min": None if self.fmin is None else [float(x) for x in self.fmin],
                "feature_max": None if self.fmax is None else [float(x) for x in self.fmax],
                "fallback": {"margin": self.margin, "gap": self.gap}, **self.meta, **extra}
        head["op"] = self.op
        with open(path + ".json", "w") as f:
            json.dump(head, f, indent=1)

    @classmethod
    def load(cls, path=None, device="cuda", op="spmm"):
        path = path or (DEFAULT_SDDMM_MODEL if op == "sddmm" else DEFAULT_MODEL)
        with open(path + ".json") as f:
            head = json.load(f)
        raw = np.fromfile(path + ".bin", dtype="<f4")
        P = head["params"]
        fb = head.get("fallback", {})
        s = cls(weights=raw[:P], norm=raw[P:P + head["norm"]], device=device, op=head.get("op", op),
                margin=fb.get("margin", 0.1), gap=fb.get("gap", 0.02))
        if head.get("feature_min") is not None:
            s.fmin = np.asarray(head["feature_min"], np.float64)
            s.fmax = np.asarray(head["feature_max"], np.float64)
        s.meta = head
        return s
