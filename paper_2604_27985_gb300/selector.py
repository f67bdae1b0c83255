"""Learned choice of the SpMM variant: features -> MLP -> the variant with the smallest
predicted time, trained on the exhaustive autotuner's timings.

Everything numerical runs in the library's kernels (gbsp_features, gbsp_autotune,
gbsp_feature_norm, gbsp_mlp_train, gbsp_mlp_predict); this module keeps the weight tensors,
turns timings into targets (log of each variant's time over the best one, masked where a
variant did not run) and saves / loads a trained model (raw FP32 weights + JSON header).
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


def label(rowptr, colidx, vals, ncols, N, dtype, reps=3, stream=None):
    """Features (device float32[16]) and the 24 variant times (ms) of one matrix, with a
    zero-filled dense operand of width N in the given dtype."""
    dev = rowptr.device
    B = torch.zeros((ncols, N), dtype=torch.bfloat16 if dtype == BF16 else torch.float32, device=dev)
    C = torch.empty((rowptr.numel() - 1, N), dtype=torch.float32, device=dev)
    v = ops.quantize_bf16(vals) if dtype == BF16 else vals
    feats = ops.features(rowptr, colidx, ncols, N, dtype, stream=stream)
    times, _ = ops.autotune(rowptr, colidx, v, B, C, reps=reps, stream=stream)
    return feats, times


class Selector:
    """The 16 -> 64 -> 64 -> 24 MLP and its feature standardisation, on the device."""

    def __init__(self, weights=None, norm=None, seed=0, device="cuda"):
        self.device = torch.device(device)
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
        self.meta = {"seed": seed}

    def fit(self, feats, times, steps=3000, batch=64, lr=1e-3, seed=0):
        """Adam on the masked squared error of log(t_v / t_best)."""
        feats = torch.as_tensor(np.asarray(feats, np.float32), device=self.device).contiguous()
        tgt, mask = targets_from_times(times)
        n = feats.shape[0]
        if self.norm is None:
            self.norm = ops.feature_norm(feats)
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

    def choose(self, rowptr, colidx, ncols, N, dtype=F32) -> int:
        """Variant index for one matrix and width (features and inference on the device)."""
        f = ops.features(rowptr, colidx, ncols, N, dtype).reshape(1, -1)
        _, choice = ops.mlp_predict(self.weights, self.norm, f)
        return int(choice.item())

    def spmm(self, rowptr, colidx, vals, B, out=None, **kw):
        dtype = BF16 if vals.dtype == torch.bfloat16 else F32
        v = self.choose(rowptr, colidx, B.shape[0], B.shape[1], dtype)
        return ops.spmm(rowptr, colidx, vals, B, out=out, **ops.variant_options(v), **kw)

    def save(self, path=DEFAULT_MODEL, **extra):
        w = self.weights.cpu().numpy().astype("<f4")
        nm = self.norm.cpu().numpy().astype("<f4")
        with open(path + ".bin", "wb") as f:
            f.write(w.tobytes())
            f.write(nm.tobytes())
        head = {"format": "gbsp-selector-1", "params": int(w.size), "norm": int(nm.size),
                "layers": [16, 64, 64, 24], "variants": [ops.variant_options(i) for i in range(ops.N_VARIANTS)],
                **self.meta, **extra}
        with open(path + ".json", "w") as f:
            json.dump(head, f, indent=1)

    @classmethod
    def load(cls, path=DEFAULT_MODEL, device="cuda"):
        with open(path + ".json") as f:
            head = json.load(f)
        raw = np.fromfile(path + ".bin", dtype="<f4")
        P = head["params"]
        s = cls(weights=raw[:P], norm=raw[P:P + head["norm"]], device=device)
        s.meta = head
        return s
