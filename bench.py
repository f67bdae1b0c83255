"""Throughput of the CSR SpMM + SDDMM hot path on one GB300 (or N replicas).

One step = one SpMM (Eq. 1, N = 64) and one SDDMM (Eq. 2, Kd = 32) over a 65,536 x 65,536
CSR matrix at 99% sparsity (42,949,673 nonzeros, uniform rows, seed 1001), FP32, inputs
resident in HBM.  The CSR arrays alone (344 MB) exceed the 129 MB L2, so no flush is
needed between steps.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores (a bounded row sample of the
same workload per step) and prints the same line with "impl": "reference".

The other rows of the hot path print one line each with --workload: precision (BF16 /
E4M3 forms and the tensor-core plans on 16,384^2 at 90%), gnn (the 512-graph chain; --gat
adds the row softmax), batched (grouped SpMM / SDDMM plans), selector (training, regret),
sweep (the FP32 scale / sparsity sweep with the selector's choice), kbin (K-binned SpMM on
1,048,576^2) and hsp (hyper-sparse SpMM).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

M = K = 65536
SPARSITY = 0.99
N_SPMM = 64
KD_SDDMM = 32
SEED = 1001
METRIC = "SpMM & SDDMM GFLOP/s (2*nnz*N) and % HBM roofline"
WORKLOAD = (f"CSR {M}x{K} at {SPARSITY:.0%} sparsity, uniform rows, seed {SEED}; "
            f"SpMM N={N_SPMM} + SDDMM Kd={KD_SDDMM}; FP32 values and dense operands")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_inputs(rank: int):
    A = gen.csr_uniform(M, K, SPARSITY, seed=SEED + 100 * rank)
    B = gen.dense_normal(K, N_SPMM, SEED + 100 * rank + 1)
    X = gen.dense_normal(M, KD_SDDMM, SEED + 100 * rank + 2)
    Y = gen.dense_normal(K, KD_SDDMM, SEED + 100 * rank + 3)
    return A, B, X, Y


def flops(nnz: int) -> float:
    return 2.0 * nnz * N_SPMM + 2.0 * nnz * KD_SDDMM


def gather_bytes_spmm(nnz, m, n, v=4, e=4):
    """Gather-model bytes of one SpMM: per nonzero its index, its value and one B row; per
    row one row pointer and one C row."""
    return nnz * (4 + v + n * e) + m * (4 + 4 * n)


def gather_bytes_sddmm(nnz, m, kd, v=4, e=4):
    """Gather-model bytes of one SDDMM: per nonzero index, value, output and one Y row;
    per row one row pointer and one X row."""
    return nnz * (4 + v + 4 + kd * e) + m * (4 + kd * e)


def compulsory_bytes_spmm(nnz, m, k, n, v=4, e=4):
    """Every operand moved once."""
    return 4 * (m + 1) + (4 + v) * nnz + k * n * e + 4 * m * n


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, start: bool):
        if start:
            self.t_start = time.time()
        else:
            self.t_end = time.time()

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        """Median SM clock and the throttle reasons seen by the samples that arrived while
        the timed region ran (the first one after it if the region was shorter than the
        sampling period)."""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "t_start", 0.0), getattr(self, "t_end", 1e30)
        inside = [ln for ts, ln in self.lines if t0 <= ts <= t1 + 0.15]
        if not inside:
            inside = [ln for ts, ln in self.lines if ts >= t0][:1]
        for line in inside:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["no nvidia-smi samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over the process group (the slowest rank
    sets the job's time)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_gflops(world, gflop_per_rank, ms_max):
    """Replicas: every rank does the same work, the job takes the slowest rank's time."""
    return world * gflop_per_rank / (ms_max / 1e3)


def kernel_traffic():
    """Per-launch DRAM bytes of the SpMM kernel from the committed ncu summary, or None
    if the kernel sources changed since those counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:
        return None, None
    try:
        if sources_sha256(t.get("sources", [])) != t.get("sources_sha256"):
            return None, None
    except OSError:
        return None, None
    return t.get("spmm_bytes_per_launch"), t.get("sddmm_bytes_per_launch")


TRAFFIC_SOURCES = ["paper_2604_27985_gb300/csrc/common.cuh", "paper_2604_27985_gb300/csrc/spmm_kernels.cuh",
                   "paper_2604_27985_gb300/csrc/spmm_launch.cuh", "paper_2604_27985_gb300/csrc/sddmm_kernels.cuh",
                   "paper_2604_27985_gb300/csrc/sddmm.cu", "paper_2604_27985_gb300/csrc/api.cu",
                   "paper_2604_27985_gb300/csrc/auto.cu"]


def sources_sha256(names):
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def write_traffic(spmm_report, spmm_re, sddmm_report, sddmm_re):
    """Stores per-launch DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the
    SpMM and SDDMM kernels from ncu reports (one report may hold both) in
    profiles/traffic.json, stamped with the sha256 of the kernel sources: bench lines carry
    them only while the kernels are unchanged."""
    import csv
    import io
    import re

    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}

    def per_launch(report, pattern):
        out = subprocess.run(["ncu", "-i", report, "--page", "raw", "--csv"], capture_output=True, text=True).stdout
        rows = list(csv.reader(io.StringIO(out)))
        hdr, units = rows[0], rows[1]
        vals = []
        for r in rows[2:]:
            d = dict(zip(hdr, r))
            if re.search(pattern, d["Kernel Name"]):
                vals.append(sum(float(d[m].replace(",", "")) * scale[units[hdr.index(m)]]
                                for m in ("dram__bytes_read.sum", "dram__bytes_write.sum")))
        return sum(vals) / len(vals) if vals else None

    t = {"reports": [os.path.basename(spmm_report), os.path.basename(sddmm_report)], "sources": TRAFFIC_SOURCES,
         "sources_sha256": sources_sha256(TRAFFIC_SOURCES),
         "spmm_bytes_per_launch": per_launch(spmm_report, spmm_re),
         "sddmm_bytes_per_launch": per_launch(sddmm_report, sddmm_re)}
    with open(os.path.join(ROOT, "profiles", "traffic.json"), "w") as f:
        json.dump(t, f, indent=1)
    print(json.dumps(t))


def _gather_ceiling(p, nnz, kernel_ms):
    """The kernel's gathered-row bytes per second against the gather probe's on the same
    indices and rows (the level that binds when the gathered operand sits in L2)."""
    achieved = nnz * p["row_bytes"] / (kernel_ms / 1e3) / 1e9
    return {"probe": "gbsp_gather_probe over the workload's colidx", "row_bytes": p["row_bytes"],
            "probe_gbs": p["gbs"], "kernel_gbs": round(achieved, 1), "frac": round(achieved / p["gbs"], 4)}


def l2_roofline(kernel, nnz, row_bytes, probe_gbs, ms, hbm_peak, hbm_kind, compulsory, gather_model, traffic):
    """Roofline of a gather kernel whose gathered operand sits in L2: the binding roof is
    the L2 -> SM gather path, measured in the same run by the gather probe over the
    workload's own column indices and rows of the same size.  achieved = the gathered-row
    bytes of one launch (nnz * row_bytes) / its event-timed duration; frac = achieved /
    probe.  Beside it: the HBM fraction on compulsory bytes (every operand moved once)
    against the measured copy peak, and the gather-model bytes (which count L2 hits and so
    exceed HBM) for reference."""
    achieved = nnz * row_bytes / (ms / 1e3) / 1e9
    return {"bound": "l2", "kernel": kernel, "achieved": round(achieved, 1), "peak": probe_gbs,
            "peak_kind": f"measured in this run: gather probe, {row_bytes}-byte rows over the workload's colidx",
            "unit": "GB/s", "frac": round(achieved / probe_gbs, 4), "traffic": traffic,
            "algorithmic_bytes_per_launch": int(nnz * row_bytes), "ms_per_launch": round(ms, 4),
            "hbm": {"bytes": int(compulsory), "achieved": round(compulsory / (ms / 1e3) / 1e9, 1), "peak": hbm_peak,
                    "peak_kind": hbm_kind, "frac": round(compulsory / (ms / 1e3) / 1e9 / hbm_peak, 4),
                    "model": "compulsory: every operand once"},
            "gather_model_bytes": int(gather_model),
            "gather_model_gbs": round(gather_model / (ms / 1e3) / 1e9, 1)}


def compulsory_bytes_sddmm(nnz, m, n, kd, v=4, e=4):
    """Every operand of one SDDMM moved once: row pointers, indices, values, X, Y, out."""
    return 4 * (m + 1) + (4 + v + 4) * nnz + (m + n) * kd * e


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2604_27985_gb300 as gb

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    A, B, X, Y = make_inputs(rank)
    nnz = A.nnz
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rp, ci, v, Bd, Xd, Yd = t(A.rowptr), t(A.colidx), t(A.vals), t(B), t(X), t(Y)
    C = torch.empty((M, N_SPMM), device=dev)
    out = torch.empty(nnz, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        gb.spmm(rp, ci, v, Bd, out=C, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        gb.sddmm(rp, ci, v, Xd, Yd, out=out, stream=stream)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = gb.launch_count()
    with ClockSampler(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        clk.mark(True)
        t0.record(stream)
        for k in range(args.steps):
            step(evs[k])
        t1.record(stream)
        torch.cuda.synchronize(dev)
        clk.mark(False)
    launches = gb.launch_count() - launches0
    if world > 1:
        dist.barrier()
    total_ms = t0.elapsed_time(t1)
    spmm_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    sddmm_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))

    # end to end through the public API with host buffers: the library's host-resident entry
    # point streams this step's inputs from pinned host memory in row chunks, computes both
    # products and streams C and out back, all inside the timed region.
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_rp, h_ci, h_v, h_B, h_X, h_Y = (pin(a) for a in (A.rowptr, A.colidx, A.vals, B, X, Y))
    h_C = torch.empty((M, N_SPMM), dtype=torch.float32).pin_memory()
    h_out = torch.empty(nnz, dtype=torch.float32).pin_memory()
    h2d = sum(h.numel() * h.element_size() for h in (h_rp, h_ci, h_v, h_B, h_X, h_Y))
    d2h = h_C.numel() * 4 + h_out.numel() * 4

    def e2e_step():
        gb.spmm_sddmm_host(h_rp, h_ci, h_v, B=h_B, C=h_C, X=h_X, Y=h_Y, out=h_out, chunks=args.e2e_chunks,
                           slots=args.e2e_slots, stream=stream)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / args.steps

    ms = total_ms / args.steps
    if world > 1:
        ms, e2e_ms, spmm_ms, sddmm_ms = max_over_ranks([ms, e2e_ms, spmm_ms, sddmm_ms], dev)
    gflop = flops(nnz) / 1e9
    value = whole_job_gflops(world, gflop, ms)
    peak, peak_kind = peaks()
    spmm_bytes = gather_bytes_spmm(nnz, M, N_SPMM)
    sddmm_bytes = gather_bytes_sddmm(nnz, M, KD_SDDMM)
    traffic_spmm, traffic_sddmm = kernel_traffic()
    comp = compulsory_bytes_spmm(nnz, M, K, N_SPMM)

    # "tuned" forms of the same step, timed after the main region: the shipped selector's
    # SpMM variant for this matrix and width, and the step with BF16 operands
    tuned = None
    if not args.no_tuned:
        from paper_2604_27985_gb300 import selector as sel

        model = sel.Selector.load()
        v_idx = model.choose(rp, ci, K, N_SPMM, 0)
        kw = gb.variant_options(v_idx)
        ms_sel = _event_ms(lambda: model.run_spmm(v_idx, rp, ci, v, Bd, C, stream=stream), 50, 5, stream)
        qa, qB, qX, qY = (gb.quantize_bf16(a) for a in (v, Bd, Xd, Yd))
        ms_bs = _event_ms(lambda: gb.spmm(rp, ci, qa, qB, out=C, stream=stream), 50, 5, stream)
        ms_bd = _event_ms(lambda: gb.sddmm(rp, ci, v, qX, qY, out=out, stream=stream), 50, 5, stream)
        tuned = {"selector_variant": v_idx, "selector_options": kw, "selector_spmm_ms": round(ms_sel, 4),
                 "bf16_spmm_ms": round(ms_bs, 4), "bf16_sddmm_ms": round(ms_bd, 4),
                 "bf16_step_gflops": round(flops(nnz) / ((ms_bs + ms_bd) / 1e3) / 1e9, 1),
                 "note": "BF16 operands, FP32 accumulation; parity in tests/test_parity_lowp.py"}

    # the ceiling of the gather pattern itself (outside the timed region): the workload's
    # column indices over B's and Y's rows, same lane layout, no arithmetic
    sink = torch.empty(8 * gb.sm_count() * 256, dtype=torch.int32, device=dev)
    probe = {}
    for name, table, rb in (("spmm", Bd, N_SPMM * 4), ("sddmm", Yd, KD_SDDMM * 4)):
        ms_p = min(_event_ms(lambda: gb.gather_probe(table, ci, rb, unroll=u, sink=sink, stream=stream), 20, 3, stream)
                   for u in (4, 8))
        probe[name] = {"row_bytes": rb, "ms": round(ms_p, 4), "gbs": round(nnz * rb / (ms_p / 1e3) / 1e9, 1)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(A, B, X, Y, budget_s=args.cpu_seconds)

    clocks = clk.summary()
    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GFLOP/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded generators; no dataset)",
        "config": {"workload": WORKLOAD, "nnz": nnz, "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (CSR arrays 344 MB per step), no flush",
                   "variant": "auto (rowsplit SpMM, rowsplit SDDMM)"},
        "roofline": l2_roofline("spmm (Eq. 1), row split", nnz, N_SPMM * 4, probe["spmm"]["gbs"], spmm_ms, peak,
                                peak_kind, comp, spmm_bytes, traffic_spmm),
        "roofline_sddmm": l2_roofline("sddmm (Eq. 2), row split", nnz, KD_SDDMM * 4, probe["sddmm"]["gbs"], sddmm_ms,
                                      peak, peak_kind, compulsory_bytes_sddmm(nnz, M, K, KD_SDDMM), sddmm_bytes,
                                      traffic_sddmm),
        "spmm_gflops": round(2.0 * nnz * N_SPMM / (spmm_ms / 1e3) / 1e9, 1),
        "sddmm_gflops": round(2.0 * nnz * KD_SDDMM / (sddmm_ms / 1e3) / 1e9, 1),
        "e2e": {"value": round(world * gflop / (e2e_ms / 1e3), 2), "unit": "GFLOP/s", "ms_per_step": round(e2e_ms, 4),
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if tuned is not None:
        line["tuned"] = tuned
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---- the other hot-path rows: one JSON line each (python bench.py --workload ...) ----------

def _event_ms(fn, steps, warmup, stream):
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _line(metric, value, unit, ms, args, dtype, config, **extra):
    out = {"metric": metric, "value": round(value, 3), "unit": unit, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": dtype, "data": "synthetic (seeded generators; no dataset)",
           "config": config}
    out.update(extra)
    print(json.dumps(out), flush=True)


def _probe_gbs(gb, table, ci, row_bytes, stream):
    """GB/s of the gather probe over these column indices and rows of row_bytes bytes (the
    better of 4 and 8 rows in flight per lane)."""
    ms = min(_event_ms(lambda: gb.gather_probe(table, ci, row_bytes, unroll=u, stream=stream), 20, 3, stream)
             for u in (4, 8))
    return round(ci.numel() * row_bytes / (ms / 1e3) / 1e9, 1)


def _errors(gpu, ref, scale):
    """max and mean of |gpu - ref| / scale over the outputs with scale > 0."""
    gpu = np.asarray(gpu, dtype=np.float64)
    nz = scale > 0
    rel = np.abs(gpu[nz] - ref[nz]) / scale[nz]
    return {"max": float(rel.max()) if rel.size else 0.0, "mean": float(rel.mean()) if rel.size else 0.0}


def run_precision(args):
    """16,384^2 at 90%, N = Kd = 256: SpMM + SDDMM in FP32, BF16, E4M3 (CUDA cores) and the
    BF16 / E4M3 condensed-tile tensor-core plans (SpMM and SDDMM), on the uniform and the
    clustered layouts.  Per form: event-timed SpMM and SDDMM, the L2 roof (gathered-row
    bytes per second against the gather probe over the same indices and row size), the HBM
    fraction on compulsory bytes, and, outside the timed region, the max and mean of
    |err| / sum |a||b| against the FP64 oracle on the ORIGINAL FP32 values over 400
    sampled rows (quantisation included)."""
    import torch

    import oracle
    import paper_2604_27985_gb300 as gb

    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    stream = torch.cuda.current_stream()
    peak, peak_kind = peaks()
    forms, launches = {}, 0
    W = 256
    for layout in args.precision_layouts.split(","):
        A = (gen.csr_uniform(16384, 16384, 0.9, seed=2001) if layout == "uniform"
             else gen.csr_clustered(16384, 16384, 0.9, seed=2002))
        B, X, Y = (gen.dense_normal(16384, W, 2003 + k) for k in range(3))
        rp, ci, v = t(A.rowptr), t(A.colidx), t(A.vals)
        Bd, Xd, Yd = t(B), t(X), t(Y)
        C = torch.empty((A.M, W), device=dev)
        out = torch.empty(A.nnz, device=dev)
        qa, qb, qx, qy = gb.quantize_bf16(v), gb.quantize_bf16(Bd), gb.quantize_bf16(Xd), gb.quantize_bf16(Yd)
        ea, sa = gb.quantize_e4m3_rows(v, rp)
        eb, sb = gb.quantize_e4m3_rows(Bd)
        ex, ux = gb.quantize_e4m3_rows(Xd)
        ey, uy = gb.quantize_e4m3_rows(Yd)
        plan = gb.TcPlan(rp, ci, qa, A.K)
        plan8 = gb.TcPlan(rp, ci, ea, A.K, row_scale=sa)
        info, info8 = plan.info(), plan8.info()
        # sampled rows and the oracle on the original FP32 values (outside any timed region)
        wins = np.sort(np.random.default_rng(17).choice(A.M // 16, 25, replace=False))
        rows = (wins[:, None] * 16 + np.arange(16)).ravel()
        lens = np.diff(A.rowptr.astype(np.int64))[rows]
        idx = np.concatenate([np.arange(A.rowptr[r], A.rowptr[r + 1]) for r in rows])
        srp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        ref_c, sc_c = oracle.spmm(srp, A.colidx[idx], A.vals[idx], B)
        ref_o, sc_o = oracle.sddmm(srp, A.colidx[idx], A.vals[idx], X[rows], Y)
        probes = {rb: _probe_gbs(gb, tb_, ci, rb, stream)
                  for rb, tb_ in ((W * 4, Bd), (W * 2, qb), (W, eb))}
        runs = {
            "fp32": (lambda: gb.spmm(rp, ci, v, Bd, out=C), lambda: gb.sddmm(rp, ci, v, Xd, Yd, out=out), 4, 4),
            "bf16": (lambda: gb.spmm(rp, ci, qa, qb, out=C), lambda: gb.sddmm(rp, ci, v, qx, qy, out=out), 2, 2),
            "e4m3": (lambda: gb.spmm(rp, ci, ea, eb, out=C, a_scale=sa, b_scale=sb),
                     lambda: gb.sddmm(rp, ci, v, ex, ey, out=out, x_scale=ux, y_scale=uy), 1, 1),
            "tc_bf16": (lambda: plan.execute(qb, out=C), lambda: plan.sddmm(v, qx, qy, out=out), 2, 2),
            "tc_e4m3": (lambda: plan8.execute(eb, out=C, row_scale=sb),
                        lambda: plan8.sddmm(v, ex, ey, out=out, x_scale=ux, y_scale=uy), 1, 1),
        }
        for name, (f_spmm, f_sddmm, vb, e_) in runs.items():
            l0 = gb.launch_count()
            ms_a = _event_ms(f_spmm, args.steps, args.warmup, stream)
            launches += gb.launch_count() - l0
            err_c = _errors(C.cpu().numpy()[rows], ref_c, sc_c)
            l0 = gb.launch_count()
            ms_b = _event_ms(f_sddmm, args.steps, args.warmup, stream)
            launches += gb.launch_count() - l0
            err_o = _errors(out.cpu().numpy()[idx], ref_o, sc_o)
            rb = W * e_
            pinfo = info if name == "tc_bf16" else info8 if name == "tc_e4m3" else None
            # gathered B rows: one per stored entry on the CSR kernels; a plan gathers 8 per
            # dense block (each once) and one per residual entry
            rows_gathered = (A.nnz if pinfo is None else pinfo["residual_nnz"] + 8 * pinfo["dense_blocks"])
            comp_a = compulsory_bytes_spmm(A.nnz, A.M, A.K, W, v=vb, e=e_)
            comp_b = compulsory_bytes_sddmm(A.nnz, A.M, A.K, W, v=4, e=e_)
            forms[f"{layout}/{name}"] = {
                "spmm_ms": round(ms_a, 4), "sddmm_ms": round(ms_b, 4),
                "spmm_gflops": round(2 * A.nnz * W / ms_a / 1e6, 1),
                "sddmm_gflops": round(2 * A.nnz * W / ms_b / 1e6, 1),
                "step_gflops": round(4 * A.nnz * W / (ms_a + ms_b) / 1e6, 1),
                "spmm_l2": {"gathered_gbs": round(rows_gathered * rb / ms_a / 1e6, 1), "probe_gbs": probes[rb],
                            "frac": round(rows_gathered * rb / ms_a / 1e6 / probes[rb], 4)},
                "spmm_hbm_frac": round(comp_a / ms_a / 1e6 / peak, 4),
                "sddmm_hbm_frac": round(comp_b / ms_b / 1e6 / peak, 4),
                "err_vs_fp64_of_fp32_inputs": {"spmm": err_c, "sddmm": err_o}}
        forms[f"{layout}/tc_plan"] = info
        forms[f"{layout}/tc_plan_e4m3"] = info8
        for p_ in (plan, plan8):
            p_.check()
            p_.close()
    best = max((k for k in forms if "/" in k and "tc_plan" not in k), key=lambda k: forms[k]["step_gflops"])
    last = args.precision_layouts.split(",")[-1]
    base = forms[f"{last}/fp32"]["spmm_ms"] + forms[f"{last}/fp32"]["sddmm_ms"]
    _line("SpMM & SDDMM GFLOP/s (2*nnz*N each), precision forms vs plain FP32", forms[best]["step_gflops"],
          "GFLOP/s", forms[best]["spmm_ms"] + forms[best]["sddmm_ms"], args, best.split("/")[1],
          {"workload": "CSR 16384x16384 at 90% (uniform seed 2001, clustered 16x8 blocks at 40% fill seed 2002), "
                       "SpMM N=256 + SDDMM Kd=256", "best_form": best,
           f"fp32_{last}_step_ms": round(base, 4),
           "errors": "max / mean of |err| / sum|a||b| against FP64 of the original FP32 values, 400 sampled rows",
           "tolerances": {"fp32": 1e-5, "bf16": 1e-2, "e4m3": 4e-2}, "hbm_peak": peak, "hbm_peak_kind": peak_kind},
          forms=forms, gpu_launches=int(launches))


def run_gnn(args):
    """512 graphs (1,000..50,000 nodes, power-law degrees with mean 16), BF16 features of
    width 64/128/256: SDDMM -> SpMM per graph in one persistent launch from a CUDA graph.
    With --gat each row's scores pass through a softmax between the two products (E then
    holds the weights); the algorithmic bytes are the same, E being written once."""
    import torch

    import paper_2604_27985_gb300 as gb

    dev = torch.device("cuda")
    graphs = gen.gnn_batch(G=512, seed=3000)[:args.gnn_graphs]
    devs, flop, gbytes = [], 0.0, 0.0
    for k, (A, N) in enumerate(graphs):
        H = torch.from_numpy(gen.dense_normal(A.M, N, 3000 * 1000 + k)).to(torch.bfloat16).to(dev)
        devs.append((torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colidx).to(dev),
                     torch.from_numpy(A.vals).to(dev), H, torch.empty_like(H),
                     torch.empty(A.nnz, dtype=torch.float32, device=dev)))
        flop += 4.0 * A.nnz * N
        gbytes += (A.nnz * (4 + 4 + 4 + 2 * N) + A.M * (4 + 2 * N + 2 * N)) / 1e9
    plan = gb.GnnPlan(devs, softmax=args.gat, edges_per_tile=args.gnn_edges_per_tile)
    stream = torch.cuda.current_stream()
    launches0 = gb.launch_count()
    ms = _event_ms(plan.execute, args.steps, args.warmup, stream)
    launches = (gb.launch_count() - launches0) // (args.steps + args.warmup)
    peak, peak_kind = peaks()
    info = plan.info()
    # L2 roof: each graph's H (at most 50,000 x 256 BF16 = 25.6 MB) sits in L2 while its
    # tiles run, so the H_j gathers (2N bytes per edge) are held against the gather probe
    # over each width class's own indices on a 50,000-row table of that row size.
    edges_by_w, idx_by_w = {}, {}
    for (A, N) in graphs:
        edges_by_w[N] = edges_by_w.get(N, 0) + A.nnz
        idx_by_w.setdefault(N, []).append(A.colidx)
    t_ceiling, gathered = 0.0, 0.0
    probe = {}
    for N, parts in sorted(idx_by_w.items()):
        ci = torch.from_numpy(np.concatenate(parts)).to(dev)
        table = torch.zeros((50000, N), dtype=torch.bfloat16, device=dev)
        probe[N] = _probe_gbs(gb, table, ci, 2 * N, stream)
        t_ceiling += edges_by_w[N] * 2 * N / (probe[N] * 1e9)
        gathered += edges_by_w[N] * 2 * N
        del ci, table
    comp = sum(A.nnz * 12 + A.M * (4 + 4 * N) for A, N in graphs)
    chain = "SDDMM->row softmax->SpMM" if args.gat else "SDDMM->SpMM"
    _line(f"batched {chain} GFLOP/s (4*nnz*N over the batch)", flop / ms / 1e6, "GFLOP/s", ms, args, "bf16",
          {"workload": f"{len(graphs)} of the 512 graphs (nodes log-uniform [1000, 50000], power-law degree "
                       "(mean 16, max 2048), row-normalised values, BF16 features N in {64,128,256}, seed 3000)",
           "softmax": bool(args.gat), **info},
          roofline={"bound": "l2", "kernel": "gnn_kernel: H_j gathered once per edge (2N bytes)",
                    "achieved": round(gathered / ms / 1e6, 1), "unit": "GB/s",
                    "peak": round(gathered / t_ceiling / 1e9, 1),
                    "peak_kind": "measured in this run: gather probe per width class over the batch's own indices",
                    "probe_gbs_by_width": probe, "frac": round(t_ceiling * 1e3 / ms, 4),
                    "algorithmic_bytes_per_launch": int(gathered),
                    "hbm": {"bytes": int(comp), "achieved": round(comp / ms / 1e6, 1), "peak": peak,
                            "peak_kind": peak_kind, "frac": round(comp / ms / 1e6 / peak, 4),
                            "model": "compulsory: indices, values, E, H and O once"},
                    "gather_model_bytes": int(gbytes * 1e9)},
          gpu_launches_per_step=int(launches))


def run_sweep(args):
    """The plain-FP32 scale / sparsity sweep: 65,536^2 at 99% and 1,048,576^2 at 99.99%
    (about 110M nonzeros; 65,536^2 at 90% too with --sweep-dense, whose generation takes
    minutes), uniform and power-law rows; SpMM at N in {32, 64, 128} and SDDMM at Kd in
    {32, 128}, each with the library's automatic variant.  Every matrix's CSR arrays exceed
    L2.  One JSON line: a point per (matrix, op, width) with its time, GFLOP/s and the
    gather-model fraction of the HBM peak; value = all points' FLOPs over their summed time
    (automatic variant).  SpMM points also time the shipped selector's variant choice."""
    import torch

    import paper_2604_27985_gb300 as gb

    from paper_2604_27985_gb300 import selector as sel

    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    peak, peak_kind = peaks()
    model = sel.Selector.load()
    mats = [(65536, 0.99, "uniform", 1001), (65536, 0.99, "powerlaw", 1002),
            (1048576, 0.9999, "uniform", 1003), (1048576, 0.9999, "powerlaw", 1004)]
    if args.sweep_dense:
        mats += [(65536, 0.9, "uniform", 1005), (65536, 0.9, "powerlaw", 1006)]
    points, flop_sum, ms_sum, launches = [], 0.0, 0.0, 0
    for n, sp, layout, seed in mats:
        A = (gen.csr_uniform if layout == "uniform" else gen.csr_powerlaw)(n, n, sp, seed=seed)
        rp, ci, v = (torch.from_numpy(a).to(dev) for a in (A.rowptr, A.colidx, A.vals))
        touched = int(np.unique(A.colidx).size)  # B (or Y) rows read at least once
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        probe = {}
        sells = {"sell_c64_sigma_all": gb.SellPlan(rp, ci, v, n, C=64, sigma=0),
                 "sell_c64_sigma4096": gb.SellPlan(rp, ci, v, n, C=64, sigma=4096)}
        for op, widths in (("spmm", (32, 64, 128)), ("sddmm", (32, 128))):
            for w in widths:
                if op == "spmm":
                    Bd = torch.randn((n, w), generator=g, device=dev)
                    C = torch.empty((n, w), device=dev)
                    fn = lambda: gb.spmm(rp, ci, v, Bd, out=C, stream=stream)
                    nbytes = gather_bytes_spmm(A.nnz, n, w)
                else:
                    Xd = torch.randn((n, w), generator=g, device=dev)
                    Yd = torch.randn((n, w), generator=g, device=dev)
                    out = torch.empty(A.nnz, device=dev)
                    fn = lambda: gb.sddmm(rp, ci, v, Xd, Yd, out=out, stream=stream)
                    nbytes = gather_bytes_sddmm(A.nnz, n, w)
                l0 = gb.launch_count()
                ms = _event_ms(fn, args.steps, args.warmup, stream)
                launches += gb.launch_count() - l0
                f = 2.0 * A.nnz * w
                flop_sum += f
                ms_sum += ms
                if w not in probe:
                    probe[w] = _probe_gbs(gb, Bd if op == "spmm" else Yd, ci, 4 * w, stream)
                comp = (compulsory_bytes_spmm(A.nnz, n, touched, w) if op == "spmm"
                        else compulsory_bytes_sddmm(A.nnz, n, touched, w))
                pt = {"n": n, "sparsity": sp, "rows": layout, "op": op, "width": w, "nnz": A.nnz,
                      "ms": round(ms, 4), "gflops": round(f / ms / 1e6, 1),
                      "gathered_gbs": round(A.nnz * 4 * w / ms / 1e6, 1), "probe_gbs": probe[w],
                      "frac": round(A.nnz * 4 * w / ms / 1e6 / probe[w], 4),
                      "hbm_frac": round(comp / ms / 1e6 / peak, 4), "gather_model_gbs": round(nbytes / ms / 1e6, 1)}
                # every explicit split beside the automatic one (untimed choice, timed runs)
                splits = ("rowsplit", "merge", "rowgroup") if op == "spmm" else ("rowsplit", "merge", "entry")
                for sp_name in splits:
                    if op == "spmm":
                        f_sp = lambda: gb.spmm(rp, ci, v, Bd, out=C, stream=stream, variant=sp_name)
                    else:
                        f_sp = lambda: gb.sddmm(rp, ci, v, Xd, Yd, out=out, stream=stream, variant=sp_name)
                    pt[f"{sp_name}_ms"] = round(_event_ms(f_sp, args.steps, args.warmup, stream), 4)
                best = min(pt[f"{x}_ms"] for x in splits)
                pt["auto_vs_best_split"] = round(ms / best - 1, 4)
                pt["auto_variant"] = gb.auto_choice(rp, n, ci, op=op, b_bytes=4 * w * n, row_bytes=4 * w)[0]
                if op == "spmm":
                    # SELL-C-sigma (plans built once per matrix, outside the timed calls)
                    for key_, sell_ in sells.items():
                        pt[f"{key_}_ms"] = round(_event_ms(lambda: sell_.execute(Bd, out=C, stream=stream),
                                                           args.steps, args.warmup, stream), 4)
                    # the shipped selector's variant for this matrix and width (untimed choice)
                    v_idx = model.choose(rp, ci, n, w, 0)
                    kw = gb.variant_options(v_idx)
                    ms_sel = _event_ms(lambda: model.run_spmm(v_idx, rp, ci, v, Bd, C, stream=stream), args.steps,
                                       args.warmup, stream)
                    pt.update(selector_variant=v_idx, selector_options=kw, selector_ms=round(ms_sel, 4),
                              selector_frac=round(A.nnz * 4 * w / ms_sel / 1e6 / probe[w], 4))
                points.append(pt)
                del fn
        for sell_ in sells.values():
            sell_.close()
        del A, rp, ci, v
        torch.cuda.empty_cache()
    _line("SpMM & SDDMM GFLOP/s (2*nnz*N) over the plain-FP32 scale/sparsity sweep", flop_sum / ms_sum / 1e6,
          "GFLOP/s", ms_sum, args, "f32",
          {"workload": "65536^2 at 99% and 1048576^2 at 99.99%" + (" and 65536^2 at 90%" if args.sweep_dense else "")
                       + ", uniform and power-law rows (Zipf 1.5, cap 4096), values U[-1,1]; SpMM N 32/64/128, "
                       "SDDMM Kd 32/128, dense operands N(0,1); automatic variant; CSR arrays larger than L2",
           "points": points},
          roofline={"bound": "l2", "kernel": "spmm / sddmm: gathered rows against the gather probe over each "
                                        "matrix's own indices and row size (measured in this run)",
                    "unit": "GB/s", "frac_min": min(p["frac"] for p in points),
                    "frac_max": max(p["frac"] for p in points),
                    "hbm": {"peak": peak, "peak_kind": peak_kind, "model": "compulsory: every operand once "
                            "(rows of B / Y that are read at least once)",
                            "frac_min": min(p["hbm_frac"] for p in points),
                            "frac_max": max(p["hbm_frac"] for p in points)}},
          gpu_launches=int(launches))


def run_kbin(args):
    """K-range-binned SpMM (gbsp_kbin_plan_*) on 1,048,576^2 at 99.99% (uniform and power-law
    rows, the sweep's matrices), where B (128 to 512 MB at N = 32 to 128) exceeds L2: the
    plan's passes over L2-sized B slices against the automatic row split and the merge path,
    for slice budgets of 24, 48 (the default) and 96 MB.  One JSON line; value = the default
    plan's GFLOP/s over all points (2*nnz*N over the summed time)."""
    import torch

    import paper_2604_27985_gb300 as gb

    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    peak, peak_kind = peaks()
    points, flop_sum, ms_sum, launches = [], 0.0, 0.0, 0
    for layout, seed in (("uniform", 1003), ("powerlaw", 1004)):
        n = 1048576
        A = (gen.csr_uniform if layout == "uniform" else gen.csr_powerlaw)(n, n, 0.9999, seed=seed)
        rp, ci, v = (torch.from_numpy(a).to(dev) for a in (A.rowptr, A.colidx, A.vals))
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        touched = int(np.unique(A.colidx).size)
        for N in (32, 64, 128):
            Bd = torch.randn((n, N), generator=g, device=dev)
            C = torch.empty((n, N), device=dev)
            f = 2.0 * A.nnz * N
            nbytes = gather_bytes_spmm(A.nnz, n, N)
            pgbs = _probe_gbs(gb, Bd, ci, 4 * N, stream)
            pt = {"rows": layout, "N": N, "nnz": A.nnz,
                  "rowsplit_ms": round(_event_ms(lambda: gb.spmm(rp, ci, v, Bd, out=C, variant="rowsplit",
                                                                 stream=stream), args.steps, args.warmup, stream), 4),
                  "merge_ms": round(_event_ms(lambda: gb.spmm(rp, ci, v, Bd, out=C, variant="merge", stream=stream),
                                              args.steps, args.warmup, stream), 4)}
            for mb in (24, 48, 96):
                plan = gb.KbinPlan(rp, ci, v, n, N, slice_cols=(mb << 20) // (4 * N))
                l0 = gb.launch_count()
                ms = _event_ms(lambda: plan.execute(Bd, out=C, stream=stream), args.steps, args.warmup, stream)
                if mb == 48:
                    launches += gb.launch_count() - l0
                    flop_sum += f
                    ms_sum += ms
                    comp = compulsory_bytes_spmm(A.nnz, n, touched, N)
                    pt.update(kbin_ms=round(ms, 4), slices=plan.info()["slices"], gflops=round(f / ms / 1e6, 1),
                              gathered_gbs=round(A.nnz * 4 * N / ms / 1e6, 1), probe_gbs=pgbs,
                              frac=round(A.nnz * 4 * N / ms / 1e6 / pgbs, 4),
                              hbm_frac=round(comp / ms / 1e6 / peak, 4), gather_model_gbs=round(nbytes / ms / 1e6, 1),
                              c_partial_bytes=int((2 * plan.info()["slices"] - 1) * n * N * 4))
                pt[f"kbin_{mb}mb_ms"] = round(ms, 4)
                plan.close()
            points.append(pt)
            del Bd, C
        del A, rp, ci, v
        torch.cuda.empty_cache()
    _line("K-binned SpMM GFLOP/s (2*nnz*N) with B larger than L2", flop_sum / ms_sum / 1e6, "GFLOP/s", ms_sum, args,
          "f32",
          {"workload": "1048576^2 at 99.99% (109,951,163 nonzeros), uniform and power-law rows, values U[-1,1]; "
                       "B N(0,1) FP32 with N 32/64/128; default 48 MB B slices; CSR larger than L2",
           "points": points},
          roofline={"bound": "l2", "kernel": "kbin_pass_kernel: gathered B rows against the gather probe over "
                                        "the same indices and row size (measured in this run)", "unit": "GB/s",
                    "frac_min": min(p["frac"] for p in points), "frac_max": max(p["frac"] for p in points),
                    "hbm": {"peak": peak, "peak_kind": peak_kind, "model": "compulsory: every operand once",
                            "frac_min": min(p["hbm_frac"] for p in points),
                            "frac_max": max(p["hbm_frac"] for p in points)}},
          gpu_launches=int(launches))


def _event_ms_flushed(fn, steps, warmup, stream, flush):
    """Mean CUDA-event time of fn with L2 flushed (a buffer larger than L2 rewritten) before
    every call, outside the events."""
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps


def run_hsp(args):
    """Hyper-sparse SpMM (gbsp_hsp_plan_*): rows binned by length in one launch, against the
    automatic row split and the merge path, on 1,048,576^2 at 99.9999% (about 1 entry per
    row), 262,144^2 at 99.999% (about 2.6), 65,536^2 at 99.99% (about 6.6) and 262,144^2 at
    99.99% with power-law rows (mean 26, most rows short); N 32 / 64 / 128.  These inputs
    fit in L2, so L2 is flushed before every timed call.  One JSON line; value = the plan's
    GFLOP/s over all points."""
    import torch

    import paper_2604_27985_gb300 as gb

    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    peak, peak_kind = peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    mats = [(1048576, 0.999999, "uniform", 1007), (262144, 0.99999, "uniform", 1008),
            (65536, 0.9999, "uniform", 1009), (262144, 0.9999, "powerlaw", 1010)]
    points, flop_sum, ms_sum, launches = [], 0.0, 0.0, 0
    for n, sp, layout, seed in mats:
        A = (gen.csr_uniform if layout == "uniform" else gen.csr_powerlaw)(n, n, sp, seed=seed)
        rp, ci, v = (torch.from_numpy(a).to(dev) for a in (A.rowptr, A.colidx, A.vals))
        plan = gb.HspPlan(rp, ci, v, n)
        touched = int(np.unique(A.colidx).size)
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        for N in (32, 64, 128):
            Bd = torch.randn((n, N), generator=g, device=dev)
            C = torch.empty((n, N), device=dev)
            f = 2.0 * A.nnz * N
            nbytes = gather_bytes_spmm(A.nnz, n, N)
            t = lambda fn: round(_event_ms_flushed(fn, args.steps, args.warmup, stream, flush), 4)
            l0 = gb.launch_count()
            ms = _event_ms_flushed(lambda: plan.execute(Bd, out=C, stream=stream), args.steps, args.warmup, stream,
                                   flush)
            launches += (gb.launch_count() - l0) // (args.steps + args.warmup)
            flop_sum += f
            ms_sum += ms
            comp = compulsory_bytes_spmm(A.nnz, n, touched, N)
            points.append({"n": n, "sparsity": sp, "rows": layout, "N": N, "nnz": A.nnz, **plan.info(),
                           "hsp_ms": round(ms, 4), "gflops": round(f / ms / 1e6, 1),
                           "hbm_gbs": round(comp / ms / 1e6, 1), "frac": round(comp / ms / 1e6 / peak, 4),
                           "gather_model_gbs": round(nbytes / ms / 1e6, 1),
                           "rowsplit_ms": t(lambda: gb.spmm(rp, ci, v, Bd, out=C, variant="rowsplit", stream=stream)),
                           "merge_ms": t(lambda: gb.spmm(rp, ci, v, Bd, out=C, variant="merge", stream=stream)),
                           "rowgroup_ms": t(lambda: gb.spmm(rp, ci, v, Bd, out=C, variant="rowgroup", stream=stream)),
                           "auto_ms": t(lambda: gb.spmm(rp, ci, v, Bd, out=C, stream=stream)),
                           "auto_variant": gb.auto_choice(rp, n, ci, b_bytes=4 * N * n, row_bytes=4 * N)[0]})
            del Bd, C
        plan.close()
        del A, rp, ci, v
        torch.cuda.empty_cache()
    _line("hyper-sparse SpMM GFLOP/s (2*nnz*N)", flop_sum / ms_sum / 1e6, "GFLOP/s", ms_sum, args, "f32",
          {"workload": "1048576^2 at 99.9999%, 262144^2 at 99.999%, 65536^2 at 99.99% (uniform rows) and 262144^2 "
                       "at 99.99% (power-law rows), values U[-1,1], B N(0,1) FP32, N 32/64/128",
           "l2": "flushed before every timed call (256 MB written)", "points": points},
          roofline={"bound": "hbm", "kernel": "hsp_kernel, compulsory bytes (every operand once; the B rows read "
                                         "at least once) with L2 flushed before each call",
                    "peak": peak, "peak_kind": peak_kind,
                    "unit": "GB/s", "frac_min": min(p["frac"] for p in points),
                    "frac_max": max(p["frac"] for p in points)},
          gpu_launches_per_call=int(launches // max(1, len(points))))


def run_batched(args):
    """Grouped SpMM and SDDMM over the 512 graphs of the batched configuration (BF16 H of
    width 64/128/256, FP32 outputs): persistent launches (one per lane-layout class) replayed
    from a CUDA graph (gbsp_batch_plan_*) against one launch per graph through spmm_csr_ex /
    sddmm_csr_ex."""
    import torch

    import paper_2604_27985_gb300 as gb

    dev = torch.device("cuda")
    graphs = gen.gnn_batch(G=512, seed=3000)[:args.gnn_graphs]
    sp, sd, flop = [], [], 0.0
    for k, (A, N) in enumerate(graphs):
        H = torch.from_numpy(gen.dense_normal(A.M, N, 3000 * 1000 + k)).to(torch.bfloat16).to(dev)
        rp, ci = torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colidx).to(dev)
        v = torch.from_numpy(A.vals).to(dev)
        sp.append((rp, ci, v.to(torch.bfloat16), H, torch.empty((A.M, N), device=dev)))
        sd.append((rp, ci, v, H, H, torch.empty(max(A.nnz, 1), device=dev)))
        flop += 2.0 * A.nnz * N
    stream = torch.cuda.current_stream()
    p_sp, p_sd = gb.BatchPlan(sp), gb.BatchPlan(sd, sddmm=True)
    launches = []
    for p_ in (p_sp, p_sd):
        l0 = gb.launch_count()
        p_.execute()
        launches.append(gb.launch_count() - l0)
    ms_sp = _event_ms(p_sp.execute, args.steps, args.warmup, stream)
    ms_sd = _event_ms(p_sd.execute, args.steps, args.warmup, stream)

    def loop_spmm():
        for rp, ci, v, H, C in sp:
            gb.spmm(rp, ci, v, H, out=C, stream=stream)

    def loop_sddmm():
        for rp, ci, v, X, Y, out in sd:
            gb.sddmm(rp, ci, v, X, Y, out=out, stream=stream)

    steps = max(3, args.steps // 10)
    ms_lsp = _event_ms(loop_spmm, steps, 2, stream)
    ms_lsd = _event_ms(loop_sddmm, steps, 2, stream)
    _line("batched SpMM + SDDMM GFLOP/s (2*nnz*N each) over many graphs", 2 * flop / (ms_sp + ms_sd) / 1e6,
          "GFLOP/s", ms_sp + ms_sd, args, "bf16",
          {"workload": f"{len(graphs)} of the 512 graphs (nodes log-uniform [1000, 50000], power-law degree "
                       "(mean 16, max 2048), row-normalised values, BF16 H of width N in {64,128,256}, seed 3000); "
                       "SpMM S H and SDDMM S o (H H^T), FP32 outputs"},
          grouped={"spmm_ms": round(ms_sp, 4), "sddmm_ms": round(ms_sd, 4),
                   "launches_per_op": {"spmm": launches[0], "sddmm": launches[1]},
                   "note": "one persistent launch per lane-layout class, replayed from one CUDA graph"},
          per_graph_launches={"spmm_ms": round(ms_lsp, 4), "sddmm_ms": round(ms_lsd, 4),
                              "launches_per_op": len(graphs)},
          speedup={"spmm": round(ms_lsp / ms_sp, 3), "sddmm": round(ms_lsd / ms_sd, 3)})


def run_selector(args):
    """Learned selectors for SpMM and SDDMM: 2,000 training and 200 held-out corpus matrices
    (rows 4,096..262,144) plus 24 held-out matrices of 1,048,576 rows (outside the training
    range), labels from the exhaustive autotuners, MLPs trained by the library's kernels.
    Regret against exhaustive autotuning is reported for the MLP alone and with the
    fallback (the autotuner run again on the matrix when a feature is out of range or the
    top two predictions are close), with the fallback rate."""
    import torch

    import paper_2604_27985_gb300 as gb
    from paper_2604_27985_gb300 import selector as sel

    n_train, n_test, n_ext = args.selector_train, args.selector_test, args.selector_extrapolate
    specs = ([gen.corpus_spec(i, 5000) for i in range(n_train)] + [gen.corpus_spec(i, 6000) for i in range(n_test)]
             + [gen.extrapolation_spec(i, 7000) for i in range(n_ext)])
    results, t_total = {}, {}
    stream = torch.cuda.current_stream()
    for op in ("spmm", "sddmm"):
        t0 = time.time()
        feats, times = [], []
        for spec in specs:
            rp, ci, v = gen.corpus_matrix(spec)
            f, tm = sel.label(rp, ci, v, spec["n"], spec["N"], spec["dtype"], reps=3, op=op)
            feats.append(f.cpu().numpy())
            times.append(tm)
            del rp, ci, v
        t_label = time.time() - t0
        feats, times = np.stack(feats), np.asarray(times)
        model = sel.Selector(seed=0, op=op, margin=args.selector_margin, gap=args.selector_gap)
        t0 = time.time()
        model.fit(feats[:n_train], times[:n_train], steps=args.selector_steps, batch=64, lr=1e-3)
        torch.cuda.synchronize()
        t_train = time.time() - t0
        evals = {}
        for name, lo, hi in (("held_out", n_train, n_train + n_test), ("extrapolation", n_train + n_test, len(specs))):
            if hi <= lo:
                continue
            mlp, fb, reasons = [], [], {"range": 0, "gap": 0}
            for k in range(lo, hi):
                spec = specs[k]
                rp, ci, _ = gen.corpus_matrix(spec)
                v_mlp = model.choose(rp, ci, spec["n"], spec["N"], spec["dtype"], fallback=False)
                before = dict(model.counts)
                v_fb = model.choose(rp, ci, spec["n"], spec["N"], spec["dtype"], fallback=True)
                for r in reasons:
                    reasons[r] += model.counts[r] - before[r]
                mlp.append(v_mlp)
                fb.append(v_fb)
                del rp, ci
            r_mlp, r_fb = sel.regret(times[lo:hi], mlp), sel.regret(times[lo:hi], fb)
            stat = lambda r: {"mean": float(r.mean()), "p50": float(np.median(r)), "p90": float(np.quantile(r, 0.9)),
                              "max": float(r.max())}
            evals[name] = {"matrices": hi - lo, "regret_mlp_only": stat(r_mlp), "regret_with_fallback": stat(r_fb),
                           "fallback_rate": round((reasons["range"] + reasons["gap"]) / (hi - lo), 4),
                           "fallback_reasons": reasons}
        nv = gb.N_SDDMM_VARIANTS if op == "sddmm" else gb.N_VARIANTS
        fixed_all = [float(np.mean(sel.regret(times[n_train:n_train + n_test], np.full(n_test, v))))
                     for v in range(nv)]
        # time of one selection (features + inference) on a held-out matrix
        spec = specs[n_train]
        rp, ci, _ = gen.corpus_matrix(spec)
        ms_sel = _event_ms(lambda: model.choose(rp, ci, spec["n"], spec["N"], spec["dtype"], fallback=False), 20, 3,
                           stream)
        results[op] = {**evals, "best_single_variant": int(np.argmin(fixed_all)),
                       "best_single_variant_regret_mean": min(fixed_all), "selection_ms": round(ms_sel, 4),
                       "seconds": {"labels": round(t_label, 1), "train": round(t_train, 2)}}
        if args.selector_save:
            base = args.selector_save + ("_sddmm" if op == "sddmm" else "")
            model.save(base, regret_mean=evals["held_out"]["regret_with_fallback"]["mean"],
                       regret_mlp_only_mean=evals["held_out"]["regret_mlp_only"]["mean"], train=n_train, test=n_test)
        t_total[op] = t_label + t_train
    head = results["spmm"]["held_out"]["regret_with_fallback"]["mean"]
    _line("selector regret vs exhaustive autotuning (mean t_chosen/t_best - 1, with fallback)", head, "fraction",
          results["spmm"]["selection_ms"], args, "f32",
          {"workload": f"corpus of {n_train} training + {n_test} held-out matrices (rows log-uniform [4096, 262144], "
                       "sparsity 90/99/99.9%, uniform/power-law/banded/block, N 32..512, FP32/BF16) and "
                       f"{n_ext} held-out 1048576-row matrices (99.99..99.9999%); 24 SpMM variants (incl. row groups "
                       "and the hyper-sparse plan), 9 SDDMM variants",
           "redraws": int(sum(s_["redraws"] for s_ in specs)),
           "fallback": {"margin": args.selector_margin, "gap": args.selector_gap}},
          higher_is_better=False, selectors=results)


def _sub(A, r0, r1):
    p0, p1 = int(A.rowptr[r0]), int(A.rowptr[r1])
    return (A.rowptr[r0:r1 + 1] - p0).astype(np.int32), A.colidx[p0:p1], A.vals[p0:p1]


def cpu_baseline(A, B, X, Y, budget_s=15.0):
    """The FP64 oracle as it stands on the host cores: SpMM and SDDMM over the first R rows
    of the workload (all rows when they fit), repeated until about budget_s seconds."""
    import oracle

    threads = oracle.max_threads()
    Bd, Xd, Yd = B.astype(np.float64), X.astype(np.float64), Y.astype(np.float64)

    def run(r):
        rp, ci, v = _sub(A, 0, r)
        vd = v.astype(np.float64)
        t0 = time.perf_counter()
        oracle.spmm(rp, ci, vd, Bd, threads=threads)
        oracle.sddmm(rp, ci, vd, Xd[:r], Yd, threads=threads)
        return time.perf_counter() - t0, int(rp[-1])

    dt, _ = run(1024)
    r = int(min(M, max(1024, 1024 * budget_s / max(dt, 1e-3))))
    total, work, reps = 0.0, 0.0, 0
    while total < budget_s or reps == 0:
        dt, nz = run(r)
        total += dt
        work += flops(nz)
        reps += 1
    # the small configuration (1,024^2 at 90%, N = Kd = 64) on one thread, mean of 5 runs
    a1 = gen.csr_uniform(1024, 1024, 0.9, seed=0)
    b1, x1, y1 = (gen.dense_normal(1024, 64, 1 + k).astype(np.float64) for k in range(3))
    t1 = []
    for _ in range(5):
        t0 = time.perf_counter()
        oracle.spmm(a1.rowptr, a1.colidx, a1.vals.astype(np.float64), b1, threads=1)
        oracle.sddmm(a1.rowptr, a1.colidx, a1.vals.astype(np.float64), x1, y1, threads=1)
        t1.append(time.perf_counter() - t0)
    return {"value": round(work / total / 1e9, 3), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"rows [0, {r}) of the workload ({nz} nonzeros), FP64 SpMM N={N_SPMM} + SDDMM "
                      f"Kd={KD_SDDMM}, {reps} repetitions in {total:.1f} s", "seconds": round(total, 2),
            "one_thread_1024sq_90pct": {"gflops": round(4.0 * a1.nnz * 64 / np.mean(t1) / 1e9, 3),
                                        "ms": round(1e3 * float(np.mean(t1)), 3),
                                        "sample": "CSR 1024x1024 at 90% (seed 0), SpMM N=64 + SDDMM Kd=64, "
                                                  "mean of 5 runs, 1 thread"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    A, B, X, Y = make_inputs(0)
    threads = oracle.max_threads()
    Bd, Xd, Yd = B.astype(np.float64), X.astype(np.float64), Y.astype(np.float64)
    # size one step's row sample so the whole run stays within about two minutes
    per_step_s = min(5.0, 120.0 / max(1, args.steps + args.warmup))

    def run(r):
        rp, ci, v = _sub(A, 0, r)
        vd = v.astype(np.float64)
        t0 = time.perf_counter()
        oracle.spmm(rp, ci, vd, Bd, threads=threads)
        oracle.sddmm(rp, ci, vd, Xd[:r], Yd, threads=threads)
        return time.perf_counter() - t0, int(rp[-1])

    dt, _ = run(512)
    r = int(min(M, max(512, 512 * per_step_s / max(dt, 1e-3))))
    for _ in range(args.warmup):
        run(r)
    times, nz = [], 0
    for _ in range(args.steps):
        dt, nz = run(r)
        times.append(dt)
    ms = 1e3 * float(np.mean(times))
    value = flops(nz) / (ms / 1e3) / 1e9
    sample = f"rows [0, {r}) of the workload per step ({nz} nonzeros): FP64 oracle SpMM + SDDMM"
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generators; no dataset)",
        "config": {"workload": WORKLOAD, "nnz": A.nnz, "sample_rows": r},
        "cpu_baseline": {"value": round(value, 3), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tuned", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=8)
    ap.add_argument("--e2e-slots", type=int, default=4)
    ap.add_argument("--workload", default="csr65536", choices=["csr65536", "precision", "gnn", "batched", "selector", "sweep", "kbin", "hsp"])
    ap.add_argument("--precision-layouts", default="uniform,clustered")
    ap.add_argument("--gnn-graphs", type=int, default=512)
    ap.add_argument("--gat", action="store_true", help="gnn workload with the row softmax (GAT-style chain)")
    ap.add_argument("--gnn-edges-per-tile", type=int, default=0, help="gnn workload: edges per work tile (0: 512)")
    ap.add_argument("--sweep-dense", action="store_true", help="sweep workload: add 65536^2 at 90%%")
    ap.add_argument("--selector-train", type=int, default=2000)
    ap.add_argument("--selector-test", type=int, default=200)
    ap.add_argument("--selector-steps", type=int, default=6000)
    ap.add_argument("--selector-save", default="")
    ap.add_argument("--selector-extrapolate", type=int, default=24)
    ap.add_argument("--selector-margin", type=float, default=0.1)
    ap.add_argument("--selector-gap", type=float, default=0.02)
    ap.add_argument("--write-traffic", nargs=4, metavar=("SPMM_REPORT", "SPMM_RE", "SDDMM_REPORT", "SDDMM_RE"),
                    help="store per-launch DRAM bytes from ncu reports and exit")
    args = ap.parse_args()
    if args.write_traffic:
        write_traffic(*args.write_traffic)
        return
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "gnn":
        run_gnn(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "selector":
        run_selector(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "kbin":
        run_kbin(args)
    elif args.workload == "hsp":
        run_hsp(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
