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
                   "paper_2604_27985_gb300/csrc/sddmm.cu", "paper_2604_27985_gb300/csrc/api.cu"]


def sources_sha256(names):
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def write_traffic(report, spmm_re, sddmm_re):
    """Stores per-launch DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the
    SpMM and SDDMM kernels from an ncu report in profiles/traffic.json, stamped with the
    sha256 of the kernel sources: bench lines carry them only while the kernels are
    unchanged."""
    import csv
    import io
    import re

    out = subprocess.run(["ncu", "-i", report, "--page", "raw", "--csv"], capture_output=True, text=True).stdout
    rows = list(csv.reader(io.StringIO(out)))
    hdr, units = rows[0], rows[1]
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}

    def per_launch(pattern):
        vals = []
        for r in rows[2:]:
            d = dict(zip(hdr, r))
            if re.search(pattern, d["Kernel Name"]):
                vals.append(sum(float(d[m].replace(",", "")) * scale[units[hdr.index(m)]]
                                for m in ("dram__bytes_read.sum", "dram__bytes_write.sum")))
        return sum(vals) / len(vals) if vals else None

    t = {"report": os.path.basename(report), "sources": TRAFFIC_SOURCES,
         "sources_sha256": sources_sha256(TRAFFIC_SOURCES),
         "spmm_bytes_per_launch": per_launch(spmm_re), "sddmm_bytes_per_launch": per_launch(sddmm_re)}
    with open(os.path.join(ROOT, "profiles", "traffic.json"), "w") as f:
        json.dump(t, f, indent=1)
    print(json.dumps(t))


def _gather_ceiling(p, nnz, kernel_ms):
    """The kernel's gathered-row bytes per second against the gather probe's on the same
    indices and rows (the level that binds when the gathered operand sits in L2)."""
    achieved = nnz * p["row_bytes"] / (kernel_ms / 1e3) / 1e9
    return {"probe": "gbsp_gather_probe over the workload's colidx", "row_bytes": p["row_bytes"],
            "probe_gbs": p["gbs"], "kernel_gbs": round(achieved, 1), "frac": round(achieved / p["gbs"], 4)}


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
    spmm_gbs = spmm_bytes / (spmm_ms / 1e3) / 1e9
    sddmm_gbs = sddmm_bytes / (sddmm_ms / 1e3) / 1e9
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
        ms_sel = _event_ms(lambda: gb.spmm(rp, ci, v, Bd, out=C, stream=stream, **kw), 50, 5, stream)
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
        "roofline": {"bound": "hbm", "kernel": "spmm (Eq. 1), gather model",
                     "achieved": round(spmm_gbs, 1), "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(spmm_gbs / peak, 4), "traffic": traffic_spmm,
                     "algorithmic_bytes_per_launch": spmm_bytes, "ms_per_launch": round(spmm_ms, 4),
                     "gather_ceiling": _gather_ceiling(probe["spmm"], nnz, spmm_ms)},
        "roofline_sddmm": {"bound": "hbm", "kernel": "sddmm (Eq. 2), gather model",
                           "achieved": round(sddmm_gbs, 1), "peak": peak, "unit": "GB/s",
                           "frac": round(sddmm_gbs / peak, 4), "traffic": traffic_sddmm,
                           "algorithmic_bytes_per_launch": sddmm_bytes, "ms_per_launch": round(sddmm_ms, 4),
                           "gather_ceiling": _gather_ceiling(probe["sddmm"], nnz, sddmm_ms)},
        "roofline_compulsory_spmm": {"bytes": comp, "achieved": round(comp / (spmm_ms / 1e3) / 1e9, 1),
                                     "frac": round(comp / (spmm_ms / 1e3) / 1e9 / peak, 4)},
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


def run_precision(args):
    """16,384^2 at 90%, N = Kd = 256: SpMM + SDDMM in FP32, BF16, E4M3 (CUDA cores) and the
    BF16 / E4M3 condensed-tile tensor-core plans (SpMM and SDDMM), on the uniform and the
    clustered layouts."""
    import torch

    import paper_2604_27985_gb300 as gb

    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    stream = torch.cuda.current_stream()
    peak, _ = peaks()
    forms = {}
    for layout in args.precision_layouts.split(","):
        A = (gen.csr_uniform(16384, 16384, 0.9, seed=2001) if layout == "uniform"
             else gen.csr_clustered(16384, 16384, 0.9, seed=2002))
        B, X, Y = (gen.dense_normal(16384, 256, 2003 + k) for k in range(3))
        rp, ci, v = t(A.rowptr), t(A.colidx), t(A.vals)
        Bd, Xd, Yd = t(B), t(X), t(Y)
        C = torch.empty((A.M, 256), device=dev)
        out = torch.empty(A.nnz, device=dev)
        qa, qb, qx, qy = gb.quantize_bf16(v), gb.quantize_bf16(Bd), gb.quantize_bf16(Xd), gb.quantize_bf16(Yd)
        ea, sa = gb.quantize_e4m3_rows(v, rp)
        eb, sb = gb.quantize_e4m3_rows(Bd)
        ex, ux = gb.quantize_e4m3_rows(Xd)
        ey, uy = gb.quantize_e4m3_rows(Yd)
        plan = gb.TcPlan(rp, ci, qa, A.K)
        plan8 = gb.TcPlan(rp, ci, ea, A.K, row_scale=sa)
        info, info8 = plan.info(), plan8.info()
        runs = {
            "fp32": (lambda: gb.spmm(rp, ci, v, Bd, out=C), lambda: gb.sddmm(rp, ci, v, Xd, Yd, out=out), 4, 4),
            "bf16": (lambda: gb.spmm(rp, ci, qa, qb, out=C), lambda: gb.sddmm(rp, ci, v, qx, qy, out=out), 2, 2),
            "e4m3": (lambda: gb.spmm(rp, ci, ea, eb, out=C, a_scale=sa, b_scale=sb),
                     lambda: gb.sddmm(rp, ci, v, ex, ey, out=out, x_scale=ux, y_scale=uy), 1, 1),
            "tc_bf16": (lambda: plan.execute(qb, out=C), lambda: plan.sddmm(v, qx, qy, out=out), 2, 2),
            "tc_e4m3": (lambda: plan8.execute(eb, out=C, row_scale=sb),
                        lambda: plan8.sddmm(v, ex, ey, out=out, x_scale=ux, y_scale=uy), 1, 1),
        }
        for name, (f_spmm, f_sddmm, vb, eb_) in runs.items():
            ms_a = _event_ms(f_spmm, args.steps, args.warmup, stream)
            ms_b = _event_ms(f_sddmm, args.steps, args.warmup, stream)
            gbytes = (A.nnz * (4 + vb + 256 * eb_) + A.M * (4 + 4 * 256)) / 1e9
            forms[f"{layout}/{name}"] = {
                "spmm_ms": round(ms_a, 4), "sddmm_ms": round(ms_b, 4),
                "spmm_gflops": round(2 * A.nnz * 256 / ms_a / 1e6, 1),
                "sddmm_gflops": round(2 * A.nnz * 256 / ms_b / 1e6, 1),
                "step_gflops": round(4 * A.nnz * 256 / (ms_a + ms_b) / 1e6, 1),
                "spmm_gather_frac": round(gbytes / (ms_a / 1e3) / peak, 3)}
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
           f"fp32_{last}_step_ms": round(base, 4)}, forms=forms)


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
    plan = gb.GnnPlan(devs, softmax=args.gat)
    stream = torch.cuda.current_stream()
    launches0 = gb.launch_count()
    ms = _event_ms(plan.execute, args.steps, args.warmup, stream)
    launches = (gb.launch_count() - launches0) // (args.steps + args.warmup)
    peak, _ = peaks()
    info = plan.info()
    chain = "SDDMM->row softmax->SpMM" if args.gat else "SDDMM->SpMM"
    _line(f"batched {chain} GFLOP/s (4*nnz*N over the batch)", flop / ms / 1e6, "GFLOP/s", ms, args, "bf16",
          {"workload": f"{len(graphs)} of the 512 graphs (nodes log-uniform [1000, 50000], power-law degree "
                       "(mean 16, max 2048), row-normalised values, BF16 features N in {64,128,256}, seed 3000)",
           "softmax": bool(args.gat), **info},
          roofline={"bound": "hbm", "kernel": "gnn_kernel, gather model", "achieved": round(gbytes / ms * 1e3, 1),
                    "peak": peak, "unit": "GB/s", "frac": round(gbytes / ms * 1e3 / peak, 4),
                    "algorithmic_bytes_per_launch": int(gbytes * 1e9)},
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
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
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
                pt = {"n": n, "sparsity": sp, "rows": layout, "op": op, "width": w, "nnz": A.nnz,
                      "ms": round(ms, 4), "gflops": round(f / ms / 1e6, 1),
                      "gather_gbs": round(nbytes / ms / 1e6, 1), "frac": round(nbytes / ms / 1e6 / peak, 4)}
                if op == "spmm":  # the shipped selector's variant for this matrix and width (untimed choice)
                    v_idx = model.choose(rp, ci, n, w, 0)
                    kw = gb.variant_options(v_idx)
                    ms_sel = _event_ms(lambda: gb.spmm(rp, ci, v, Bd, out=C, stream=stream, **kw), args.steps,
                                       args.warmup, stream)
                    ms_mp = _event_ms(lambda: gb.spmm(rp, ci, v, Bd, out=C, stream=stream, variant="merge"),
                                      args.steps, args.warmup, stream)
                    pt.update(selector_variant=v_idx, selector_options=kw, selector_ms=round(ms_sel, 4),
                              selector_frac=round(nbytes / ms_sel / 1e6 / peak, 4), merge_ms=round(ms_mp, 4))
                points.append(pt)
                del fn
        del A, rp, ci, v
        torch.cuda.empty_cache()
    _line("SpMM & SDDMM GFLOP/s (2*nnz*N) over the plain-FP32 scale/sparsity sweep", flop_sum / ms_sum / 1e6,
          "GFLOP/s", ms_sum, args, "f32",
          {"workload": "65536^2 at 99% and 1048576^2 at 99.99%" + (" and 65536^2 at 90%" if args.sweep_dense else "")
                       + ", uniform and power-law rows (Zipf 1.5, cap 4096), values U[-1,1]; SpMM N 32/64/128, "
                       "SDDMM Kd 32/128, dense operands N(0,1); automatic variant; CSR arrays larger than L2",
           "points": points},
          roofline={"bound": "hbm", "kernel": "spmm / sddmm, gather model", "peak": peak, "peak_kind": peak_kind,
                    "unit": "GB/s", "frac_min": min(p["frac"] for p in points),
                    "frac_max": max(p["frac"] for p in points)},
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
        for N in (32, 64, 128):
            Bd = torch.randn((n, N), generator=g, device=dev)
            C = torch.empty((n, N), device=dev)
            f = 2.0 * A.nnz * N
            nbytes = gather_bytes_spmm(A.nnz, n, N)
            pt = {"rows": layout, "N": N, "nnz": A.nnz,
                  "rowsplit_ms": round(_event_ms(lambda: gb.spmm(rp, ci, v, Bd, out=C, stream=stream), args.steps,
                                                 args.warmup, stream), 4),
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
                    pt.update(kbin_ms=round(ms, 4), slices=plan.info()["slices"], gflops=round(f / ms / 1e6, 1),
                              gather_gbs=round(nbytes / ms / 1e6, 1), frac=round(nbytes / ms / 1e6 / peak, 4),
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
          roofline={"bound": "hbm", "kernel": "kbin_pass_kernel, gather model", "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac_min": min(p["frac"] for p in points),
                    "frac_max": max(p["frac"] for p in points)},
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
            points.append({"n": n, "sparsity": sp, "rows": layout, "N": N, "nnz": A.nnz, **plan.info(),
                           "hsp_ms": round(ms, 4), "gflops": round(f / ms / 1e6, 1),
                           "gather_gbs": round(nbytes / ms / 1e6, 1), "frac": round(nbytes / ms / 1e6 / peak, 4),
                           "rowsplit_ms": t(lambda: gb.spmm(rp, ci, v, Bd, out=C, stream=stream)),
                           "merge_ms": t(lambda: gb.spmm(rp, ci, v, Bd, out=C, variant="merge", stream=stream))})
            del Bd, C
        plan.close()
        del A, rp, ci, v
        torch.cuda.empty_cache()
    _line("hyper-sparse SpMM GFLOP/s (2*nnz*N)", flop_sum / ms_sum / 1e6, "GFLOP/s", ms_sum, args, "f32",
          {"workload": "1048576^2 at 99.9999%, 262144^2 at 99.999%, 65536^2 at 99.99% (uniform rows) and 262144^2 "
                       "at 99.99% (power-law rows), values U[-1,1], B N(0,1) FP32, N 32/64/128",
           "l2": "flushed before every timed call (256 MB written)", "points": points},
          roofline={"bound": "hbm", "kernel": "hsp_kernel, gather model", "peak": peak, "peak_kind": peak_kind,
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
    """Learned selector: 2,000 training and 200 held-out corpus matrices, labels from the
    exhaustive autotuner, the MLP trained by the library's kernels; regret vs exhaustive."""
    import torch

    import paper_2604_27985_gb300 as gb
    from paper_2604_27985_gb300 import selector as sel

    n_train, n_test = args.selector_train, args.selector_test
    feats, times, specs = [], [], []
    t_label = time.time()
    for i in range(n_train + n_test):
        spec = gen.corpus_spec(i, 5000 if i < n_train else 6000)
        rp, ci, v = gen.corpus_matrix(spec)
        f, tm = sel.label(rp, ci, v, spec["n"], spec["N"], spec["dtype"], reps=3)
        feats.append(f.cpu().numpy())
        times.append(tm)
        specs.append(spec)
    t_label = time.time() - t_label
    feats, times = np.stack(feats), np.asarray(times)
    model = sel.Selector(seed=0)
    t0 = time.time()
    model.fit(feats[:n_train], times[:n_train], steps=args.selector_steps, batch=64, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    _, choice = model.predict(feats[n_train:])
    r = sel.regret(times[n_train:], choice.cpu().numpy())
    fixed_all = [float(np.mean(sel.regret(times[n_train:], np.full(n_test, v)))) for v in range(gb.N_VARIANTS)]
    fixed = {"best_single_variant": int(np.argmin(fixed_all)), "best_single_mean": min(fixed_all),
             "rowsplit_v2_u4": fixed_all[4], "merge_v2_u4": fixed_all[13]}
    # time of one selection (features + inference) on a held-out matrix
    spec = specs[n_train]
    rp, ci, v = gen.corpus_matrix(spec)
    ms_sel = _event_ms(lambda: model.choose(rp, ci, spec["n"], spec["N"], spec["dtype"]), 20, 3,
                       torch.cuda.current_stream())
    if args.selector_save:
        model.save(args.selector_save, regret_mean=float(r.mean()), regret_p90=float(np.quantile(r, 0.9)),
                   regret_max=float(r.max()), train=n_train, test=n_test)
    _line("selector regret vs exhaustive autotuning (mean t_chosen/t_best - 1)", float(r.mean()), "fraction",
          ms_sel, args, "f32",
          {"workload": f"corpus of {n_train} training + {n_test} held-out matrices (rows log-uniform "
                       "[4096, 262144], sparsity 90/99/99.9%, uniform/power-law/banded/block, N 32..512, "
                       "FP32/BF16), 24 SpMM variants", "redraws": int(sum(s["redraws"] for s in specs))},
          higher_is_better=False, regret={"mean": float(r.mean()), "p50": float(np.median(r)),
                                          "p90": float(np.quantile(r, 0.9)), "max": float(r.max()),
                                          "fixed_choices_mean": fixed},
          seconds={"labels": round(t_label, 1), "train": round(t_train, 2)}, selection_ms=round(ms_sel, 4))


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
    ap.add_argument("--sweep-dense", action="store_true", help="sweep workload: add 65536^2 at 90%%")
    ap.add_argument("--selector-train", type=int, default=2000)
    ap.add_argument("--selector-test", type=int, default=200)
    ap.add_argument("--selector-steps", type=int, default=6000)
    ap.add_argument("--selector-save", default="")
    ap.add_argument("--write-traffic", nargs=3, metavar=("REPORT", "SPMM_RE", "SDDMM_RE"),
                    help="store per-launch DRAM bytes from an ncu report and exit")
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
