"""Throughput of the CSR SpMM + SDDMM hot path on one GB300 (or N replicas).

One step = one SpMM (Eq. 1, N = 64) and one SDDMM (Eq. 2, Kd = 32) over a 65,536 x 65,536
CSR matrix at 99% sparsity (42,949,673 nonzeros, uniform rows, seed 1001), FP32, inputs
resident in HBM.  The CSR arrays alone (344 MB) exceed the 129 MB L2, so no flush is
needed between steps.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores (a bounded row sample of the
same workload per step) and prints the same line with "impl": "reference".
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

    # end to end through the public API with host buffers: pinned host -> device copies of
    # this step's inputs, the two calls, device -> pinned host copies of both results.
    h_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (A.rowptr, A.colidx, A.vals, B, X, Y)]
    d_in = [torch.empty_like(h, device=dev) for h in h_in]
    h_C = torch.empty((M, N_SPMM), dtype=torch.float32).pin_memory()
    h_out = torch.empty(nnz, dtype=torch.float32).pin_memory()
    h2d = sum(h.numel() * h.element_size() for h in h_in)
    d2h = h_C.numel() * 4 + h_out.numel() * 4

    def e2e_step():
        for d, h in zip(d_in, h_in):
            d.copy_(h, non_blocking=True)
        drp, dci, dv, dB, dX, dY = d_in
        gb.spmm(drp, dci, dv, dB, out=C, stream=stream)
        gb.sddmm(drp, dci, dv, dX, dY, out=out, stream=stream)
        h_C.copy_(C, non_blocking=True)
        h_out.copy_(out, non_blocking=True)

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
        tt = torch.tensor([ms, e2e_ms, spmm_ms, sddmm_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms, e2e_ms, spmm_ms, sddmm_ms = tt.tolist()
    gflop = flops(nnz) / 1e9
    value = world * gflop / (ms / 1e3)
    peak, peak_kind = peaks()
    spmm_bytes = gather_bytes_spmm(nnz, M, N_SPMM)
    sddmm_bytes = gather_bytes_sddmm(nnz, M, KD_SDDMM)
    spmm_gbs = spmm_bytes / (spmm_ms / 1e3) / 1e9
    sddmm_gbs = sddmm_bytes / (sddmm_ms / 1e3) / 1e9
    traffic_spmm, traffic_sddmm = kernel_traffic()
    comp = compulsory_bytes_spmm(nnz, M, K, N_SPMM)

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
                     "algorithmic_bytes_per_launch": spmm_bytes, "ms_per_launch": round(spmm_ms, 4)},
        "roofline_sddmm": {"bound": "hbm", "kernel": "sddmm (Eq. 2), gather model",
                           "achieved": round(sddmm_gbs, 1), "peak": peak, "unit": "GB/s",
                           "frac": round(sddmm_gbs / peak, 4), "traffic": traffic_sddmm,
                           "algorithmic_bytes_per_launch": sddmm_bytes, "ms_per_launch": round(sddmm_ms, 4)},
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
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _sub(A, r0, r1):
    p0, p1 = int(A.rowptr[r0]), int(A.rowptr[r1])
    return (A.rowptr[r0:r1 + 1] - p0).astype(np.int32), A.colidx[p0:p1], A.vals[p0:p1]


def cpu_baseline(A, B, X, Y, budget_s=15.0):
    """The FP64 oracle as it stands on the host cores, on the first R rows of the workload
    (SpMM and SDDMM), R chosen so the timed run takes about budget_s seconds."""
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
    dt, nz = run(r)
    return {"value": round(flops(nz) / dt / 1e9, 3), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "sample": f"rows [0, {r}) of the workload ({nz} nonzeros): FP64 SpMM N={N_SPMM} + SDDMM Kd={KD_SDDMM}, "
                      f"{dt:.1f} s", "seconds": round(dt, 2)}


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
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
