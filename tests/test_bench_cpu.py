"""The benchmark's host-side parts on CPU: the byte and FLOP models against the per-unit
figures written out by hand, and the reference arm (the FP64 oracle timed on the host
cores) end to end, including a non-zero rank that must exit without work."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_byte_and_flop_models():
    import bench

    nnz, M, N, Kd = 42_949_673, 65_536, 64, 32
    # SpMM: per nonzero index + value + one B row (N floats); per row one row pointer + one C row
    assert bench.gather_bytes_spmm(nnz, M, N) == nnz * (4 + 4 + 4 * N) + M * (4 + 4 * N) == 11_355_753_032
    # SDDMM: per nonzero index + value + output + one Y row; per row one row pointer + one X row
    assert bench.gather_bytes_sddmm(nnz, M, Kd) == nnz * (4 + 4 + 4 + 4 * Kd) + M * (4 + 4 * Kd) == 6_021_604_972
    # every operand once: rowptr, colidx + vals, B, C
    assert bench.compulsory_bytes_spmm(nnz, M, M, N) == 4 * (M + 1) + 8 * nnz + 4 * M * N * 2 == 377_413_964
    assert bench.flops(nnz) == 2 * nnz * N + 2 * nnz * Kd
    # BF16 operands halve the gathered rows
    assert bench.gather_bytes_spmm(10, 1, 64, v=2, e=2) == 10 * (4 + 2 + 128) + (4 + 256)


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_other_rank_exits_without_work():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_line():
    r = _run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GFLOP/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["nnz"] == 42_949_673


def test_l2_roofline_fields():
    """The L2 roof holds the gathered-row bytes of one launch against the gather probe, and
    reports the HBM fraction on compulsory bytes beside it (figures from one GB300 run:
    SpMM 0.515 ms, probe 21,187.7 GB/s over 256-byte rows)."""
    import bench

    nnz = 42_949_673
    r = bench.l2_roofline("spmm", nnz, 256, 21187.7, 0.515, 6663.2, "measured", 377_413_964, 11_355_753_032, None)
    assert r["bound"] == "l2" and r["unit"] == "GB/s" and r["peak"] == 21187.7
    assert r["algorithmic_bytes_per_launch"] == nnz * 256
    assert abs(r["achieved"] - 21349.6) < 0.2 and abs(r["frac"] - 1.0076) < 1e-4
    assert abs(r["hbm"]["achieved"] - 732.8) < 0.1 and abs(r["hbm"]["frac"] - 0.11) < 1e-3
    # every fraction is a fraction of the peak it names
    assert r["frac"] == round(r["achieved"] / r["peak"], 4)
    # SDDMM compulsory bytes: row pointers, index + value + output per entry, X and Y once
    assert bench.compulsory_bytes_sddmm(nnz, 65_536, 65_536, 32) == 4 * 65_537 + 12 * nnz + 2 * 65_536 * 32 * 4
