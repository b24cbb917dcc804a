"""Host-side parts of the benchmark on CPU: the oracle baseline it prints
(timed steps, parity fields, host description), the CPU description read
from /proc/cpuinfo on both kinds of host, the clock samples it summarises,
and the DRAM traffic it takes from the committed ncu summary only while the
sweep sources match its stamp."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_host_cpu_names_x86_and_arm_models(tmp_path):
    x86 = tmp_path / "x86"
    x86.write_text("processor\t: 0\nvendor_id\t: GenuineIntel\nmodel name\t: Some Xeon\n")
    assert bench.host_cpu(str(x86))["model"] == "Some Xeon"
    arm = tmp_path / "arm"
    arm.write_text("processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\n"
                   "CPU architecture: 8\nCPU part\t: 0xd4f\n")
    assert bench.host_cpu(str(arm))["model"] == "implementer 0x41 part 0xd4f"
    h = bench.host_cpu(str(tmp_path / "missing"))
    assert h["model"] is None and h["nproc"] >= 1 and h["arch"]


def test_cpu_baseline_on_the_headline_workload():
    """One oracle step of the n = 160,000 band matrix, as the bench line's
    cpu_baseline reports it, with the parity fields filled from the oracle's
    own results (so both mismatch counts are 0)."""
    Pb = bench.workload(2)
    F, x, it = bench.oracle_step(Pb)
    cb, parity = bench.cpu_baseline(Pb, 1, F["val"], x)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["unit"] == "ms"
    assert cb["value"] > 0 and cb["host"]["nproc"] >= 1
    assert parity == {"factor_ulp_mismatches": 0, "x_bit_mismatches": 0, "oracle_iters": it}
    assert it == 4  # GMRES(50) with ILU(2) on this matrix
    json.dumps({"cpu_baseline": cb, "parity": parity})


def test_operand_stream_bytes_against_a_loop():
    import numpy as np

    import oracle
    from paper_0803_0048_gb300 import workloads as W
    A = W.random_sparse(120, 0.05, 5)
    F = oracle.factor(A, 2)
    frp, fci, n = F["rowptr"], F["colind"], A.n
    fdg = np.array([frp[i] + np.searchsorted(fci[frp[i]:frp[i + 1]], i) for i in range(n)],
                   dtype=np.int64)
    want = 0
    for i in range(n):
        for p in range(frp[i], fdg[i]):  # lower entries (i, h): row h's strictly upper part
            h = fci[p]
            want += 12 * (frp[h + 1] - fdg[h] - 1)
    assert want > 0
    assert bench.operand_stream_bytes(frp, fci.astype(np.int32), fdg) == want


def test_bench_line_contract_with_stand_ins():
    """bench.ours() end to end on CPU, the CUDA runtime and libiluk replaced
    by stand-ins (tests/stand_in_bench.py): the one JSON line carries every
    key of the contract, and the derived numbers follow from the inputs."""
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "stand_in_bench.py")],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "e2e", "gpu_launches", "clocks", "operand_stream", "kernels"):
        assert key in d, key
    assert d["value"] == 119.0 and d["n_gpus"] == 1 and d["steps"] == 3
    assert d["higher_is_better"] is False and d["dtype"] == "f64"
    assert d["config"]["workload"].startswith("random_band_n160000")
    assert d["gpu_launches"] == 59
    rf = d["roofline"]
    assert rf["kernel"] == "sweep_bwd" and rf["bound"] == "hbm" and rf["unit"] == "GB/s"
    assert abs(rf["achieved"] - rf["alg_bytes_per_launch"] / 11.25e-3 / 1e9) < 1e-3
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-5
    assert abs(rf["nominal_frac"] - rf["achieved"] / 7900.0) < 1e-5
    assert d["e2e"]["h2d_bytes_per_step"] == 160001 * 8 + 1_600_000 * 12 + 160000 * 8
    assert d["e2e"]["d2h_bytes_per_step"] == 160000 * 8
    assert d["e2e"]["call"].startswith("iluk_solve_host")
    assert d["dag"] == {"depth_lower": 15777, "depth_upper": 15629}
    assert set(d["config"]) == {"workload", "n", "nnz_A", "nnz_F", "k", "restart", "rtol", "l2",
                                "parallelism"}
    assert d["operand_stream"]["kernel"] == "factor"
    assert d["operand_stream"]["bytes_per_launch"] > 10 * d["kernels"]["factor"]["alg_bytes_per_launch"]


def test_measured_traffic_only_while_the_sweep_sources_match(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from the committed ncu summary only
    while the sweep kernels' sources are the ones it was captured on."""
    import shutil
    csrc = tmp_path / "paper_0803_0048_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("sweeps.cu", "common.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_0803_0048_gb300", "csrc", f), csrc / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    digest = bench.sources_digest()
    assert len(digest) == 16 and int(digest, 16) >= 0
    prof = tmp_path / "profiles" / "sweep_band160k_k2.md"
    prof.write_text("# summary\n"
                    f"traffic: kernel=sweep_bwd k=2 bytes=123456 sources={digest}\n"
                    f"traffic: kernel=sweep k=2 bytes=777 sources={digest}\n"
                    "traffic: kernel=sweep_bwd k=3 bytes=999 sources=0000000000000000\n")
    assert bench.measured_traffic("sweep_bwd", 2) == 123456
    assert bench.measured_traffic("sweep", 2) == 777
    assert bench.measured_traffic("sweep_bwd", 3) is None  # captured on other sources
    assert bench.measured_traffic("factor", 2) is None     # no line for that kernel
    with open(csrc / "sweeps.cu", "a") as fh:
        fh.write("\n// changed\n")
    assert bench.sources_digest() != digest
    assert bench.measured_traffic("sweep_bwd", 2) is None  # the kernel changed since
    prof.unlink()
    assert bench.measured_traffic("sweep_bwd", 2) is None  # no summary at all


def test_clock_sampler_summary_parses_nvidia_smi_rows():
    """The clocks object of the bench line: median SM clock under load, the
    maximum clock, and every throttle reason seen active; malformed rows (a
    header, a short row, "[N/A]" values) are skipped."""
    c = bench.ClockSampler(0)
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    c.lines = [
        "clocks.current.sm [MHz], clocks.max.sm [MHz], power.draw [W], ...",
        "2070, 2070, 650.1, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1390.5, Not Active, Not Active, Not Active, Active",
        "1995, 2070, 1400.0, Not Active, Not Active, Not Active, Active",
        "[N/A], 2070, 10.0, Not Active, Not Active, Not Active, Not Active",
        "2070, 2070",
        "2070, 2070, 700.0, Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s["samples"] == 4
    assert s["sm_mhz"] == 2062.5 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
