#!/usr/bin/env python
"""Benchmark of the ILU(k)-preconditioned solve on one GB300.

Workload (default): the random banded non-symmetric system with n = 160,000
rows, 9 off-diagonals per row inside |j - i| <= 2000, values uniform in
[-1, 1] and diagonal 1.2 * sum |a_ij|, b = A x* for a uniform x*.  One step is
one pass of the whole hot path on it: pattern check + symbolic ILU(2) +
numeric ILU(2) (one launch, iluk_factor) + right-preconditioned GMRES(50) with
the ILU(2) sweeps to a 1e-8 relative residual, all in libiluk's kernels.

Printed: one JSON line with ms per step (device-timed, inputs resident in
HBM), the same measured end to end from pinned host buffers, the roofline of
the dominant kernel, the sequential CPU oracle as a baseline, clocks sampled
during the timed region, and per-phase times.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--k 2] [--impl reference]

With --impl reference the arm timed is the sequential oracle (C, one host
core) on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ILU(k) factor+apply ms & HBM GB/s (% peak); batched/adjoint vs plain, 1e-8 res"
L2_BYTES = 129 * 1024 * 1024
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal


def host_cpu(cpuinfo="/proc/cpuinfo"):
    """The host the CPU baseline ran on: architecture, CPU model (when
    /proc/cpuinfo names one) and the number of cores."""
    import platform
    fields = {}
    try:
        with open(cpuinfo) as f:
            for line in f:
                key, _, val = line.partition(":")
                fields.setdefault(key.strip().lower(), val.strip())
    except OSError:
        pass
    model = fields.get("model name") or fields.get("cpu model")
    if not model and "cpu part" in fields:  # Arm: implementer and part numbers
        model = f"implementer {fields.get('cpu implementer', '?')} part {fields['cpu part']}"
    return {"arch": platform.machine(), "model": model or None, "nproc": os.cpu_count()}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--k", type=int, default=2)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=2, help="oracle steps for cpu_baseline")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--workload", default="band",
                    choices=["band", "batched", "adjoint", "suite", "ratio"],
                    help="band: the n=160,000 headline; batched: 512 value sets on 32^3 plus "
                         "64 uneven grids in one launch; adjoint: 256^2 differentiable solve; "
                         "suite: every phase of every single-system configuration")
    ap.add_argument("--nsets", type=int, default=512)
    ap.add_argument("--ngrids", type=int, default=64)
    ap.add_argument("--batch-schedule", default="auto",
                    help="batched: 'auto' (the autotuner) or WIDTH/spin or WIDTH/level, "
                         "e.g. 512/spin, fixed before the first solve")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(k):
    from paper_0803_0048_gb300 import workloads as W
    return W.random_band_160k(k=k)


def workload_config(Pb, nnzF, world):
    """The config dict both arms print: the workload and its sizes."""
    return {"workload": f"random_band_n{Pb.A.n}_hw2000_k{Pb.k}_gmres{Pb.restart}_rtol1e-8",
            "n": Pb.A.n, "nnz_A": Pb.A.nnz, "nnz_F": int(nnzF), "k": Pb.k,
            "restart": Pb.restart, "rtol": Pb.rtol,
            "l2": f"inputs larger than L2: F is {(12 * nnzF) / 2**20:.0f} MiB > 129 MiB",
            "parallelism": "replicas" if world > 1 else "single"}


def alg_bytes(n, nnzA, nnzF, nnzL):
    """Compulsory bytes per launch of each kernel kind (each array touched once)."""
    nnzU = nnzF - nnzL
    return {
        # A values + A->F map + both row-pointer arrays + F columns + diagonal + F values out
        "numeric": 12 * nnzA + 16 * (n + 1) + 4 * nnzF + 8 * n + 8 * nnzF,
        # read A pattern, write F pattern + levels via the arena, diagonal
        "symbolic": 8 * (n + 1) + 4 * nnzA + 5 * nnzF,
        # forward sweep: F's strictly lower half (cols + vals), row pointers, diagonal
        # positions, the input read, the output written, the next buffer re-armed
        "sweep": 12 * nnzL + 8 * (n + 1) + 8 * n + 24 * n,
        # backward sweep: F's upper half with the diagonal, the same vectors, and the
        # diagonal with its fixed-point reciprocals (16 bytes per row)
        "sweep_bwd": 12 * nnzU + 8 * (n + 1) + 8 * n + 24 * n + 16 * n,
        "spmv": 12 * nnzA + 8 * (n + 1) + 16 * n,
        # symbolic and numeric in one launch: the two phases' bytes
        "factor": (8 * (n + 1) + 4 * nnzA + 5 * nnzF)
        + (12 * nnzA + 16 * (n + 1) + 4 * nnzF + 8 * n + 8 * nnzF),
    }


def operand_stream_bytes(frp, fci, fdg):
    """Bytes of pivot rows the numeric phase streams, re-reads included: for
    every lower entry (i, h) of F, row h's strictly upper part (a 4-byte column
    and an 8-byte value per entry).  Against the compulsory bytes it shows how
    much of the pivot-row traffic L2 has to absorb."""
    frp = np.asarray(frp, dtype=np.int64)
    fci = np.asarray(fci, dtype=np.int64)
    fdg = np.asarray(fdg, dtype=np.int64)
    n = fdg.size
    ustrict = frp[1:] - fdg - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(frp))
    lower = fci < rows
    return int(12 * ustrict[fci[lower]].sum())


def sources_digest():
    """Digest of the sweep kernels' sources, as stamped on measured traffic."""
    import hashlib
    h = hashlib.sha256()
    for f in ("sweeps.cu", "common.cuh"):
        with open(os.path.join(ROOT, "paper_0803_0048_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kind, k):
    """DRAM bytes per launch of `kind` from the committed ncu summary, or None
    when there is none or the kernel sources changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "sweep_band160k_k2.md")
    if not os.path.exists(path):
        return None
    digest = sources_digest()
    for line in open(path):
        if not line.startswith("traffic:"):
            continue
        f = dict(x.split("=", 1) for x in line.split()[1:])
        if f.get("kernel") == kind and f.get("k") == str(k) and f.get("sources") == digest:
            return int(f["bytes"])
    return None


def ranks_max(values, dev, world):
    """Each value's maximum over the ranks of the process group (a plain copy
    when world == 1).  Backend-agnostic: dev is the device the backend reduces
    on (cuda for NCCL, cpu for gloo)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def ours(args):
    import torch
    import torch.distributed as dist

    import paper_0803_0048_gb300 as P
    from paper_0803_0048_gb300 import _lib as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    Pb = workload(args.k)
    A = Pb.A
    n, nnzA = A.n, A.nnz
    rp = torch.from_numpy(A.rowptr).to(dev)
    ci = torch.from_numpy(A.colind).to(dev)
    av = torch.from_numpy(A.val).to(dev)
    b = torch.from_numpy(Pb.b).to(dev)
    stream = torch.cuda.current_stream()

    sched = [L.SCHED_AUTO]

    def step(rp_, ci_, av_, b_):
        # one C call (iluk_solve): pattern check; v_1 = b / ||b||; symbolic and
        # numeric phases in one launch (the numeric rows start as soon as
        # their patterns are final, and each factored row also takes its
        # entry of L^-1 v_1); GMRES, whose first application then needs only
        # the backward sweep
        x, info, (S, F) = P.solve(rp_, ci_, av_, b_, k=Pb.k, restart=Pb.restart, rtol=Pb.rtol,
                                  sched=sched[0], return_factors=True)
        return S, F, x, info

    # warm-up (the first apply times both sweep schedules; keep its choice)
    for _ in range(max(args.warmup, 1)):
        S, F, x, info = step(rp, ci, av, b)
        sched[0] = F.schedule()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # device-timed region: inputs resident in HBM (F alone is larger than L2)
    launches0 = P.launch_count()
    P.prof_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            S, F, x, info = step(rp, ci, av, b)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = P.prof_read()
    P.prof_enable(False)
    launches = (P.launch_count() - launches0) // args.steps

    # end to end through the C ABI's host-buffer call (iluk_solve_host): the
    # inputs cross from pinned host memory and x comes back inside each call
    h_rp = torch.from_numpy(A.rowptr).pin_memory()
    h_ci = torch.from_numpy(A.colind).pin_memory()
    h_av = torch.from_numpy(A.val).pin_memory()
    h_b = torch.from_numpy(Pb.b).pin_memory()
    h_x = torch.empty(n, dtype=torch.float64).pin_memory()
    P.solve_host(h_rp, h_ci, h_av, h_b, Pb.k, Pb.restart, Pb.rtol, sched=sched[0], x=h_x)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, info2 = P.solve_host(h_rp, h_ci, h_av, h_b, Pb.k, Pb.restart, Pb.rtol,
                                sched=sched[0], x=h_x)
    e1.record(stream)
    barrier()
    ms_e2e = e0.elapsed_time(e1) / args.steps
    e2e_bits_equal = bool(torch.equal(h_x.view(torch.int64), x.cpu().view(torch.int64)))
    # every replica runs the same step: the slowest one sets both times
    ms, ms_e2e = ranks_max([ms, ms_e2e], dev, world)
    h2d = h_rp.numel() * 8 + h_ci.numel() * 4 + h_av.numel() * 8 + h_b.numel() * 8
    d2h = n * 8

    # structure of the factors (for the roofline numerators)
    frp, fci, flev, fdg = [t.cpu().numpy() for t in S.pattern()]
    nnzF = int(frp[-1])
    nnzL = int(np.sum(fdg - frp[:-1]))
    depth = S.depth()
    ab = alg_bytes(n, nnzA, nnzF, nnzL)
    hbm, peak_src = measured_peaks()
    kinds = {"numeric": "numeric", "symbolic": "symbolic", "sweep": "sweep",
             "sweep_bwd": "sweep_bwd", "spmv": "spmv", "factor": "factor"}
    per_kind = {}
    for kname, (tot_ms, cnt) in prof.items():
        if cnt:
            per_kind[kname] = {"ms_total_per_step": tot_ms / args.steps,
                               "launches_per_step": cnt / args.steps,
                               "ms_per_launch": tot_ms / cnt}
    # per phase: algorithmic GB/s, fraction of the measured HBM peak, and the time
    # per level of the dependency DAG the phase walks (its critical path)
    levels_of = {"symbolic": depth[0], "numeric": depth[0], "sweep": depth[0],
                 "sweep_bwd": depth[1], "factor": depth[0]}
    for kname, rec in per_kind.items():
        if kname in kinds:
            gbps = ab[kinds[kname]] / (rec["ms_per_launch"] / 1e3) / 1e9
            rec["alg_bytes_per_launch"] = ab[kinds[kname]]
            rec["alg_GBps"] = round(gbps, 3)
            rec["hbm_frac"] = round(gbps / hbm, 6)
        if kname in levels_of and levels_of[kname] > 0:
            rec["levels"] = levels_of[kname]
            rec["ns_per_level"] = round(rec["ms_per_launch"] * 1e6 / levels_of[kname], 1)
    dom = max((k for k in per_kind if k in kinds), key=lambda k: per_kind[k]["ms_total_per_step"])
    dur_s = per_kind[dom]["ms_per_launch"] / 1e3
    achieved = ab[kinds[dom]] / dur_s / 1e9
    traffic = measured_traffic(dom, Pb.k)
    ob = operand_stream_bytes(frp, fci, fdg)
    kn = "factor" if "factor" in per_kind else "numeric" if "numeric" in per_kind else None

    out = {
        "metric": METRIC, "value": round(ms, 4), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(Pb, nnzF, world),
        "dag": {"depth_lower": depth[0], "depth_upper": depth[1]},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 3), "peak": hbm,
                     "unit": "GB/s", "frac": round(achieved / hbm, 6), "traffic": traffic,
                     "alg_bytes_per_launch": ab[kinds[dom]], "peak_source": peak_src,
                     "nominal_peak": HBM_NOMINAL_GBS,
                     "nominal_frac": round(achieved / HBM_NOMINAL_GBS, 6)},
        "e2e": {"value": round(ms_e2e, 4), "unit": "ms", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "call": "iluk_solve_host (host buffers)",
                "x_bits_equal_device_run": e2e_bits_equal},
        "operand_stream": {"kernel": kn, "bytes_per_launch": ob,
                           "GBps": (round(ob / (per_kind[kn]["ms_per_launch"] / 1e3) / 1e9, 3)
                                    if kn else None)},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "gmres": {"iters": info.iters, "relres": info.relres,
                  "sweep_schedule": {"forward": L.sched_name(sched[0] & 0xff),
                                     "backward": L.sched_name((sched[0] >> 8) & 0xff)}},
        "kernels": per_kind,
    }

    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"], parity = cpu_baseline(Pb, args.cpu_steps, F.values().cpu().numpy(),
                                                   x.cpu().numpy())
        out["parity"] = parity
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def oracle_step(Pb):
    import oracle
    A = Pb.A
    st, bad = oracle.check_pattern(A.n, A.rowptr, A.colind)
    F = oracle.factor(A, Pb.k)
    st, x, it, rel, _ = oracle.gmres(A.n, A.rowptr, A.colind, A.val, Pb.b, oracle.PREC_ILU,
                                     (F["rowptr"], F["colind"], F["val"]), Pb.restart, Pb.rtol,
                                     dotmode=oracle.DOT_TREE)
    return F, x, it


def cpu_baseline(Pb, steps, fv_gpu=None, x_gpu=None):
    import oracle
    oracle.build()
    ts = []
    for _ in range(max(steps, 1)):
        t0 = time.perf_counter()
        F, x, it = oracle_step(Pb)
        ts.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.median(ts)
    parity = None
    if fv_gpu is not None:
        fo = F["val"]
        parity = {"factor_ulp_mismatches": int(np.sum(fo.view(np.int64) != fv_gpu.view(np.int64))),
                  "x_bit_mismatches": int(np.sum(x.view(np.int64) != x_gpu.view(np.int64))),
                  "oracle_iters": it}
    return ({"value": round(ms, 2), "unit": "ms", "cores": 1, "kind": "oracle",
             "sample": f"{len(ts)} full steps (pattern check + symbolic + numeric + GMRES, "
                       f"fixed-tree dots) of the same workload, median",
             "host": host_cpu()}, parity)


def reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    Pb = workload(args.k)
    for _ in range(args.warmup):
        F, _, _ = oracle_step(Pb)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        F, _, _ = oracle_step(Pb)
        ts.append(time.perf_counter() - t0)
    ms = 1e3 * sum(ts) / len(ts)
    out = {"impl": "reference", "metric": METRIC, "value": round(ms, 3), "unit": "ms",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(Pb, F["rowptr"][-1], world),
           "cpu_baseline": {"value": round(ms, 3), "unit": "ms", "cores": 1, "kind": "oracle",
                            "sample": "each step one full oracle pass of the workload",
                            "host": host_cpu()},
           "e2e": {"value": round(ms, 3), "unit": "ms", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def batched(args):
    """512 value sets on one 32^3 7-point pattern + 64 uneven grids 16^3-40^3,
    ILU(1) factor + GMRES(30) to 1e-8, all in one persistent launch; against
    looping the single-instance path (iluk_numeric + gmres_solve) over the same
    items on the same GPU.  Under torchrun the items are partitioned across
    the ranks by estimated work (shard.partition): each GPU solves its share
    in its own launch, nothing crosses GPUs, the per-item results are
    gathered on rank 0, and the time is the slowest rank's (strong scaling:
    the batch is fixed)."""
    import torch
    import torch.distributed as dist

    import paper_0803_0048_gb300 as P
    from paper_0803_0048_gb300 import shard
    from paper_0803_0048_gb300 import workloads as W
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    A0, vals, bs, _ = W.batched_values(args.nsets, 32)
    grids = W.uneven_grids(args.ngrids)
    rp = torch.from_numpy(A0.rowptr).to(dev)
    ci = torch.from_numpy(A0.colind).to(dev)
    S0 = P.symbolic(rp, ci, 1)
    # every rank builds every pattern's symbolic handle (cheap) to cost the items
    pats = [(S0, rp, ci)] * args.nsets
    for g in grids:
        r = torch.from_numpy(g.A.rowptr).to(dev)
        c = torch.from_numpy(g.A.colind).to(dev)
        pats.append((P.symbolic(r, c, 1), r, c))
    costs = [shard.item_cost(S.n, *S.depth()) for S, _, _ in pats]
    parts = shard.partition(costs, world)
    mine = parts[rank]
    items, plain = [], []
    for idx in mine:
        S, r, c = pats[idx]
        if idx < args.nsets:
            v = torch.from_numpy(vals[idx]).to(dev)
            b = torch.from_numpy(bs[idx]).to(dev)
        else:
            g = grids[idx - args.nsets]
            v = torch.from_numpy(g.A.val).to(dev)
            b = torch.from_numpy(g.b).to(dev)
        items.append((S, v, b, torch.empty(S.n, dtype=torch.float64, device=dev)))
        plain.append((S, r, c, v, b))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    B = P.BatchSolve(items, restart=30, rtol=1e-8)
    if args.batch_schedule != "auto":
        width, kind = args.batch_schedule.split("/")
        B.set_schedule(int(width), kind == "spin")
    for _ in range(max(args.warmup, 1)):
        B.solve()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            B.solve()
        ev1.record()
        barrier()
    ms_local = ev0.elapsed_time(ev1) / args.steps
    res = B.results()
    chosen = (B.width(), B.spin())
    # every schedule the autotuner chooses from, one timed run each
    sched_ms = {}
    for sp in (False, True):
        for w in (256, 512, 1024):
            B.set_schedule(w, sp)
            B.solve()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            B.solve()
            e1.record()
            torch.cuda.synchronize()
            sched_ms[f"{w}/{'spin' if sp else 'level'}"] = round(e0.elapsed_time(e1), 3)
    B.set_schedule(*chosen)
    B.solve()
    res = B.results()
    # the same items, one at a time through the single-instance path; the
    # results are compared after the timed loop
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    loop_out = []
    t0.record()
    for (S, r, c, v, b) in plain:
        F = P.numeric(S, v)
        x, info = P.gmres(r, c, v, b, F, restart=30, rtol=1e-8, check=False)
        loop_out.append((x, info.iters))
    t1.record()
    barrier()
    loop_local = t0.elapsed_time(t1)
    mism = 0
    for (x, iters), (_, _, _, xb), rr in zip(loop_out, items, res):
        mism += int((x.view(torch.int64) != xb.view(torch.int64)).sum().item())
        mism += int(iters != rr.iters)
    ms, loop_ms, mism_max = ranks_max([ms_local, loop_local, mism], dev, world)
    merged = shard.gather_results(
        [(idx, (r.status, r.iters, r.cycles, r.relres)) for idx, r in zip(mine, res)],
        len(pats), rank, world)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    out = {"metric": METRIC, "value": round(ms, 3), "unit": "ms", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
           "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": f"batched_{args.nsets}x32^3_plus_{args.ngrids}_uneven_k1_gmres30",
                      "items": len(pats), "width": chosen[0],
                      "sweeps": "spin" if chosen[1] else "level",
                      "parallelism": f"items partitioned over {world} GPU(s)" if world > 1
                      else "single"},
           "partition": {"items_per_rank": [len(p) for p in parts],
                         "est_work_per_rank": shard.loads(costs, parts)},
           "schedules_ms": sched_ms,
           "loop_single_path_ms": round(loop_ms, 3),
           "speedup_vs_loop": round(loop_ms / ms, 2),
           "bit_mismatches_vs_single": int(mism_max),
           "max_iters": max(r[1] for r in merged),
           "all_converged": all(r[0] == 0 for r in merged),
           "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def adjoint(args):
    """2D 256^2 diffusion-convection with per-cell theta: x = A(theta)^-1 b by
    ILU(2)-GMRES(30) to 1e-8, L = ||x - x_t||^2, dL/dtheta and dL/db by the
    adjoint (the forward's factors reused, transposed).

    Two arms of the plain single-instance path on the same GPU, both timed:
    * plain gradient: the same gradient by plain calls without factor reuse --
      numeric ILU(2) of A, GMRES for x, then the explicit A^T (iluk_transpose),
      its own numeric ILU(2) (its symbolic phase, and with it the sweep
      schedule tuned on the pattern, kept from an untimed first call: the
      most favourable case for the plain path), GMRES for lambda, the
      -lambda_i x_j scatter and autograd through the assembly;
    * finite-difference loop: central differences need 2 n_theta plain
      solves (numeric + GMRES); a sample of them is timed and the loop's time
      is extrapolated from the measured mean (labelled as such)."""
    import torch

    import paper_0803_0048_gb300 as P
    from paper_0803_0048_gb300 import workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    Pt, theta, beta, b, xt = W.adjoint_problem(256)
    rp = torch.from_numpy(Pt.rowptr).to(dev)
    ci = torch.from_numpy(Pt.colind).to(dev)
    solver = P.IlukSolver(rp, ci, k=2, restart=30, rtol=1e-8)
    bd = torch.from_numpy(b).to(dev)
    xtd = torch.from_numpy(xt).to(dev)
    th0 = torch.from_numpy(theta).to(dev)

    def fwd_bwd():
        th = th0.clone().requires_grad_(True)
        bb = bd.clone().requires_grad_(True)
        x = solver.solve(W.fd_values(Pt, th, beta), bb)
        L = ((x - xtd) ** 2).sum()
        L.backward()
        return th.grad, bb.grad

    def fwd_only():
        with torch.no_grad():
            return solver.solve(W.fd_values(Pt, th0, beta), bd)

    # the plain path: A^T's pattern and symbolic phase fixed once
    v0 = W.fd_values(Pt, th0, beta).detach()
    trp, tci, _ = P.transpose(rp, ci, v0)
    St = P.symbolic(trp, tci, 2)
    plain_info = {}

    def plain_gradient():
        th = th0.clone().requires_grad_(True)
        vals = W.fd_values(Pt, th, beta)
        v = vals.detach()
        F = P.numeric(solver.S, v)
        x, info = P.gmres(rp, ci, v, bd, F, restart=30, rtol=1e-8)
        _, _, tv = P.transpose(rp, ci, v)
        Ft = P.numeric(St, tv)
        lam, info_t = P.gmres(trp, tci, tv, 2.0 * (x - xtd), Ft, restart=30, rtol=1e-8)
        gA = P.adjoint_scatter(rp, ci, lam, x)
        (gth,) = torch.autograd.grad(vals, th, grad_outputs=gA)
        plain_info["iters"] = (info.iters, info_t.iters)
        return gth, lam

    def plain_solve(th):
        v = W.fd_values(Pt, th, beta)
        F = P.numeric(solver.S, v)
        return P.gmres(rp, ci, v, bd, F, restart=30, rtol=1e-8)[0]

    for _ in range(max(args.warmup, 1)):
        fwd_bwd()
        fwd_only()
        plain_gradient()
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with ClockSampler(0) as clk:
        e[0].record()
        for _ in range(args.steps):
            fwd_bwd()
        e[1].record()
        for _ in range(args.steps):
            fwd_only()
        e[2].record()
        for _ in range(args.steps):
            plain_gradient()
        e[3].record()
        torch.cuda.synchronize()
    ms_fb = e[0].elapsed_time(e[1]) / args.steps
    ms_f = e[1].elapsed_time(e[2]) / args.steps
    ms_plain = e[2].elapsed_time(e[3]) / args.steps
    # agreement of the two gradients (different preconditioners for A^T,
    # both solved to 1e-8)
    g_ours, lam_ours = fwd_bwd()
    g_plain, lam_plain = plain_gradient()
    rel_theta = float((g_ours - g_plain).norm() / g_plain.norm())
    rel_lam = float((lam_ours - lam_plain).norm() / lam_plain.norm())
    # finite differences: time a sample of the 2 n_theta plain solves
    n_theta = Pt.n
    cells = [int(c) for c in np.linspace(0, n_theta - 1, 4)]
    sample = []
    for c in cells:
        for sgn in (1.0, -1.0):
            th = th0.clone()
            th[c] += sgn * 1e-6 * th[c]
            sample.append(th)
    plain_solve(sample[0])
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for th in sample:
        plain_solve(th)
    f1.record()
    torch.cuda.synchronize()
    ms_solve = f0.elapsed_time(f1) / len(sample)
    fd_ms = 2 * n_theta * ms_solve
    out = {"metric": METRIC, "value": round(ms_fb, 3), "unit": "ms", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_fb, 3),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "adjoint_2d_256^2_k2_gmres30", "n": Pt.n,
                      "n_theta": n_theta, "rtol": 1e-8},
           "forward_only_ms": round(ms_f, 3),
           "backward_over_forward": round((ms_fb - ms_f) / ms_f, 3),
           "forward_iters": solver.last_forward.iters,
           "adjoint_iters": solver.last_backward.iters if solver.last_backward else None,
           "plain_gradient": {"ms": round(ms_plain, 3), "measured": True,
                              "what": "numeric ILU(2) of A + GMRES, explicit A^T + its own "
                                      "numeric ILU(2) (symbolic phase and sweep schedule "
                                      "kept) + GMRES, scatter, autograd through the assembly",
                              "iters_forward_adjoint": list(plain_info.get("iters", ())),
                              "rel_diff_dtheta": rel_theta, "rel_diff_lambda": rel_lam},
           "speedup_vs_plain_gradient": round(ms_plain / ms_fb, 3),
           "fd_loop": {"solves": 2 * n_theta, "sampled_solves": len(sample),
                       "ms_per_solve_measured": round(ms_solve, 3),
                       "ms_extrapolated": round(fd_ms, 1), "extrapolated": True},
           "speedup_vs_fd_loop_extrapolated": round(fd_ms / ms_fb, 1),
           "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def suite(args):
    """Every phase of every single-system configuration: C1 (2D 64^2, ILU(2)),
    C2 (random band n=160,000, ILU(k) for k = 0..3), C3 (3D 64^3, ILU(2) and
    TPIILU(2)), C6 (27-point Poisson on 50^3 and 90^3, k = 0, 1, ILU(k)
    against TPIILU(k) and the TPILU(k) policy).  Per phase: median ms of 20 CUDA-event-timed runs after 5
    warm-ups, algorithmic GB/s and fraction of the measured HBM peak, ns per
    level of the DAG the phase walks; per configuration the bit mismatches
    against the oracle and the oracle's own times on one host core (where it
    finishes in seconds; C2 k=3 takes minutes and is skipped)."""
    import torch

    import oracle
    import paper_0803_0048_gb300 as P
    from paper_0803_0048_gb300 import workloads as W

    torch.cuda.set_device(0)
    hbm, peak_src = measured_peaks()

    def med_ms(fn, reps=20, warm=5):
        for _ in range(warm):
            fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    def cpu_s(fn):
        t0 = time.perf_counter()
        r = fn()
        return time.perf_counter() - t0, r

    def bits(t):
        a = t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)
        return np.ascontiguousarray(a).view(np.uint64)

    cases = [("C1 2D 64^2", W.conv_diff_2d_64, 2, False),
             ("C2 band n=160000", lambda: W.random_band_160k(k=0), 0, False),
             ("C2 band n=160000", lambda: W.random_band_160k(k=1), 1, False),
             ("C2 band n=160000", lambda: W.random_band_160k(k=2), 2, True),
             ("C2 band n=160000", lambda: W.random_band_160k(k=3), 3, False),
             ("C3 3D 64^3", W.conv_diff_3d, 2, True),
             ("C6 27-point Poisson 50^3", lambda: W.poisson27_problem(50, 0), 0, True),
             ("C6 27-point Poisson 50^3", lambda: W.poisson27_problem(50, 1), 1, True),
             ("C6 27-point Poisson 90^3", lambda: W.poisson27_problem(90, 0), 0, True),
             ("C6 27-point Poisson 90^3", lambda: W.poisson27_problem(90, 1), 1, True)]
    rows = []
    for name, make, k, with_iilu in cases:
        Pb = make()
        A = Pb.A
        n, nnzA = A.n, A.nnz
        rp, ci, av, b = (torch.from_numpy(a).cuda() for a in (A.rowptr, A.colind, A.val, Pb.b))
        S = P.symbolic(rp, ci, k)
        F = P.numeric(S, av)
        depth = S.depth()
        frp, fci, flev, fdg = [t.cpu().numpy() for t in S.pattern()]
        nnzF = int(frp[-1])
        nnzL = int(np.sum(fdg - frp[:-1]))
        nnzU = nnzF - nnzL
        pvec = torch.from_numpy(W.uniform(W.stream_key(11, "suite"), np.arange(n), -1.0, 1.0)).cuda()
        y = F.apply(pvec)  # first application: autotunes the sweep schedules
        by = {  # algorithmic bytes (each array touched once)
            "symbolic": 8 * (n + 1) + 4 * nnzA + 8 * (n + 1) + 5 * nnzF + 8 * n,
            "numeric": 12 * nnzA + 16 * (n + 1) + 4 * nnzF + 8 * n + 8 * nnzF,
            "apply": 12 * nnzF + 16 * (n + 1) + 8 * n + 32 * n + 16 * n,
            "iilu_build": 12 * nnzF + 8 * nnzF + 16 * (n + 1) + 8 * n,
            "iilu_apply": 12 * nnzF + 16 * (n + 1) + 8 * n + 40 * n,
        }
        ph = {}
        big = k == 3 or n > 500000
        ph["symbolic"] = med_ms(lambda: P.symbolic(rp, ci, k), reps=5 if big else 20,
                                warm=1 if big else 5)
        ph["numeric"] = med_ms(lambda: F.refactor(av), reps=5 if big else 20,
                               warm=1 if big else 5)
        ph["apply"] = med_ms(lambda: F.apply(pvec))
        ph["factor"] = med_ms(lambda: P.factor(rp, ci, av, k), reps=5 if big else 20,
                              warm=1 if big else 5)
        x, info = P.gmres(rp, ci, av, b, F, restart=Pb.restart, rtol=Pb.rtol)
        ph["gmres"] = med_ms(lambda: P.gmres(rp, ci, av, b, F, restart=Pb.restart, rtol=Pb.rtol),
                             reps=5, warm=1)
        xb, info_b = P.bicgstab(rp, ci, av, b, F, rtol=Pb.rtol, maxit=5000, check=False)
        ph["bicgstab"] = med_ms(lambda: P.bicgstab(rp, ci, av, b, F, rtol=Pb.rtol, maxit=5000,
                                                   check=False), reps=5, warm=1)
        M = None
        if with_iilu:
            M = P.iiluk_build(F)
            ph["iilu_build"] = med_ms(lambda: P.iiluk_build(F), reps=10, warm=2)
            ph["iilu_apply"] = med_ms(lambda: M.apply(pvec))
            xi, info_i = P.gmres(rp, ci, av, b, M, restart=Pb.restart, rtol=Pb.rtol,
                                 maxit=5000, check=False)
            ph["gmres_iilu"] = med_ms(lambda: P.gmres(rp, ci, av, b, M, restart=Pb.restart,
                                                      rtol=Pb.rtol, maxit=5000, check=False),
                                      reps=3, warm=1)
            # the TPILU(k) policy: TPIILU for at most one GMRES cycle, then ILU(k)
            xt, info_t, used_t = P.tpilu_solve(rp, ci, av, b, F, M, restart=Pb.restart,
                                               rtol=Pb.rtol, iilu_maxit=Pb.restart, maxit=5000)
            ph["tpilu_policy"] = med_ms(lambda: P.tpilu_solve(
                rp, ci, av, b, F, M, restart=Pb.restart, rtol=Pb.rtol, iilu_maxit=Pb.restart,
                maxit=5000), reps=3, warm=1)
            xbi, info_bi = P.bicgstab(rp, ci, av, b, M, rtol=Pb.rtol, maxit=5000, check=False)
            ph["bicgstab_iilu"] = med_ms(lambda: P.bicgstab(rp, ci, av, b, M, rtol=Pb.rtol,
                                                            maxit=5000, check=False),
                                         reps=3, warm=1)
        phases = {}
        lev = {"symbolic": depth[0], "numeric": depth[0], "apply": depth[0] + depth[1],
               "iilu_build": max(depth)}
        for key, ms_ in ph.items():
            rec = {"ms": round(ms_, 4)}
            if key in by:
                gbps = by[key] / (ms_ / 1e3) / 1e9
                rec.update({"alg_bytes": by[key], "alg_GBps": round(gbps, 2),
                            "hbm_frac": round(gbps / hbm, 6)})
            if key in lev:
                rec["ns_per_level"] = round(ms_ * 1e6 / lev[key], 1)
            phases[key] = rec
        row = {"config": name, "k": k, "n": n, "nnz_A": nnzA, "nnz_F": nnzF, "nnz_L": nnzL,
               "nnz_U": nnzU, "depth_forward": depth[0], "depth_backward": depth[1],
               "sweep_schedule": [L_sched(F.schedule() & 0xff), L_sched((F.schedule() >> 8) & 0xff)],
               "gmres_iters": info.iters, "gmres_relres": info.relres,
               "bicgstab_iters": info_b.iters, "bicgstab_relres": info_b.relres,
               "phases": phases}
        if with_iilu:
            row["gmres_iilu_iters"] = info_i.iters
            row["bicgstab_iilu_iters"] = info_bi.iters
            row["tpilu_policy_used"] = used_t
            row["tpilu_policy_iters"] = info_t.iters
        if k <= 2 and n <= 300000:
            t_fac, ref = cpu_s(lambda: oracle.factor(A, k))
            t_app, yo = cpu_s(lambda: oracle.apply(n, ref["rowptr"], ref["colind"], ref["val"],
                                                   pvec.cpu().numpy()))
            par = {"pattern_equal": bool(np.array_equal(frp, ref["rowptr"]) and
                                         np.array_equal(fci, ref["colind"]) and
                                         np.array_equal(flev, ref["level"])),
                   "factor_bit_mismatches": int(np.sum(bits(F.values()) != bits(ref["val"]))),
                   "apply_bit_mismatches": int(np.sum(bits(y) != bits(yo)))}
            orc = {"factor_s": round(t_fac, 3), "apply_s": round(t_app, 4)}
            t_g, (st, xo, it, rel, cyc) = cpu_s(lambda: oracle.gmres(
                n, A.rowptr, A.colind, A.val, Pb.b, oracle.PREC_ILU,
                (ref["rowptr"], ref["colind"], ref["val"]), Pb.restart, Pb.rtol,
                dotmode=oracle.DOT_TREE))
            orc["gmres_s"] = round(t_g, 3)
            par["gmres_x_bit_mismatches"] = int(np.sum(bits(x) != bits(xo)))
            par["gmres_iters_equal"] = it == info.iters
            t_b, (stb, xbo, itb, relb, _) = cpu_s(lambda: oracle.bicgstab(
                n, A.rowptr, A.colind, A.val, Pb.b, oracle.PREC_ILU,
                (ref["rowptr"], ref["colind"], ref["val"]), Pb.rtol, 5000, oracle.DOT_TREE))
            orc["bicgstab_s"] = round(t_b, 3)
            par["bicgstab_x_bit_mismatches"] = int(np.sum(bits(xb) != bits(xbo)))
            par["bicgstab_iters_equal"] = itb == info_b.iters
            if with_iilu:
                t_ib, go = cpu_s(lambda: oracle.iiluk_build(n, ref["rowptr"], ref["colind"],
                                                            ref["val"]))
                orc["iilu_build_s"] = round(t_ib, 3)
                par["iilu_bit_mismatches"] = int(np.sum(bits(M.values()) != bits(go)))
            row["parity"] = par
            row["oracle_one_core"] = orc
        else:
            row["parity"] = "oracle skipped: too slow on one core for this case"
        rows.append(row)
        print(json.dumps({"progress": name, "k": k}), file=sys.stderr, flush=True)
    out = {"metric": METRIC, "workload": "suite", "unit": "ms", "dtype": "f64",
           "data": "synthetic", "peak_GBps": hbm, "peak_source": peak_src,
           "timing": "CUDA events, median of 20 runs after 5 warm-ups (5 runs for C2 k=3 "
                     "and for GMRES solves)", "configs": rows}
    print(json.dumps(out), flush=True)


def ratio(args):
    """Symbolic against numeric time for k = 1..5, the experiment of the
    paper's Sec. 4.6 (the sequential symbolic phase's share grows with k and
    passes the numeric phase's for large k).  The paper's matgen matrices are
    not available; seeded random sparse matrices of its sizes and densities
    (1,000-4,000 rows, 0.01-0.002) stand in, beside the random band matrix
    (n = 160,000) and the 27-point Poisson matrix (50^3).  Per case and k: the
    sizes (nnz_F, longest row, DAG depths), the GPU symbolic phase and the GPU
    numeric phase (a refactorization on level orders; both median ms), their
    ratio, and where the oracle finishes in seconds its own two phases on one
    host core, their ratio, and the GPU's bit parity against it.  For k = 1
    the three symbolic walks (iluk_set_symbolic_variant) are timed too."""
    import torch

    import oracle
    import paper_0803_0048_gb300 as P
    from paper_0803_0048_gb300 import workloads as W
    torch.cuda.set_device(0)

    def med_ms(fn, reps, warm=2):
        for _ in range(warm):
            fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    def u64(a):
        a = a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)
        return np.ascontiguousarray(a).view(np.uint64)

    cases = [("random n=1000 density 0.01", lambda: W.random_sparse(1000, 0.01, 77), range(1, 6),
              True),
             ("random n=2000 density 0.004", lambda: W.random_sparse(2000, 0.004, 77),
              range(1, 6), True),
             ("random n=4000 density 0.002", lambda: W.random_sparse(4000, 0.002, 77),
              range(1, 6), True),
             ("27-point Poisson 50^3", lambda: W.poisson27(50), range(0, 4), False),
             ("random band n=160000", lambda: W.random_band_160k(k=1).A, range(1, 5), False)]
    rows = []
    for name, make, ks, with_oracle in cases:
        A = make()
        rp, ci, av = (torch.from_numpy(a).cuda() for a in (A.rowptr, A.colind, A.val))
        for k in ks:
            S = P.symbolic(rp, ci, k)
            F = P.numeric(S, av)
            depth = S.depth()
            frp = S.pattern()[0].cpu().numpy()
            nnzF = int(frp[-1])
            big = nnzF > 50_000_000
            reps = 3 if big else 10
            t_sym = med_ms(lambda: P.symbolic(rp, ci, k), reps, 1 if big else 2)
            t_num = med_ms(lambda: F.refactor(av), reps, 1 if big else 2)
            row = {"case": name, "k": k, "n": A.n, "nnz_A": A.nnz, "nnz_F": nnzF,
                   "max_row": int(np.diff(frp).max()), "depth": list(depth),
                   "gpu_symbolic_ms": round(t_sym, 4), "gpu_numeric_ms": round(t_num, 4),
                   "gpu_ratio": round(t_sym / t_num, 3)}
            if k == 1:
                var = {}
                for v in (0, 1, 2):
                    prev = P.set_symbolic_variant(v)
                    try:
                        var[["ascending", "descending", "general_walk"][v]] = round(
                            med_ms(lambda: P.symbolic(rp, ci, k), reps), 4)
                    finally:
                        P.set_symbolic_variant(prev)
                row["k1_symbolic_variants_ms"] = var
            if with_oracle:
                t0 = time.perf_counter()
                st, bad, orp, oci, olev = oracle.symbolic(A.n, A.rowptr, A.colind, k)
                t1 = time.perf_counter()
                st2, bad2, ov = oracle.numeric(A.n, A.rowptr, A.colind, A.val, orp, oci)
                t2 = time.perf_counter()
                grp, gci, glev, _ = [t.cpu().numpy() for t in S.pattern()]
                row["oracle_one_core"] = {"symbolic_s": round(t1 - t0, 4),
                                          "numeric_s": round(t2 - t1, 4),
                                          "ratio": round((t1 - t0) / max(t2 - t1, 1e-9), 3)}
                row["parity"] = {
                    "pattern_equal": bool(np.array_equal(grp, orp) and np.array_equal(gci, oci)
                                          and np.array_equal(glev, olev)),
                    "factor_bit_mismatches": int(np.sum(u64(F.values()) != u64(ov)))}
            rows.append(row)
            print(json.dumps({"progress": name, "k": k}), file=sys.stderr, flush=True)
            del S, F
            torch.cuda.empty_cache()
    out = {"metric": METRIC, "workload": "ratio", "unit": "ms", "dtype": "f64",
           "data": "synthetic", "timing": "CUDA events, median of 10 runs (3 above 50 M "
           "factor entries); oracle: one run on one host core", "host": host_cpu(),
           "cases": rows}
    print(json.dumps(out), flush=True)


def L_sched(byte):
    from paper_0803_0048_gb300 import _lib as L
    return L.sched_name(byte)


def main():
    args = parse()
    if args.impl == "reference":
        reference(args)
    elif args.workload == "batched":
        batched(args)
    elif args.workload == "adjoint":
        adjoint(args)
    elif args.workload == "ratio":
        ratio(args)
    elif args.workload == "suite":
        suite(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
