"""Runs bench.ours() on CPU with the CUDA runtime and libiluk replaced by
stand-ins that return the oracle's factors, so that the bench line's host
logic (timing arithmetic, roofline, operand stream, JSON keys) runs without a
GPU.  Not a measurement: the times are made up.  Run it as a separate process:
it patches torch.device and torch.cuda for the whole interpreter.
"""
import os
import sys
import types

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import bench  # noqa: E402
import oracle  # noqa: E402
import paper_0803_0048_gb300 as P  # noqa: E402

STEPS = 3
STEP_MS = 119.0

Pb = bench.workload(2)
Fo = oracle.factor(Pb.A, 2)
n = Pb.A.n
frp, fci, flev = Fo["rowptr"], Fo["colind"], Fo["level"]
rows = np.repeat(np.arange(n), np.diff(frp))
fdg = np.flatnonzero(fci == rows).astype(np.int64)

_device = torch.device
torch.device = lambda *a, **k: _device("cpu")
torch.cuda.set_device = lambda d: None
torch.cuda.current_stream = lambda *a: None
torch.cuda.synchronize = lambda *a: None
torch.Tensor.pin_memory = lambda self: self


class Event:
    def __init__(self, **kw):
        pass

    def record(self, *a):
        pass

    def elapsed_time(self, other):
        return STEP_MS * STEPS


torch.cuda.Event = Event


class Sym:
    def pattern(self):
        return [torch.from_numpy(a) for a in (frp, fci, flev, fdg)]

    def depth(self):
        return (15777, 15629)


class Fac:
    def set_schedule(self, s):
        pass

    def schedule(self):
        return 5 | (5 << 8)

    def values(self):
        return torch.from_numpy(Fo["val"])


launches = [0]


def launch_count():
    launches[0] += 59 * STEPS  # 59 launches in each timed step
    return launches[0]


info = types.SimpleNamespace(iters=4, relres=7.8e-11)
P.validate = lambda rp, ci: (0, -1)
P.factor = lambda rp, ci, av, k: (Sym(), Fac())
P.gmres = lambda *a, **k: (torch.zeros(n, dtype=torch.float64), info)


def solve(rp, ci, av, b, k=2, restart=30, rtol=1e-8, sched=0, return_factors=False, **kw):
    assert return_factors
    return torch.zeros(n, dtype=torch.float64), info, (Sym(), Fac())


P.solve = solve


def solve_host(rp, ci, av, b, k, restart, rtol, sched=0, x=None):
    assert rp.device.type == "cpu" and x is not None and x.device.type == "cpu"
    x.zero_()
    return x, info


P.solve_host = solve_host
P.launch_count = launch_count
P.prof_enable = lambda on=True: None
P.prof_read = lambda: {"validate": (0.05, STEPS), "factor": (32.5 * STEPS, STEPS),
                       "compact": (0.35 * STEPS, 2 * STEPS), "sweep": (38.0 * STEPS, 4 * STEPS),
                       "sweep_bwd": (45.0 * STEPS, 4 * STEPS), "spmv": (0.1 * STEPS, 3 * STEPS),
                       "dot": (0.2 * STEPS, 10 * STEPS), "vector": (0.06 * STEPS, 7 * STEPS),
                       "numeric": (0.0, 0)}
bench.measured_peaks = lambda: (6781.8, "measured")
sys.argv = ["bench.py", "--steps", str(STEPS), "--warmup", "3", "--no-cpu"]
bench.ours(bench.parse())
