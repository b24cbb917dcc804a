"""Writes band160k_k3.json: SHA-256 digests of the oracle's results on the
random band matrix (n = 160,000, 9 off-diagonals per row within |i - j| <= 2000)
at level k = 3, where F has about 87 million entries and the oracle needs
minutes, too long to run inside a test.  Calls only the oracle (and the input
generator); the GPU test compares the CUDA library's arrays with these digests
bit for bit.

Digested, each as the little-endian bytes of the array:
  pattern   rowptr (int64[n+1]) followed by colind (int32[nnz_F])
  levels    uint8[nnz_F] (Def. 2.3)
  values    float64[nnz_F] (Eq. 1, IKJ order)
  apply     y = (L~U~)^-1 p for p uniform in [-1, 1] from stream ("k3", 3)
  tpiilu    g (Sec. 3.5), float64[nnz_F]
  gmres_x   GMRES(50) to 1e-8 with the ILU(3) sweeps and the fixed-tree inner
            products, plus its iterations, cycles and the bits of relres

    python tests/golden/make_band160k_k3.py
"""
import hashlib
import json
import os
import platform
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_0803_0048_gb300 import workloads as W  # noqa: E402

K = 3
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "band160k_k3.json")


def sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).view(np.uint8).tobytes())
    return h.hexdigest()


def apply_input(n: int) -> np.ndarray:
    return W.uniform(W.stream_key(3, "k3"), np.arange(n), -1.0, 1.0)


def main():
    Pb = W.random_band_160k(k=K)
    A = Pb.A
    secs = {}
    t = time.perf_counter()
    st, bad, frp, fci, flev = oracle.symbolic(A.n, A.rowptr, A.colind, K)
    secs["symbolic"] = time.perf_counter() - t
    assert st == oracle.OK, (st, bad)
    t = time.perf_counter()
    st, bad, fv = oracle.numeric(A.n, A.rowptr, A.colind, A.val, frp, fci)
    secs["numeric"] = time.perf_counter() - t
    assert st == oracle.OK, (st, bad)
    t = time.perf_counter()
    y = oracle.apply(A.n, frp, fci, fv, apply_input(A.n))
    secs["apply"] = time.perf_counter() - t
    t = time.perf_counter()
    g = oracle.iiluk_build(A.n, frp, fci, fv)
    secs["tpiilu_build"] = time.perf_counter() - t
    t = time.perf_counter()
    st, x, it, rel, cyc = oracle.gmres(A.n, A.rowptr, A.colind, A.val, Pb.b, oracle.PREC_ILU,
                                       (frp, fci, fv), Pb.restart, Pb.rtol,
                                       dotmode=oracle.DOT_TREE)
    secs["gmres"] = time.perf_counter() - t
    assert st == oracle.OK
    out = {"case": "random_band_n160000_hw2000", "k": K, "n": A.n, "nnz_A": int(A.rowptr[-1]),
           "nnz_F": int(frp[-1]),
           "pattern": sha(frp, fci), "levels": sha(flev), "values": sha(fv), "apply": sha(y),
           "tpiilu": sha(g), "gmres_x": sha(x), "gmres_iters": it, "gmres_cycles": cyc,
           "gmres_relres_bits": int(np.float64(rel).view(np.int64)),
           "oracle_seconds": {k: round(v, 2) for k, v in secs.items()},
           "oracle_host": f"{platform.machine()}, one core"}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
