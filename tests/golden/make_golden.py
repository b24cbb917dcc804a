"""Writes oracle_snapshots.json: digests of the oracle's outputs on a few fixed
synthetic problems.  Calls only the oracle (and the input generator).  The
paper prints no worked example to pin against (its Fig. 1 is not recoverable),
so these snapshots are regression anchors for the oracle itself: they must
come out the same on every machine (x86 here, Arm on the GPU host), which the
-ffp-contract=off build is meant to guarantee.

    python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_0803_0048_gb300 import workloads as W  # noqa: E402


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:32]


def snapshot(name, A, k, restart):
    F = oracle.factor(A, k)
    g = oracle.iiluk_build(A.n, F["rowptr"], F["colind"], F["val"])
    b = W.matvec_rowseq(A, W.uniform(W.stream_key(7, "golden"), np.arange(A.n), -1.0, 1.0))
    st, x, it, rel, cyc = oracle.gmres(A.n, A.rowptr, A.colind, A.val, b, oracle.PREC_ILU,
                                       (F["rowptr"], F["colind"], F["val"]), restart, 1e-10,
                                       dotmode=oracle.DOT_TREE)
    return {"case": name, "k": k, "n": A.n, "nnz_F": int(F["rowptr"][-1]),
            "pattern": digest(np.concatenate([F["rowptr"].view(np.uint8), F["colind"].view(np.uint8)])),
            "levels": digest(F["level"]), "values": digest(F["val"]), "tpiilu": digest(g),
            "gmres_x": digest(x), "gmres_iters": it, "gmres_status": st,
            "first_values": [float(v) for v in F["val"][:4]]}


def cases():
    return [("convdiff2d_64x64", W.conv_diff(64, 2, (20.0, 20.0)), 2, 30),
            ("random_sparse_300", W.random_sparse(300, 0.02, 5), 3, 30),
            ("random_band_2000", W.random_band(2000, 9, 200, 11), 2, 50)]


def main():
    snaps = [snapshot(*c) for c in cases()]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_snapshots.json")
    with open(out, "w") as f:
        json.dump(snaps, f, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
