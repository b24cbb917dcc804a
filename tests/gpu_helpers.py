"""Shared helpers for the GPU parity tests (CUDA path vs. oracle)."""
import numpy as np
import torch

from paper_0803_0048_gb300 import workloads as W


def bits(a) -> np.ndarray:
    """float64 array as int64 bit patterns (so -0.0 != +0.0 and NaNs compare)."""
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


def assert_bits_equal(got, want, what=""):
    g, w = bits(got), bits(want)
    assert g.shape == w.shape, f"{what}: shape {g.shape} vs {w.shape}"
    bad = np.nonzero(g != w)[0]
    assert bad.size == 0, (f"{what}: {bad.size} of {g.size} differ, first at {bad[0]}: "
                           f"{np.asarray(got).reshape(-1)[bad[0]] if not isinstance(got, torch.Tensor) else got.reshape(-1)[bad[0]].item()!r} "
                           f"vs {np.asarray(want).reshape(-1)[bad[0]]!r}")


def to_dev(A: W.CSR, dev="cuda"):
    return (torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colind).to(dev),
            torch.from_numpy(A.val).to(dev))


def vec(seed: int, n: int, dev="cuda"):
    v = W.uniform(W.stream_key(seed, "vec"), np.arange(n), -1.0, 1.0)
    return v, torch.from_numpy(v).to(dev)


def small_cases():
    """(name, CSR, k) cases the oracle finishes quickly; several tiles of rows
    and ragged row lengths."""
    cases = []
    for n, dens, seed in [(1, 1.0, 1), (2, 0.5, 2), (37, 0.15, 3), (150, 0.04, 4),
                          (301, 0.02, 5), (1000, 0.006, 6)]:
        A = W.random_sparse(n, dens, seed)
        for k in (0, 1, 2, 3):
            cases.append((f"rand{n}_k{k}", A, k))
    A = W.random_sparse(120, 0.05, 7, dominance=0.7)
    cases.append(("nondominant120_k2", A, 2))
    cases.append(("convdiff2d_20_k2", W.conv_diff(20, 2, (20.0, 20.0)), 2))
    cases.append(("convdiff3d_9_k1", W.conv_diff(9, 3, (50.0, 50.0, 50.0)), 1))
    cases.append(("convdiff3d_9_k3", W.conv_diff(9, 3, (50.0, 50.0, 50.0)), 3))
    cases.append(("band3000_k2", W.random_band(3000, 9, 100, 11), 2))
    A = W.random_sparse(60, 0.3, 8)  # dense-ish: long rows, full fill at high k
    cases.append(("dense60_k250", A, 250))
    return cases
