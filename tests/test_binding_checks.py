"""Argument checks of the Python binding, on CPU.

The C ABI takes plain pointers and reads lengths from the handle or the
pattern, so a float32 tensor or one of the wrong length would become an
out-of-bounds device read.  The binding rejects both with ValueError before
any pointer crosses the boundary; these tests use stand-in handles and CPU
tensors, so the library is never called.
"""
from types import SimpleNamespace

import pytest
import torch

import paper_0803_0048_gb300 as P
from paper_0803_0048_gb300 import api


def fake_sym(n=5, nnz_a=13, nnz_f=17):
    S = api.Symbolic.__new__(api.Symbolic)
    S.h = None
    S.n, S.nnz, S.max_row, S.k = n, nnz_f, 4, 2
    S.A = SimpleNamespace(n=n, nnz=nnz_a, rowptr=torch.zeros(n + 1, dtype=torch.int64))
    return S


def fake_fac(S):
    F = api.Factors.__new__(api.Factors)
    F.h, F.S = None, S
    return F


def f64(n):
    return torch.zeros(n, dtype=torch.float64)


def test_vecs_checks_dtype_and_length_before_device():
    with pytest.raises(ValueError, match="p: expected torch.float64"):
        api._vecs((torch.zeros(4, dtype=torch.float32), 4, "p"))
    with pytest.raises(ValueError, match="q: expected 4 elements, got 3"):
        api._vecs((f64(4), 4, "p"), (f64(3), 4, "q"))
    with pytest.raises(ValueError, match="CUDA device"):
        api._vecs((f64(4), 4, "p"), (None, 4, "out"))
    api._vecs((None, 4, "out"))  # optional outputs


@pytest.mark.parametrize("rp,ci", [
    (torch.zeros(3, dtype=torch.int32), torch.zeros(2, dtype=torch.int32)),
    (torch.zeros(3, dtype=torch.int64), torch.zeros(2, dtype=torch.int64)),
    (torch.zeros(1, 3, dtype=torch.int64), torch.zeros(2, dtype=torch.int32)),
    (torch.zeros(0, dtype=torch.int64), torch.zeros(0, dtype=torch.int32)),
])
def test_pattern_dtype_and_shape(rp, ci):
    with pytest.raises(ValueError, match="CSR pattern"):
        api.CsrPattern(rp, ci)


def test_pattern_on_host_is_rejected():
    with pytest.raises(ValueError, match="CUDA device"):
        api.CsrPattern(torch.zeros(3, dtype=torch.int64), torch.zeros(2, dtype=torch.int32))


def test_numeric_and_refactor_value_length():
    S = fake_sym()
    with pytest.raises(ValueError, match="values of A: expected 13"):
        P.numeric(S, f64(17))
    with pytest.raises(ValueError, match="float64"):
        P.numeric(S, torch.zeros(13, dtype=torch.float32))
    with pytest.raises(ValueError, match="values of A: expected 13"):
        fake_fac(S).refactor(f64(12))


def test_apply_vector_lengths():
    F = fake_fac(fake_sym())
    with pytest.raises(ValueError, match="p: expected 5"):
        F.apply(f64(6))
    with pytest.raises(ValueError, match="CUDA device"):
        F.apply(f64(5))
    M = api.IncompleteInverse.__new__(api.IncompleteInverse)
    M.h, M.F = None, F
    with pytest.raises(ValueError, match="p: expected 5"):
        M.apply(f64(4))


def test_batched_shapes():
    S = fake_sym()
    with pytest.raises(ValueError, match="nbatch, nnz_A"):
        P.numeric_batched(S, f64(13))
    with pytest.raises(ValueError, match="expected 26 elements"):
        P.numeric_batched(S, torch.zeros(2, 12, dtype=torch.float64))
    with pytest.raises(ValueError, match="item 1: b: expected 5"):
        P.BatchSolve([(S, f64(13), f64(5), f64(5)), (S, f64(13), f64(4), f64(5))])


def test_dot_and_division_lengths():
    with pytest.raises(ValueError, match="y: expected 7"):
        P.dot(f64(7), f64(6))
    with pytest.raises(ValueError, match="b: expected 3"):
        P.div_rn(f64(3), f64(2))
