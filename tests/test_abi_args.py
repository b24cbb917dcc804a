"""CPU checks of the C ABI's argument errors.

Every call below is refused by its argument checks with ILUK_EINVAL (or the
documented status) before it touches CUDA, so the library runs here without a
GPU.  The non-NULL pointers handed over point at host memory that the refused
calls never read: each case is one where a check on sizes, handles or NULL
pointers returns first.  The last test alone passes the checks, and runs only
where no GPU is present: there the first CUDA call fails and the entry point
must return ILUK_ECUDA through its cleanup path.
"""
import ctypes as C

import pytest

from paper_0803_0048_gb300 import _lib as L


@pytest.fixture(scope="module")
def lib():
    from paper_0803_0048_gb300 import build
    build.build()
    return L.load()


_dummy = (C.c_double * 8)()
DUMMY = C.cast(_dummy, C.c_void_p)


def pat(n=4, nnz=4, rowptr=True, colind=True):
    return L.Pattern(n, nnz, DUMMY.value if rowptr else None, DUMMY.value if colind else None)


def einval(st, info=None):
    assert st == L.EINVAL
    if info is not None:
        assert info.status == L.EINVAL and info.row == -1


def test_validate_rejects_bad_sizes_and_pointers(lib):
    for A in (pat(n=-1), pat(nnz=-1), pat(rowptr=False), pat(colind=False),
              pat(n=1 << 31, nnz=0)):
        info = L.Info()
        einval(lib.iluk_validate(C.byref(A), C.byref(info), None), info)
    einval(lib.iluk_validate(None, None, None))


def test_symbolic_and_factor_reject_k_and_missing_outputs(lib):
    A = pat()
    h, h2 = C.c_void_p(), C.c_void_p()
    for k in (-1, 251):
        info = L.Info()
        einval(lib.iluk_symbolic(C.byref(A), k, C.byref(h), C.byref(info), None), info)
        einval(lib.iluk_factor(C.byref(A), DUMMY, k, C.byref(h), C.byref(h2), None, None))
    einval(lib.iluk_symbolic(C.byref(A), 2, None, None, None))
    # values missing for a non-empty pattern
    einval(lib.iluk_factor(C.byref(A), None, 2, C.byref(h), C.byref(h2), None, None))
    assert h.value is None and h2.value is None


def test_handle_calls_reject_null_handles(lib):
    h = C.c_void_p()
    einval(lib.iluk_numeric(None, DUMMY, C.byref(h), None, None))
    einval(lib.iluk_refactor(None, DUMMY, None, None))
    einval(lib.iluk_sym_query(None, DUMMY))
    einval(lib.iluk_sym_depth(None, None, None, None))
    einval(lib.iluk_sym_export(None, None, None, None, None, None))
    einval(lib.iluk_fac_values(None, C.byref(h)))
    einval(lib.iluk_fac_export(None, DUMMY, None))
    einval(lib.iluk_apply(None, DUMMY, DUMMY, 0, None))
    einval(lib.iluk_apply_sched(None, DUMMY, DUMMY, 0, 0, None))
    einval(lib.iluk_set_schedule(None, 0))
    assert lib.iluk_get_schedule(None) == -1
    einval(lib.iiluk_build(None, C.byref(h), None, None))
    einval(lib.iiluk_values(None, C.byref(h)))
    einval(lib.iiluk_export(None, DUMMY, None))
    einval(lib.iiluk_apply(None, DUMMY, DUMMY, None))
    einval(lib.iluk_batch_solve(None, None))
    einval(lib.iluk_batch_results(None, None, None))
    einval(lib.iluk_batch_set_schedule(None, 512, 0))
    assert lib.iluk_batch_width(None) == 0 and lib.iluk_batch_spin(None) == 0
    # destroying nothing is a no-op
    for d in (lib.iluk_sym_destroy, lib.iluk_fac_destroy, lib.iiluk_destroy,
              lib.iluk_batch_destroy):
        d(None)


def test_vector_calls_reject_missing_vectors(lib):
    A = pat()
    einval(lib.iluk_spmv(C.byref(A), DUMMY, None, DUMMY, None))
    einval(lib.iluk_spmv(C.byref(A), DUMMY, DUMMY, None, None))
    einval(lib.iluk_spmv(C.byref(A), None, DUMMY, DUMMY, None))
    einval(lib.iluk_spmv(C.byref(pat(n=-2)), DUMMY, DUMMY, DUMMY, None))
    einval(lib.iluk_adjoint_scatter(C.byref(A), DUMMY, DUMMY, None, None))
    einval(lib.iluk_adjoint_scatter(C.byref(A), None, DUMMY, DUMMY, None))
    einval(lib.iluk_dot(-1, DUMMY, DUMMY, DUMMY, None))
    einval(lib.iluk_dot(5, None, DUMMY, DUMMY, None))
    einval(lib.iluk_dot(0, None, None, None, None))
    for args in ((-1, 4, DUMMY, DUMMY, DUMMY, DUMMY, DUMMY, 2, 30, 1e-8, 10, 0),
                 (4, 4, None, DUMMY, DUMMY, DUMMY, DUMMY, 2, 30, 1e-8, 10, 0),
                 (4, 4, DUMMY, None, DUMMY, DUMMY, DUMMY, 2, 30, 1e-8, 10, 0),
                 (4, 4, DUMMY, DUMMY, DUMMY, None, DUMMY, 2, 30, 1e-8, 10, 0),
                 (4, 4, DUMMY, DUMMY, DUMMY, DUMMY, None, 2, 30, 1e-8, 10, 0),
                 (4, 4, DUMMY, DUMMY, DUMMY, DUMMY, DUMMY, 251, 30, 1e-8, 10, 0),
                 (4, 4, DUMMY, DUMMY, DUMMY, DUMMY, DUMMY, 2, 0, 1e-8, 10, 0)):
        info = L.Info()
        einval(lib.iluk_solve_host(*args, C.byref(info), None), info)
    # iluk_solve: A, values, k, b, x, m, rtol, maxit, sched, S_out, F_out
    A4 = pat()
    for args in ((C.byref(pat(n=-1)), DUMMY, 2, DUMMY, DUMMY, 30, 1e-8, 10, 0),
                 (None, DUMMY, 2, DUMMY, DUMMY, 30, 1e-8, 10, 0),
                 (C.byref(A4), None, 2, DUMMY, DUMMY, 30, 1e-8, 10, 0),    # values
                 (C.byref(A4), DUMMY, -1, DUMMY, DUMMY, 30, 1e-8, 10, 0),  # k
                 (C.byref(A4), DUMMY, 251, DUMMY, DUMMY, 30, 1e-8, 10, 0),
                 (C.byref(A4), DUMMY, 2, None, DUMMY, 30, 1e-8, 10, 0),    # b
                 (C.byref(A4), DUMMY, 2, DUMMY, None, 30, 1e-8, 10, 0),    # x
                 (C.byref(A4), DUMMY, 2, DUMMY, DUMMY, 0, 1e-8, 10, 0),    # m
                 (C.byref(A4), DUMMY, 2, DUMMY, DUMMY, 30, 1e-8, -1, 0),   # maxit
                 (C.byref(A4), DUMMY, 2, DUMMY, DUMMY, 30, 1e-8, 10, -1),  # sched
                 (C.byref(A4), DUMMY, 2, DUMMY, DUMMY, 30, 1e-8, 10, 0x10000),
                 (C.byref(A4), DUMMY, 2, DUMMY, DUMMY, 30, 1e-8, 10, 0x9F)):  # no such kind
        info = L.Info()
        hs, hf = C.c_void_p(123), C.c_void_p(456)
        einval(lib.iluk_solve(*args, C.byref(hs), C.byref(hf), C.byref(info), None), info)
        assert hs.value is None and hf.value is None  # outputs cleared first
    einval(lib.iluk_transpose(C.byref(pat(n=-1)), DUMMY, DUMMY, DUMMY, DUMMY, None))
    for args in ((None, DUMMY, DUMMY, DUMMY), (DUMMY, None, DUMMY, DUMMY),
                 (DUMMY, DUMMY, None, DUMMY), (DUMMY, DUMMY, DUMMY, None)):
        einval(lib.iluk_transpose(C.byref(pat()), *args, None))
    einval(lib.iluk_div_rn(-1, DUMMY, DUMMY, DUMMY, None))
    einval(lib.iluk_div_rn(3, DUMMY, None, DUMMY, None))
    einval(lib.iiluk_apply_noalloc(-1, DUMMY, DUMMY, DUMMY, DUMMY, DUMMY, DUMMY, None))
    einval(lib.iiluk_apply_noalloc(4, DUMMY, DUMMY, DUMMY, DUMMY, None, DUMMY, None))
    assert lib.iiluk_apply_noalloc((1 << 20) + 1, DUMMY, DUMMY, DUMMY, DUMMY, DUMMY, DUMMY,
                                   None) == L.ENOMEM
    assert lib.iiluk_apply_noalloc(0, None, None, None, None, None, None, None) == L.OK


def test_solvers_reject_bad_arguments(lib):
    A = pat()
    gm = lib.gmres_solve
    cases = [
        (C.byref(pat(n=-1)), DUMMY, L.PREC_NONE, None, DUMMY, DUMMY, 30, 1e-8, 10, 0),
        (C.byref(A), DUMMY, L.PREC_NONE, None, None, DUMMY, 30, 1e-8, 10, 0),   # b
        (C.byref(A), DUMMY, L.PREC_NONE, None, DUMMY, None, 30, 1e-8, 10, 0),   # x
        (C.byref(A), None, L.PREC_NONE, None, DUMMY, DUMMY, 30, 1e-8, 10, 0),   # values
        (C.byref(A), DUMMY, L.PREC_NONE, None, DUMMY, DUMMY, 0, 1e-8, 10, 0),   # m
        (C.byref(A), DUMMY, L.PREC_NONE, None, DUMMY, DUMMY, 30, 1e-8, -1, 0),  # maxit
        (C.byref(A), DUMMY, L.PREC_ILU, None, DUMMY, DUMMY, 30, 1e-8, 10, 0),   # prec
        (C.byref(A), DUMMY, L.PREC_IILU, DUMMY, DUMMY, DUMMY, 30, 1e-8, 10, 1),  # IILU^T
    ]
    for args in cases:
        info = L.Info()
        einval(gm(*args, C.byref(info), None), info)
    for args in cases:
        info = L.Info()
        einval(lib.gmres_solve_ex(*args, L.BASIS["auto"], C.byref(info), None), info)
    for basis in (-1, 4):  # unknown basis mode
        info = L.Info()
        einval(lib.gmres_solve_ex(C.byref(A), DUMMY, L.PREC_NONE, None, DUMMY, DUMMY, 30, 1e-8,
                                  10, 0, basis, C.byref(info), None), info)
    for b, x, vals in ((None, DUMMY, DUMMY), (DUMMY, None, DUMMY), (DUMMY, DUMMY, None)):
        info = L.Info()
        einval(lib.bicgstab_solve(C.byref(A), vals, L.PREC_NONE, None, b, x, 1e-8, 10,
                                  C.byref(info), None), info)
    used = C.c_int(-1)
    for F, solver, m, b in ((None, L.SOLVER_GMRES, 30, DUMMY), (DUMMY, 7, 30, DUMMY),
                            (DUMMY, L.SOLVER_GMRES, 0, DUMMY), (DUMMY, L.SOLVER_GMRES, 30, None)):
        info = L.Info()
        einval(lib.tpilu_solve(C.byref(A), DUMMY, F, None, solver, b, DUMMY, m, 1e-8, 50, 100,
                               C.byref(used), C.byref(info), None), info)


def test_batch_calls_reject_bad_arguments(lib):
    h = C.c_void_p()
    einval(lib.iluk_numeric_batched(None, 2, DUMMY, DUMMY, None, None))
    einval(lib.iluk_batch_create(None, 1, 30, 1e-8, 10, C.byref(h), None))
    einval(lib.iluk_batch_create(DUMMY, 1, 30, 1e-8, 10, None, None))
    einval(lib.iluk_batch_create(DUMMY, -1, 30, 1e-8, 10, C.byref(h), None))
    for restart in (0, 65):
        einval(lib.iluk_batch_create(DUMMY, 1, restart, 1e-8, 10, C.byref(h), None))
    items = (L.BatchItem * 1)()  # every pointer NULL
    einval(lib.iluk_batch_create(items, 1, 30, 1e-8, 10, C.byref(h), None))


def test_prof_read_and_strerror(lib):
    einval(lib.iluk_prof_read(None, None, -1))
    einval(lib.iluk_prof_read(None, None, 3))
    msgs = [lib.iluk_strerror(s) for s in range(10)]
    assert all(msgs) and len(set(msgs)) == 10


def _cuda_available():
    import torch
    return torch.cuda.is_available()


@pytest.mark.skipif(_cuda_available(), reason="host-only: with a GPU these calls would launch "
                    "kernels on host pointers")
def test_failing_cuda_calls_surface_as_ecuda(lib):
    """Without a GPU the first CUDA call of each entry point fails; the call
    returns ILUK_ECUDA through its cleanup path instead of crashing."""
    A = pat()
    info = L.Info()
    assert lib.iluk_validate(C.byref(A), C.byref(info), None) == L.ECUDA
    assert info.status == L.ECUDA
    assert lib.iluk_dot(4, DUMMY, DUMMY, DUMMY, None) == L.ECUDA
    for transpose in (0, 1):
        assert lib.gmres_solve(C.byref(A), DUMMY, L.PREC_NONE, None, DUMMY, DUMMY, 30, 1e-8, 10,
                               transpose, C.byref(info), None) == L.ECUDA
        for basis in L.BASIS.values():
            assert lib.gmres_solve_ex(C.byref(A), DUMMY, L.PREC_NONE, None, DUMMY, DUMMY, 30,
                                      1e-8, 10, transpose, basis, C.byref(info), None) == L.ECUDA
    assert lib.bicgstab_solve(C.byref(A), DUMMY, L.PREC_NONE, None, DUMMY, DUMMY, 1e-8, 10,
                              C.byref(info), None) == L.ECUDA
    h = C.c_void_p()
    assert lib.iluk_symbolic(C.byref(A), 2, C.byref(h), C.byref(info), None) == L.ECUDA
    assert h.value is None
