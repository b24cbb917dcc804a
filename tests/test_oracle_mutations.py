"""The pins must be able to fail: each plausible mistake planted in a copy of
the oracle's C source (a dropped term, a wrong sign, a wrong index or bound, a
transposed operation) has to be caught by at least one pin.

The mutants are compiled into a temporary directory and loaded in place of
the real oracle for the duration of one check; the real oracle is untouched.
"""
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_0803_0048_gb300 import workloads as W

from test_oracle_symbolic import path_levels

SRC = os.path.join(os.path.dirname(oracle.__file__), "iluk_oracle.c")

MUTANTS = {
    "level_sum_drops_plus_one": ("int weight = level[i] + (int)rlev[i][q] + 1;",
                                 "int weight = level[i] + (int)rlev[i][q];"),
    "level_uses_max": ("int weight = level[i] + (int)rlev[i][q] + 1;",
                       "int weight = (level[i] > (int)rlev[i][q] ? level[i] : (int)rlev[i][q]) + 1;"),
    "fill_bound_strict": ("} else if (weight <= k) {", "} else if (weight < k) {"),
    "merge_skips_lower_fill": ("if (t <= i) continue;", "if (t <= j) continue;"),
    "multiplier_times_pivot": ("w[h] = w[h] / piv;", "w[h] = w[h] * piv;"),
    "update_adds": ("          w[j] = w[j] - prod;", "          w[j] = w[j] + prod;"),
    "forward_sweep_adds": ("""      double prod = fv[q] * x[fci[q]];
      s = s - prod;""", """      double prod = fv[q] * x[fci[q]];
      s = s + prod;"""),
    "backward_no_divide": ("    y[i] = s / fv[d];", "    y[i] = s;"),
    "tpiilu_lower_adds": ("""          double prod = lih * b[q];
          b[pos[t]] = b[pos[t]] - prod;""", """          double prod = lih * b[q];
          b[pos[t]] = b[pos[t]] + prod;"""),
    "tpiilu_no_flip": ("g[p] = (p == d) ? fv[p] : -b[p];", "g[p] = (p == d) ? fv[p] : b[p];"),
    "tpiilu_upper_unscaled": ("      double uih = fv[p] / uii;                     /* u^_ih */",
                              "      double uih = fv[p];                           /* u^_ih */"),
    "givens_sign": ("H[(i + 1) * m + j] = t4 - t3;", "H[(i + 1) * m + j] = t4 + t3;"),
    "tree_dot_skips_partner": ("for (int p = 0; p < w; ++p) part[p] = part[p] + part[p + w];",
                               "for (int p = 0; p < w; ++p) part[p] = part[p] + part[p];"),
    "adjoint_sign": ("      gA[p] = -prod;", "      gA[p] = prod;"),
    "bicgstab_omega_sign": ("      x[i] = xa + ws;", "      x[i] = xa - ws;"),
    "bicgstab_beta_inverted": ("double b1 = rho / rho_prev, b2 = alpha / omega;",
                               "double b1 = rho / rho_prev, b2 = omega / alpha;"),
    "pattern_allows_duplicates": ("if (p > rp[i] && ci[p] <= ci[p - 1])",
                                  "if (p > rp[i] && ci[p] < ci[p - 1])"),
    "pattern_allows_column_n": ("if (ci[p] < 0 || ci[p] >= n)", "if (ci[p] < 0 || ci[p] > n)"),
    "initial_level_one": ("level[t] = 0; in[t] = 1; next[t] = END;",
                          "level[t] = 1; in[t] = 1; next[t] = END;"),
    "level_keeps_larger": ("if (weight < level[t]) level[t] = weight;",
                           "if (weight > level[t]) level[t] = weight;"),
    "numeric_update_from_diagonal": ("for (int64_t q = diag[h] + 1; q < frp[h + 1]; ++q) {",
                                     "for (int64_t q = diag[h]; q < frp[h + 1]; ++q) {"),
    "forward_sweep_takes_diagonal": ("q < frp[i + 1] && fci[q] < i; ++q) {",
                                     "q < frp[i + 1] && fci[q] <= i; ++q) {"),
    "backward_sweep_skips_last": ("""    for (int64_t q = frp[i + 1] - 1; q > d; --q) {
      double prod = fv[q] * y[fci[q]];""", """    for (int64_t q = frp[i + 1] - 2; q > d; --q) {
      double prod = fv[q] * y[fci[q]];"""),
    "transpose_copies_wrong_value": ("if (v && tv) tv[dst] = v[p];",
                                     "if (v && tv) tv[dst] = v[dst];"),
    "transpose_forward_no_divide": ("    z[i] = s / tv[d];", "    z[i] = s;"),
    "iilu_apply_drops_own_term": ("      x = s + p[i];", "      x = s;"),
    "iilu_apply_no_diagonal": ("    z[i] = x / g[d];", "    z[i] = x;"),
    "spmv_reads_row_index": ("{ double prod = v[p] * x[ci[p]]; s = s + prod; }",
                             "{ double prod = v[p] * x[i]; s = s + prod; }"),
    "residual_sign": ("r[i] = b[i] - w[i];", "r[i] = w[i] - b[i];"),
    "mgs_adds": ("double prod = hij * vi[q]; w[q] = w[q] - prod;",
                 "double prod = hij * vi[q]; w[q] = w[q] + prod;"),
    "update_forgets_preconditioner": ("const double *Bas = update == ORC_UPDATE_MVY ? V : Z;",
                                      "const double *Bas = V;"),
    "mvy_update_combines_z": ("const double *Bas = update == ORC_UPDATE_MVY ? V : Z;",
                              "const double *Bas = Z;"),
    "mvy_update_skips_preconditioner": ("""      prec_apply(&M, n, u, w);
      for (int64_t q = 0; q < n; ++q) x[q] = x[q] + w[q];""",
                                        """      for (int64_t q = 0; q < n; ++q) x[q] = x[q] + u[q];"""),
    "back_substitution_transposed": ("double prod = H[i * m + l] * yv[l];",
                                     "double prod = H[l * m + i] * yv[l];"),
    "givens_cos_sin_swapped": ("cs[j] = a / rr; sn[j] = c / rr;", "cs[j] = c / rr; sn[j] = a / rr;"),
    "tree_dot_wrong_stride": ("for (int64_t i = p; i < n; i += ORC_TREE_P)",
                              "for (int64_t i = p; i < n; i += ORC_TREE_P / 2)"),
    "sequential_dot_drops_last": ("for (int64_t i = 0; i < n; ++i) { double prod = x[i] * y[i];",
                                  "for (int64_t i = 0; i + 1 < n; ++i) { double prod = x[i] * y[i];"),
    "adjoint_scatter_transposed": ("double prod = lambda[i] * x[aci[p]];",
                                   "double prod = lambda[aci[p]] * x[i];"),
    "adjoint_solves_untransposed": ("int st = orc_gmres(n, atrp, atci, atv, ORC_PREC_ILU, 1,",
                                    "int st = orc_gmres(n, arp, aci, av, ORC_PREC_ILU, 1,"),
    "transpose_backward_divides": ("""      double prod = tv[q] * y[tci[q]];
      s = s - prod;
    }
    y[i] = s;""", """      double prod = tv[q] * y[tci[q]];
      s = s - prod;
    }
    y[i] = s / tv[d];"""),
}


def build_mutant(name, tmp):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src.replace(old, new, 1)
    path_c = os.path.join(tmp, f"{name}.c")
    path_so = os.path.join(tmp, f"{name}.so")
    with open(path_c, "w") as f:
        f.write(mutated)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                    path_so, path_c, "-lm"], check=True)
    return path_so


def pins_pass():
    """A compact run of the oracle's pins; returns the names that fail."""
    failed = []
    try:  # sparse storage (Sec. 2.1): each defect reported with its row
        bad = [([0, 2, 3], [1, 0, 1], 0), ([0, 2, 3], [0, 0, 1], 0), ([0, 1, 3], [0, 0, 2], 1),
               ([0, 2, 1, 3], [0, 1, 1], 1)]
        for rp, ci, row in bad:
            if oracle.check_pattern(len(rp) - 1, rp, ci) != (oracle.EPATTERN, row):
                raise AssertionError
        if oracle.check_pattern(3, [0, 2, 3, 5], [0, 2, 1, 0, 2])[0] != 0:
            raise AssertionError
    except Exception:
        failed.append("pattern")
    try:  # Def. 2.3 against lower-numbered paths
        for n, dens, seed in [(10, 0.2, 3), (12, 0.15, 4)]:
            A = W.random_sparse(n, dens, seed, dominance=None)
            lev = path_levels(A)
            for k in range(0, 4):
                st, bad, frp, fci, flev = oracle.symbolic(A.n, A.rowptr, A.colind, k)
                got = {(i, int(fci[p])): int(flev[p]) for i in range(n)
                       for p in range(frp[i], frp[i + 1])}
                want = {(i, j): lev[i][j] for i in range(n) for j in range(n)
                        if lev[i][j] is not None and lev[i][j] <= k}
                if got != want:
                    raise AssertionError
    except Exception:
        failed.append("levels")
    try:  # complete LU when k >= n
        n = 12
        key = W.stream_key(3, "m")
        M = W.uniform(key, np.arange(n * n), -1, 1).reshape(n, n)
        M[np.arange(n), np.arange(n)] = 2 * (np.abs(M).sum(axis=0) - np.abs(np.diag(M))) + 1
        A = W.dense_to_csr(M, np.ones_like(M, dtype=bool))
        F = oracle.factor(A, 250)
        L = np.eye(n)
        U = np.zeros((n, n))
        for i in range(n):
            for p in range(F["rowptr"][i], F["rowptr"][i + 1]):
                j = int(F["colind"][p])
                (L if j < i else U)[i, j] = F["val"][p]
        _, Lr, Ur = sla.lu(M)
        if not (np.allclose(L, Lr, atol=1e-13) and np.allclose(U, Ur, atol=1e-12)):
            raise AssertionError
    except Exception:
        failed.append("dense_lu")
    try:  # sweeps, transposed sweeps, TPIILU on a full pattern
        n = 15
        key = W.stream_key(5, "m")
        M = W.uniform(key, np.arange(n * n), -1, 1).reshape(n, n)
        M[np.arange(n), np.arange(n)] = 2 * (np.abs(M).sum(axis=0) - np.abs(np.diag(M))) + 1
        A = W.dense_to_csr(M, np.ones_like(M, dtype=bool))
        F = oracle.factor(A, 250)
        p = W.uniform(W.stream_key(6, "p"), np.arange(n), -1, 1)
        ref = np.linalg.solve(M, p)
        if not np.allclose(oracle.apply(n, F["rowptr"], F["colind"], F["val"], p), ref, atol=1e-12):
            raise AssertionError("apply")
        trp, tci, tv = oracle.transpose(n, F["rowptr"], F["colind"], F["val"])
        if not np.allclose(oracle.apply_t(n, trp, tci, tv, p), np.linalg.solve(M.T, p), atol=1e-12):
            raise AssertionError("apply_t")
        g = oracle.iiluk_build(n, F["rowptr"], F["colind"], F["val"])
        if not np.allclose(oracle.iiluk_apply(n, F["rowptr"], F["colind"], g, p), ref, atol=1e-11):
            raise AssertionError("iilu")
    except Exception:
        failed.append("solves")
    try:  # GMRES and the adjoint against dense solves; tree dot vs fsum
        A = W.conv_diff(8, 2, (20.0, 20.0))
        n = A.n
        b = W.uniform(W.stream_key(7, "b"), np.arange(n), -1, 1)
        F = oracle.factor(A, 1)
        st, x, *_ = oracle.gmres(n, A.rowptr, A.colind, A.val, b, oracle.PREC_ILU,
                                 (F["rowptr"], F["colind"], F["val"]), 20, 1e-12,
                                 dotmode=oracle.DOT_TREE)
        Ad = W.csr_to_dense(A)
        if st != 0 or np.linalg.norm(x - np.linalg.solve(Ad, b)) > 1e-9 * np.linalg.norm(x):
            raise AssertionError("gmres")
        # the textbook update x += M^-1 (V y), over several restart cycles:
        # the same iterates as x += Z y in exact arithmetic, so the same
        # iteration counts and the same x to rounding level
        runs = [oracle.gmres(n, A.rowptr, A.colind, A.val, b, oracle.PREC_ILU,
                             (F["rowptr"], F["colind"], F["val"]), 4, 1e-12, update=u)
                for u in (oracle.UPDATE_Z, oracle.UPDATE_MVY)]
        (stz, xz, itz, _, cycz), (st2, x2, it2, _, cyc2) = runs
        if st2 != 0 or cyc2 < 2 or (it2, cyc2) != (itz, cycz) or \
                np.linalg.norm(x2 - xz) > 1e-10 * np.linalg.norm(xz):
            raise AssertionError("gmres mvy")
        g = W.uniform(W.stream_key(7, "g"), np.arange(n), -1, 1)
        st, lam, gA, *_ = oracle.adjoint(n, A.rowptr, A.colind, A.val, F["rowptr"], F["colind"],
                                         F["val"], x, g, 20, 1e-12)
        if np.linalg.norm(lam - np.linalg.solve(Ad.T, g)) > 1e-9 * np.linalg.norm(lam):
            raise AssertionError("adjoint")
        r = np.repeat(np.arange(n), np.diff(A.rowptr))
        if not np.array_equal(gA, -(lam[r] * x[A.colind])):
            raise AssertionError("scatter")
        # GMRES(m >= n) without preconditioning ends within one cycle
        B = W.random_sparse(20, 0.25, 9, dominance=0.9)
        bb = W.uniform(W.stream_key(9, "b"), np.arange(20), -1, 1)
        st, xb, it, rel, cyc = oracle.gmres(20, B.rowptr, B.colind, B.val, bb, oracle.PREC_NONE,
                                            None, 20, 1e-10)
        if st != 0 or cyc != 1 or it > 20:
            raise AssertionError("gmres one cycle")
        xs = W.uniform(W.stream_key(8, "x"), np.arange(9000), -1, 1)
        exact = math.fsum((xs * xs).tolist())
        for mode in (oracle.DOT_TREE, oracle.DOT_SEQ):
            if abs(oracle.dot(xs, xs, mode) - exact) > 9000 * 2.3e-16 * exact:
                raise AssertionError("dot")
    except Exception:
        failed.append("krylov")
    try:  # BiCGSTAB against a dense solve, with and without preconditioning
        A = W.conv_diff(8, 2, (20.0, 20.0))
        n = A.n
        b = W.uniform(W.stream_key(10, "b"), np.arange(n), -1, 1)
        F = oracle.factor(A, 1)
        Ad = W.csr_to_dense(A)
        xd = np.linalg.solve(Ad, b)
        for kind, Fa in ((oracle.PREC_NONE, None),
                         (oracle.PREC_ILU, (F["rowptr"], F["colind"], F["val"]))):
            st, x, it, rel, half = oracle.bicgstab(n, A.rowptr, A.colind, A.val, b, kind, Fa,
                                                   1e-12, 500, oracle.DOT_TREE)
            if st != 0 or np.linalg.norm(x - xd) > 1e-9 * np.linalg.norm(xd):
                raise AssertionError("bicgstab")
    except Exception:
        failed.append("bicgstab")
    return failed


def test_real_oracle_passes_the_compact_pins():
    assert pins_pass() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_every_planted_mistake_is_caught(name, monkeypatch):
    import ctypes
    with tempfile.TemporaryDirectory() as tmp:
        so = build_mutant(name, tmp)
        real = oracle._load()
        mutant = ctypes.CDLL(so)
        # give the mutant the same signatures as the real library
        for attr in ("orc_check_pattern", "orc_symbolic", "orc_sym_status", "orc_sym_copy",
                     "orc_sym_free", "orc_numeric", "orc_lsolve", "orc_usolve", "orc_apply",
                     "orc_apply_t", "orc_iiluk_apply", "orc_iiluk_build", "orc_transpose",
                     "orc_dot", "orc_spmv", "orc_gmres", "orc_gmres_update", "orc_adjoint",
                     "orc_bicgstab"):
            f_real, f_mut = getattr(real, attr), getattr(mutant, attr)
            f_mut.argtypes = f_real.argtypes
            f_mut.restype = f_real.restype
        monkeypatch.setattr(oracle, "_lib", mutant)
        failed = pins_pass()
    assert failed, f"mutant {name} passed every pin"
