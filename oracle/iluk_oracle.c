/*
 * iluk_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential CPU restatement of the ILU(k) method of Dong &
 * Cooperman, "A Bit-Compatible Shared Memory Parallelization for ILU(k)
 * Preconditioning and a Bit-Compatible Generalization to Distributed Memory"
 * (arXiv 0803.0048).  It exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA library against an
 * independent statement of what the method computes.  Nothing in the product
 * path links, loads or calls this file.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no -ffast-math).  Every
 * floating-point operation below is one IEEE-754 double operation rounded to
 * nearest; contraction into fused multiply-adds is disabled so that each
 * product and each difference is rounded separately.
 *
 * Conventions: 0-based indices; CSR with int64 row pointers, int32 column
 * indices sorted ascending and unique, double values.  The filled matrix F
 * holds L~ (strictly lower part, unit diagonal not stored) and U~ (diagonal
 * and upper part) in one array (Sec. 2).
 *
 * Status codes: 0 ok, 1 invalid argument, 2 bad pattern, 3 no diagonal,
 * 4 zero pivot, 5 non-finite value, 6 out of memory, 8 no convergence.
 *
 * Pins (see tests/test_oracle_*.py): symbolic levels against shortest
 * lower-numbered paths (the path form of Def. 2.3) by brute force; k >= n
 * against dense LU; tridiagonal ILU(0) against the Thomas algorithm;
 * (L~U~)_ij = a_ij on the kept pattern; TPIILU against exact inverses when
 * the pattern is full; GMRES against dense solves; the adjoint against dense
 * transposed solves and finite differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
  ORC_OK = 0, ORC_EINVAL = 1, ORC_EPATTERN = 2, ORC_ENODIAG = 3, ORC_EZEROPIVOT = 4,
  ORC_ENONFINITE = 5, ORC_ENOMEM = 6, ORC_ENOCONV = 8
};

#define ORC_KMAX 250

/* ------------------------------------------------------------------------ */
/* Pattern check (sparse storage, Sec. 2.1)                                  */
/* ------------------------------------------------------------------------ */
int orc_check_pattern(int64_t n, const int64_t *rp, const int32_t *ci, int64_t *bad_row)
{
  *bad_row = -1;
  if (n < 0 || rp[0] != 0) return ORC_EINVAL;
  for (int64_t i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) { *bad_row = i; return ORC_EPATTERN; }
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] < 0 || ci[p] >= n) { *bad_row = i; return ORC_EPATTERN; }
      if (p > rp[i] && ci[p] <= ci[p - 1]) { *bad_row = i; return ORC_EPATTERN; }
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Phase I: symbolic factorization, Algorithm 1 (Sec. 2.2) with the level    */
/* of Def. 2.3.  permitted(j) is kept as a sorted singly linked list over    */
/* column numbers; finished rows are stored in growable row-major arrays and */
/* converted to CSR at the end (the row storage of Sec. 3.4).               */
/* ------------------------------------------------------------------------ */
typedef struct {
  int status;
  int64_t bad_row;
  int64_t n, nnz;
  int64_t *rowptr;
  int32_t *col;
  uint8_t *lev;
} orc_sym;

void orc_sym_free(orc_sym *S)
{
  if (!S) return;
  free(S->rowptr); free(S->col); free(S->lev); free(S);
}

orc_sym *orc_symbolic(int64_t n, const int64_t *arp, const int32_t *aci, int k)
{
  orc_sym *S = (orc_sym *)calloc(1, sizeof(orc_sym));
  S->n = n; S->bad_row = -1;
  if (k < 0 || k > ORC_KMAX) { S->status = ORC_EINVAL; return S; }
  int64_t bad;
  int st = orc_check_pattern(n, arp, aci, &bad);
  if (st) { S->status = st; S->bad_row = bad; return S; }

  int32_t **rcol = (int32_t **)calloc((size_t)n, sizeof(int32_t *));
  uint8_t **rlev = (uint8_t **)calloc((size_t)n, sizeof(uint8_t *));
  int64_t *rlen = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  const int64_t END = n;               /* list terminator */
  int64_t *next = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  int *level = (int *)malloc((size_t)n * sizeof(int));
  char *in = (char *)calloc((size_t)n, 1);
  int64_t total = 0;

  for (int64_t j = 0; j < n; ++j) {
    /* Initialisation: admit the entries of A at level zero (Alg. 1; an      */
    /* entry stored in A counts as non-zero whatever its value).             */
    int64_t head = END, tail = END;
    for (int64_t p = arp[j]; p < arp[j + 1]; ++p) {
      int64_t t = aci[p];
      level[t] = 0; in[t] = 1; next[t] = END;
      if (head == END) head = t; else next[tail] = t;
      tail = t;
    }
    /* Row-merge update pass: each i in permitted(j), i < j, ascending,      */
    /* including entries inserted during this pass (they lie beyond i).     */
    for (int64_t i = head; i != END && i < j; i = next[i]) {
      int64_t prev = i;                 /* insertion point moves forward */
      for (int64_t q = 0; q < rlen[i]; ++q) {
        int64_t t = rcol[i][q];
        if (t <= i) continue;           /* only t in permitted(i) with t > i */
        int weight = level[i] + (int)rlev[i][q] + 1;
        if (in[t]) {
          if (weight < level[t]) level[t] = weight;
        } else if (weight <= k) {
          while (next[prev] != END && next[prev] < t) prev = next[prev];
          next[t] = next[prev];
          next[prev] = t;
          in[t] = 1;
          level[t] = weight;
        }
        if (in[t]) prev = t;
      }
    }
    /* Store row j (growable row-major storage). */
    int64_t len = 0, has_diag = 0;
    for (int64_t t = head; t != END; t = next[t]) { ++len; if (t == j) has_diag = 1; }
    rcol[j] = (int32_t *)malloc((size_t)(len ? len : 1) * sizeof(int32_t));
    rlev[j] = (uint8_t *)malloc((size_t)(len ? len : 1));
    rlen[j] = len;
    int64_t q = 0;
    for (int64_t t = head; t != END; t = next[t]) {
      rcol[j][q] = (int32_t)t;
      rlev[j][q] = (uint8_t)level[t];
      in[t] = 0;
      ++q;
    }
    total += len;
    if (!has_diag && S->status == ORC_OK) { S->status = ORC_ENODIAG; S->bad_row = j; }
  }

  /* Conversion to CSR. */
  S->nnz = total;
  S->rowptr = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  S->col = (int32_t *)malloc((size_t)(total ? total : 1) * sizeof(int32_t));
  S->lev = (uint8_t *)malloc((size_t)(total ? total : 1));
  S->rowptr[0] = 0;
  for (int64_t j = 0; j < n; ++j) {
    memcpy(S->col + S->rowptr[j], rcol[j], (size_t)rlen[j] * sizeof(int32_t));
    memcpy(S->lev + S->rowptr[j], rlev[j], (size_t)rlen[j]);
    S->rowptr[j + 1] = S->rowptr[j] + rlen[j];
    free(rcol[j]); free(rlev[j]);
  }
  free(rcol); free(rlev); free(rlen); free(next); free(level); free(in);
  return S;
}

int orc_sym_status(const orc_sym *S, int64_t *bad_row, int64_t *nnz)
{
  *bad_row = S->bad_row; *nnz = S->nnz; return S->status;
}

void orc_sym_copy(const orc_sym *S, int64_t *rowptr, int32_t *col, uint8_t *lev)
{
  memcpy(rowptr, S->rowptr, ((size_t)S->n + 1) * sizeof(int64_t));
  memcpy(col, S->col, (size_t)S->nnz * sizeof(int32_t));
  memcpy(lev, S->lev, (size_t)S->nnz);
}

/* ------------------------------------------------------------------------ */
/* Phase II: numeric factorization in IKJ order (Sec. 2.2, Eq. 1; the row    */
/* update of Eqs. lufactor2 / lufactor).  F starts as A scattered onto the   */
/* filled pattern (fill-in positions hold +0.0).  For each row i and each    */
/* h in L(i) ascending: f_ih <- f_ih / f_hh, then f_ij <- f_ij - f_ih*f_hj   */
/* for every j > h stored in row h and in row i.                             */
/* ------------------------------------------------------------------------ */
static int64_t find_col(const int32_t *ci, int64_t lo, int64_t hi, int64_t c)
{
  for (int64_t p = lo; p < hi; ++p) if (ci[p] == c) return p;
  return -1;
}

int orc_numeric(int64_t n, const int64_t *arp, const int32_t *aci, const double *av,
                const int64_t *frp, const int32_t *fci, double *fv, int64_t *bad_row)
{
  *bad_row = -1;
  int64_t *diag = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  int64_t *pos = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  double *w = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
  int st = ORC_OK;
  for (int64_t c = 0; c < n; ++c) pos[c] = -1;
  for (int64_t i = 0; i < n && st == ORC_OK; ++i) {
    diag[i] = find_col(fci, frp[i], frp[i + 1], i);
    if (diag[i] < 0) { st = ORC_ENODIAG; *bad_row = i; break; }
    for (int64_t p = frp[i]; p < frp[i + 1]; ++p) { pos[fci[p]] = p; w[fci[p]] = 0.0; }
    for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
      if (!isfinite(av[p])) { st = ORC_ENONFINITE; *bad_row = i; break; }
      if (pos[aci[p]] < 0) { st = ORC_EPATTERN; *bad_row = i; break; }
      w[aci[p]] = av[p];
    }
    if (st) break;
    for (int64_t p = frp[i]; p < diag[i]; ++p) {
      int64_t h = fci[p];
      double piv = fv[diag[h]];
      w[h] = w[h] / piv;                          /* multiplier l_ih */
      for (int64_t q = diag[h] + 1; q < frp[h + 1]; ++q) {
        int64_t j = fci[q];
        if (pos[j] >= 0) {
          double prod = w[h] * fv[q];
          w[j] = w[j] - prod;
        }
      }
    }
    for (int64_t p = frp[i]; p < frp[i + 1]; ++p) { fv[p] = w[fci[p]]; pos[fci[p]] = -1; }
    if (fv[diag[i]] == 0.0) { st = ORC_EZEROPIVOT; *bad_row = i; }
  }
  free(diag); free(pos); free(w);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Triangular sweeps, Eq. triangleSolve: L~ U~ y = p.                        */
/* Forward (Eq. forwardsubA): x_i = p_i - sum_{h<i} f_ih x_h, h ascending    */
/* (left to right, farthest column first).                                   */
/* Backward: y_i = (x_i - sum_{j>i} f_ij y_j) / f_ii, j descending: the      */
/* mirror image of the forward sweep, rows last to first and each row right  */
/* to left (the order Sec. 3.5 gives for the upper factor), so again the     */
/* farthest column is subtracted first and the nearest last.                 */
/* ------------------------------------------------------------------------ */
static int64_t diag_pos(const int64_t *frp, const int32_t *fci, int64_t i)
{
  return find_col(fci, frp[i], frp[i + 1], i);
}

void orc_lsolve(int64_t n, const int64_t *frp, const int32_t *fci, const double *fv,
                const double *p, double *x)
{
  for (int64_t i = 0; i < n; ++i) {
    double s = p[i];
    for (int64_t q = frp[i]; q < frp[i + 1] && fci[q] < i; ++q) {
      double prod = fv[q] * x[fci[q]];
      s = s - prod;
    }
    x[i] = s;
  }
}

void orc_usolve(int64_t n, const int64_t *frp, const int32_t *fci, const double *fv,
                const double *x, double *y)
{
  for (int64_t i = n - 1; i >= 0; --i) {
    int64_t d = diag_pos(frp, fci, i);
    double s = x[i];
    for (int64_t q = frp[i + 1] - 1; q > d; --q) {
      double prod = fv[q] * y[fci[q]];
      s = s - prod;
    }
    y[i] = s / fv[d];
  }
}

void orc_apply(int64_t n, const int64_t *frp, const int32_t *fci, const double *fv,
               const double *p, double *y)
{
  double *x = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
  orc_lsolve(n, frp, fci, fv, p, x);
  orc_usolve(n, frp, fci, fv, x, y);
  free(x);
}

/* ------------------------------------------------------------------------ */
/* CSR transpose (exact data movement); rows of the result are sorted by     */
/* the original row index because rows are visited in ascending order.       */
/* ------------------------------------------------------------------------ */
void orc_transpose(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                   int64_t *trp, int32_t *tci, double *tv)
{
  int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t p = 0; p < rp[n]; ++p) cnt[ci[p] + 1]++;
  trp[0] = 0;
  for (int64_t c = 0; c < n; ++c) trp[c + 1] = trp[c] + cnt[c + 1];
  for (int64_t c = 0; c < n; ++c) cnt[c] = trp[c];
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t dst = cnt[ci[p]]++;
      tci[dst] = (int32_t)i;
      if (v && tv) tv[dst] = v[p];
    }
  free(cnt);
}

/* Transposed sweeps: (L~U~)^T y = p, i.e. U~^T z = p then L~^T y = z.       */
/* On T = F^T (row i of T holds column i of F): U~^T is the part with        */
/* column <= i (diagonal u_ii at column i), L~^T the part with column > i    */
/* (unit diagonal).                                                          */
/* Forward:  z_i = (p_i - sum_{c<i} t_ic z_c) / t_ii, c ascending.           */
/* Backward: y_i = z_i - sum_{c>i} t_ic y_c, c descending, i = n-1..0.        */
void orc_apply_t(int64_t n, const int64_t *trp, const int32_t *tci, const double *tv,
                 const double *p, double *y)
{
  double *z = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
  for (int64_t i = 0; i < n; ++i) {
    int64_t d = diag_pos(trp, tci, i);
    double s = p[i];
    for (int64_t q = trp[i]; q < d; ++q) {
      double prod = tv[q] * z[tci[q]];
      s = s - prod;
    }
    z[i] = s / tv[d];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    int64_t d = diag_pos(trp, tci, i);
    double s = z[i];
    for (int64_t q = trp[i + 1] - 1; q > d; --q) {
      double prod = tv[q] * y[tci[q]];
      s = s - prod;
    }
    y[i] = s;
  }
  free(z);
}

/* ------------------------------------------------------------------------ */
/* TPIILU: level-based incomplete inverses (Sec. 3.5).                       */
/*                                                                           */
/* Lower part, Eq. inversedefine restricted to F's own L pattern:            */
/*   beta_it = f_it - sum_{t<h<i} f_ih beta_ht,                              */
/* accumulated into b_it (initially the final multiplier f_it) with h        */
/* ascending, which is the order of Eq. inversefactor inside the row loop;   */
/* the stored value is -beta_it (Eq. flipfactor), taken after every row is   */
/* done so the recurrence always reads unflipped beta.                       */
/*                                                                           */
/* Upper part, the mirror image (Sec. 3.5 runs it backwards: rows from the  */
/* last to the first, each row read right to left): with u^_it = u_it/u_ii, */
/*   gamma_it = u^_it - sum_{i<h<t} u^_ih gamma_ht,                          */
/* rows n-1..0, pivots h descending; stored value -gamma_it.                 */
/*                                                                           */
/* Output g[] is aligned with F: lower positions hold -beta, strictly upper  */
/* positions hold -gamma, diagonal positions hold u_ii.                      */
/* ------------------------------------------------------------------------ */
void orc_iiluk_build(int64_t n, const int64_t *frp, const int32_t *fci, const double *fv,
                     double *g)
{
  int64_t nnz = frp[n];
  double *b = (double *)malloc((size_t)(nnz ? nnz : 1) * sizeof(double));
  int64_t *pos = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  for (int64_t c = 0; c < n; ++c) pos[c] = -1;
  memcpy(b, fv, (size_t)nnz * sizeof(double));
  /* lower: rows ascending */
  for (int64_t i = 0; i < n; ++i) {
    int64_t d = diag_pos(frp, fci, i);
    for (int64_t p = frp[i]; p < d; ++p) pos[fci[p]] = p;
    for (int64_t p = frp[i]; p < d; ++p) {          /* pivot h = fci[p] */
      int64_t h = fci[p];
      double lih = fv[p];
      int64_t dh = diag_pos(frp, fci, h);
      for (int64_t q = frp[h]; q < dh; ++q) {       /* t < h in row h */
        int64_t t = fci[q];
        if (pos[t] >= 0) {
          double prod = lih * b[q];
          b[pos[t]] = b[pos[t]] - prod;
        }
      }
    }
    for (int64_t p = frp[i]; p < d; ++p) pos[fci[p]] = -1;
  }
  /* upper: rows descending, pivots right to left */
  for (int64_t i = n - 1; i >= 0; --i) {
    int64_t d = diag_pos(frp, fci, i);
    double uii = fv[d];
    for (int64_t p = d + 1; p < frp[i + 1]; ++p) { b[p] = fv[p] / uii; pos[fci[p]] = p; }
    for (int64_t p = frp[i + 1] - 1; p > d; --p) {  /* pivot h = fci[p], descending */
      int64_t h = fci[p];
      double uih = fv[p] / uii;                     /* u^_ih */
      int64_t dh = diag_pos(frp, fci, h);
      for (int64_t q = dh + 1; q < frp[h + 1]; ++q) {
        int64_t t = fci[q];
        if (pos[t] >= 0) {
          double prod = uih * b[q];
          b[pos[t]] = b[pos[t]] - prod;
        }
      }
    }
    for (int64_t p = d + 1; p < frp[i + 1]; ++p) pos[fci[p]] = -1;
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t d = diag_pos(frp, fci, i);
    for (int64_t p = frp[i]; p < frp[i + 1]; ++p) g[p] = (p == d) ? fv[p] : -b[p];
  }
  free(b); free(pos);
}

/* Apply, Eq. forwardsubB and its upper mirror: x_i = sum_{t<i} g_it p_t     */
/* + p_i (products summed left to right, p_i added last; an empty row gives  */
/* p_i); z_i = x_i / u_ii; y_i = sum_{t>i} g_it z_t + z_i.                   */
void orc_iiluk_apply(int64_t n, const int64_t *frp, const int32_t *fci, const double *g,
                     const double *p, double *y)
{
  double *z = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
  for (int64_t i = 0; i < n; ++i) {
    int64_t d = diag_pos(frp, fci, i);
    double x;
    if (d == frp[i]) {
      x = p[i];
    } else {
      double s = g[frp[i]] * p[fci[frp[i]]];
      for (int64_t q = frp[i] + 1; q < d; ++q) {
        double prod = g[q] * p[fci[q]];
        s = s + prod;
      }
      x = s + p[i];
    }
    z[i] = x / g[d];
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t d = diag_pos(frp, fci, i);
    if (d + 1 == frp[i + 1]) {
      y[i] = z[i];
    } else {
      double s = g[d + 1] * z[fci[d + 1]];
      for (int64_t q = d + 2; q < frp[i + 1]; ++q) {
        double prod = g[q] * z[fci[q]];
        s = s + prod;
      }
      y[i] = s + z[i];
    }
  }
  free(z);
}

/* ------------------------------------------------------------------------ */
/* Restarted GMRES(m), right preconditioned (Sec. 2: the solver works with   */
/* A U~^-1 L~^-1), x0 = 0, modified Gram-Schmidt, Givens rotations.  The     */
/* preconditioned basis vectors z_j = M^-1 v_j of a cycle are kept, and the  */
/* cycle ends with x = x + Z y (the flexible-GMRES form of Saad 1993, equal  */
/* to x + M^-1 V y in exact arithmetic for a fixed M), so no extra           */
/* application of M is needed.                                               */
/*                                                                           */
/* Inner products (Sec. 3.5 keeps them in a fixed order): mode 0 sums        */
/* x_i*y_i left to right; mode 1 uses a fixed tree: 4096 partial sums, the   */
/* p-th summing indices i = p, p+4096, ... left to right from +0.0, then a   */
/* pairwise tree s[p] = s[p] + s[p+w] for w = 2048, 1024, ..., 1.            */
/* ------------------------------------------------------------------------ */
#define ORC_TREE_P 4096

static double dot_mode(int64_t n, const double *x, const double *y, int mode)
{
  if (mode == 0) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) { double prod = x[i] * y[i]; s = s + prod; }
    return s;
  }
  double part[ORC_TREE_P];
  for (int p = 0; p < ORC_TREE_P; ++p) {
    double s = 0.0;
    for (int64_t i = p; i < n; i += ORC_TREE_P) { double prod = x[i] * y[i]; s = s + prod; }
    part[p] = s;
  }
  for (int w = ORC_TREE_P / 2; w >= 1; w /= 2)
    for (int p = 0; p < w; ++p) part[p] = part[p] + part[p + w];
  return part[0];
}

double orc_dot(int64_t n, const double *x, const double *y, int mode)
{
  return dot_mode(n, x, y, mode);
}

/* y = A x, each row summed left to right from +0.0. */
void orc_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
              const double *x, double *y)
{
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) { double prod = v[p] * x[ci[p]]; s = s + prod; }
    y[i] = s;
  }
}

enum { ORC_PREC_NONE = 0, ORC_PREC_ILU = 1, ORC_PREC_IILU = 2 };

typedef struct {
  int kind;          /* ORC_PREC_* */
  int transpose;     /* ILU only: apply (L~U~)^-T using the transposed F */
  const int64_t *frp; const int32_t *fci; const double *fv;  /* F, or F^T if transpose, or g */
} orc_prec;

static void prec_apply(const orc_prec *M, int64_t n, const double *v, double *z)
{
  if (M->kind == ORC_PREC_ILU) {
    if (M->transpose) orc_apply_t(n, M->frp, M->fci, M->fv, v, z);
    else orc_apply(n, M->frp, M->fci, M->fv, v, z);
  } else if (M->kind == ORC_PREC_IILU) {
    orc_iiluk_apply(n, M->frp, M->fci, M->fv, v, z);
  } else {
    memcpy(z, v, (size_t)n * sizeof(double));
  }
}

/* info_out: [0] iterations, [1] true relative residual, [2] cycles.        */
/* update selects how a cycle ends (both are right-preconditioned GMRES,    */
/* equal in exact arithmetic for a fixed M; they round differently):        */
/*   ORC_UPDATE_Z:   x = x + Z y, Z = the preconditioned basis z_j = M^-1 v_j */
/*                   kept during the cycle (the flexible form, Saad 1993);   */
/*   ORC_UPDATE_MVY: x = x + M^-1 (V y), only V kept (the textbook form of   */
/*                   right preconditioning, Saad & Schultz 1986).            */
/* In both, each entry of the combination is summed over j in order from    */
/* +0.0, one rounding per product and per addition.                          */
#define ORC_UPDATE_Z 0
#define ORC_UPDATE_MVY 1
int orc_gmres_update(int64_t n, const int64_t *arp, const int32_t *aci, const double *av,
                     int prec_kind, int prec_transpose,
                     const int64_t *frp, const int32_t *fci, const double *fv,
                     const double *b, double *x, int m, double rtol, int maxit, int dotmode,
                     int update, double *info_out)
{
  orc_prec M = { prec_kind, prec_transpose, frp, fci, fv };
  if (m < 1 || n < 0) return ORC_EINVAL;
  size_t N = (size_t)(n ? n : 1);
  double *V = (double *)malloc(N * (size_t)(m + 1) * sizeof(double));
  double *Z = (double *)malloc(N * (size_t)m * sizeof(double));
  double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double)); /* H[i*m+j] */
  double *cs = (double *)malloc((size_t)m * sizeof(double));
  double *sn = (double *)malloc((size_t)m * sizeof(double));
  double *gv = (double *)malloc(((size_t)m + 1) * sizeof(double));
  double *yv = (double *)malloc((size_t)m * sizeof(double));
  double *r = (double *)malloc(N * sizeof(double));
  double *w = (double *)malloc(N * sizeof(double));
  double *u = (double *)malloc(N * sizeof(double));
  int status = ORC_ENOCONV;
  int iters = 0, cycles = 0;
  double relres = 0.0;

  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  double bnorm = sqrt(dot_mode(n, b, b, dotmode));
  if (bnorm == 0.0) { status = ORC_OK; relres = 0.0; goto done; }

  for (;;) {
    /* r = b - A x */
    orc_spmv(n, arp, aci, av, x, w);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - w[i];
    double beta = sqrt(dot_mode(n, r, r, dotmode));
    relres = beta / bnorm;
    if (relres <= rtol) { status = ORC_OK; break; }
    if (iters >= maxit) { status = ORC_ENOCONV; break; }
    ++cycles;
    for (int64_t i = 0; i < n; ++i) V[i] = r[i] / beta;
    gv[0] = beta;
    int jend = -1;
    for (int j = 0; j < m; ++j) {
      double *vj = V + (size_t)j * N;
      double *zj = Z + (size_t)j * N;
      prec_apply(&M, n, vj, zj);
      orc_spmv(n, arp, aci, av, zj, w);
      for (int i = 0; i <= j; ++i) {                 /* modified Gram-Schmidt */
        double *vi = V + (size_t)i * N;
        double hij = dot_mode(n, w, vi, dotmode);
        H[i * m + j] = hij;
        for (int64_t q = 0; q < n; ++q) { double prod = hij * vi[q]; w[q] = w[q] - prod; }
      }
      double hn = sqrt(dot_mode(n, w, w, dotmode));
      H[(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {                  /* previous rotations */
        double a = H[i * m + j], c = H[(i + 1) * m + j];
        double t1 = cs[i] * a, t2 = sn[i] * c;
        double t3 = sn[i] * a, t4 = cs[i] * c;
        H[i * m + j] = t1 + t2;
        H[(i + 1) * m + j] = t4 - t3;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j];
      double aa = a * a, cc = c * c;
      double rr = sqrt(aa + cc);
      if (rr == 0.0) { status = ORC_EINVAL; goto done; }
      cs[j] = a / rr; sn[j] = c / rr;
      H[j * m + j] = rr; H[(j + 1) * m + j] = 0.0;
      gv[j + 1] = -(sn[j] * gv[j]);
      gv[j] = cs[j] * gv[j];
      ++iters;
      jend = j;
      int breakdown = (hn == 0.0);
      if (!breakdown) {
        double *vn = V + (size_t)(j + 1) * N;
        for (int64_t q = 0; q < n; ++q) vn[q] = w[q] / hn;
      }
      if (fabs(gv[j + 1]) / bnorm <= rtol || iters >= maxit || breakdown) break;
    }
    /* y = H^-1 g (back substitution), then u = Z y and x = x + u, or      */
    /* u = V y and x = x + M^-1 u                                          */
    for (int i = jend; i >= 0; --i) {
      double s = gv[i];
      for (int l = i + 1; l <= jend; ++l) { double prod = H[i * m + l] * yv[l]; s = s - prod; }
      yv[i] = s / H[i * m + i];
    }
    const double *Bas = update == ORC_UPDATE_MVY ? V : Z;
    for (int64_t q = 0; q < n; ++q) {
      double s = 0.0;
      for (int j = 0; j <= jend; ++j) { double prod = yv[j] * Bas[(size_t)j * N + q]; s = s + prod; }
      u[q] = s;
    }
    if (update == ORC_UPDATE_MVY) {
      prec_apply(&M, n, u, w);
      for (int64_t q = 0; q < n; ++q) x[q] = x[q] + w[q];
    } else {
      for (int64_t q = 0; q < n; ++q) x[q] = x[q] + u[q];
    }
  }
done:
  info_out[0] = iters; info_out[1] = relres; info_out[2] = cycles;
  free(V); free(Z); free(H); free(cs); free(sn); free(gv); free(yv); free(r); free(w); free(u);
  return status;
}

int orc_gmres(int64_t n, const int64_t *arp, const int32_t *aci, const double *av,
              int prec_kind, int prec_transpose,
              const int64_t *frp, const int32_t *fci, const double *fv,
              const double *b, double *x, int m, double rtol, int maxit, int dotmode,
              double *info_out)
{
  return orc_gmres_update(n, arp, aci, av, prec_kind, prec_transpose, frp, fci, fv, b, x, m,
                          rtol, maxit, dotmode, ORC_UPDATE_Z, info_out);
}

/* ------------------------------------------------------------------------ */
/* Preconditioned BiCGSTAB (van der Vorst 1992), the solver of the paper's    */
/* experiments (Sec. 4, through Hypre), right preconditioned, x0 = 0, shadow  */
/* residual r^ = r0 = b.  Per iteration, with every operation rounded once   */
/* and no fused multiply-add:                                                */
/*   rho = (r^, r); beta = (rho / rho_prev) * (alpha / omega);               */
/*   p = r + beta * (p - omega * v)  (p = r on the first iteration);         */
/*   p^ = M^-1 p; v = A p^; alpha = rho / (r^, v); s = r - alpha * v;        */
/*   if ||s|| / ||b|| <= rtol: x = x + alpha * p^ and stop;                  */
/*   s^ = M^-1 s; t = A s^; omega = (t, s) / (t, t);                         */
/*   x = (x + alpha * p^) + omega * s^; r = s - omega * t;                   */
/*   stop when ||r|| / ||b|| <= rtol.                                        */
/* A zero rho, (r^, v), (t, t) or omega is a breakdown (ORC_EINVAL).  The    */
/* reported residual is the true ||b - A x|| / ||b|| at exit.               */
/* info_out: [0] iterations, [1] true relative residual, [2] 1 if the solve  */
/* ended at a half step.                                                     */
/* ------------------------------------------------------------------------ */
int orc_bicgstab(int64_t n, const int64_t *arp, const int32_t *aci, const double *av,
                 int prec_kind, const int64_t *frp, const int32_t *fci, const double *fv,
                 const double *b, double *x, double rtol, int maxit, int dotmode,
                 double *info_out)
{
  orc_prec M = { prec_kind, 0, frp, fci, fv };
  if (n < 0 || maxit < 0) return ORC_EINVAL;
  size_t N = (size_t)(n ? n : 1);
  double *r = (double *)malloc(N * sizeof(double));
  double *rh = (double *)malloc(N * sizeof(double));
  double *p = (double *)calloc(N, sizeof(double));
  double *v = (double *)calloc(N, sizeof(double));
  double *ph = (double *)malloc(N * sizeof(double));
  double *sv = (double *)malloc(N * sizeof(double));
  double *sh = (double *)malloc(N * sizeof(double));
  double *t = (double *)malloc(N * sizeof(double));
  int status = ORC_ENOCONV, iters = 0, half = 0;
  double relres = 0.0;
  for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; rh[i] = b[i]; }
  double bnorm = sqrt(dot_mode(n, b, b, dotmode));
  if (bnorm == 0.0) { status = ORC_OK; goto done; }
  double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
  for (int it = 1; it <= maxit; ++it) {
    double rho = dot_mode(n, rh, r, dotmode);
    if (rho == 0.0) { status = ORC_EINVAL; break; }
    if (it == 1) {
      for (int64_t i = 0; i < n; ++i) p[i] = r[i];
    } else {
      double b1 = rho / rho_prev, b2 = alpha / omega;
      double beta = b1 * b2;
      for (int64_t i = 0; i < n; ++i) {
        double wv = omega * v[i];
        double d = p[i] - wv;
        double bd = beta * d;
        p[i] = r[i] + bd;
      }
    }
    prec_apply(&M, n, p, ph);
    orc_spmv(n, arp, aci, av, ph, v);
    double sigma = dot_mode(n, rh, v, dotmode);
    if (sigma == 0.0) { status = ORC_EINVAL; break; }
    alpha = rho / sigma;
    for (int64_t i = 0; i < n; ++i) { double av_ = alpha * v[i]; sv[i] = r[i] - av_; }
    iters = it;
    double snorm = sqrt(dot_mode(n, sv, sv, dotmode));
    if (snorm / bnorm <= rtol) {
      for (int64_t i = 0; i < n; ++i) { double ap = alpha * ph[i]; x[i] = x[i] + ap; }
      status = ORC_OK;
      half = 1;
      break;
    }
    prec_apply(&M, n, sv, sh);
    orc_spmv(n, arp, aci, av, sh, t);
    double tt = dot_mode(n, t, t, dotmode);
    if (tt == 0.0) { status = ORC_EINVAL; break; }
    double ts = dot_mode(n, t, sv, dotmode);
    omega = ts / tt;
    for (int64_t i = 0; i < n; ++i) {
      double ap = alpha * ph[i];
      double xa = x[i] + ap;
      double ws = omega * sh[i];
      x[i] = xa + ws;
      double wt = omega * t[i];
      r[i] = sv[i] - wt;
    }
    double rnorm = sqrt(dot_mode(n, r, r, dotmode));
    if (rnorm / bnorm <= rtol) { status = ORC_OK; break; }
    if (omega == 0.0) { status = ORC_EINVAL; break; }
    rho_prev = rho;
  }
  if (bnorm != 0.0) {  /* true residual */
    orc_spmv(n, arp, aci, av, x, t);
    for (int64_t i = 0; i < n; ++i) t[i] = b[i] - t[i];
    relres = sqrt(dot_mode(n, t, t, dotmode)) / bnorm;
  }
done:
  info_out[0] = iters; info_out[1] = relres; info_out[2] = half;
  free(r); free(rh); free(p); free(v); free(ph); free(sv); free(sh); free(t);
  return status;
}

/* Adjoint of x = A^-1 b for a loss with gradient gx = dL/dx:                */
/*   A^T lambda = gx (GMRES on the explicit transpose, preconditioned with   */
/*   (L~U~)^-T from the transposed factors), dL/db = lambda,                 */
/*   dL/da_ij = -lambda_i x_j on A's pattern.                                */
int orc_adjoint(int64_t n, const int64_t *arp, const int32_t *aci, const double *av,
                const int64_t *frp, const int32_t *fci, const double *fv,
                const double *x, const double *gx, double *lambda, double *gA,
                int m, double rtol, int maxit, int dotmode, double *info_out)
{
  int64_t nnzA = arp[n], nnzF = frp[n];
  int64_t *atrp = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  int32_t *atci = (int32_t *)malloc((size_t)(nnzA ? nnzA : 1) * sizeof(int32_t));
  double *atv = (double *)malloc((size_t)(nnzA ? nnzA : 1) * sizeof(double));
  int64_t *ftrp = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  int32_t *ftci = (int32_t *)malloc((size_t)(nnzF ? nnzF : 1) * sizeof(int32_t));
  double *ftv = (double *)malloc((size_t)(nnzF ? nnzF : 1) * sizeof(double));
  orc_transpose(n, arp, aci, av, atrp, atci, atv);
  orc_transpose(n, frp, fci, fv, ftrp, ftci, ftv);
  int st = orc_gmres(n, atrp, atci, atv, ORC_PREC_ILU, 1, ftrp, ftci, ftv, gx, lambda,
                     m, rtol, maxit, dotmode, info_out);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {
      double prod = lambda[i] * x[aci[p]];
      gA[p] = -prod;
    }
  free(atrp); free(atci); free(atv); free(ftrp); free(ftci); free(ftv);
  return st;
}
