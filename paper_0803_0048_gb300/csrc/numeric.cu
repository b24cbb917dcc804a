// numeric.cu -- a3: numeric ILU(k) factorization, row-wise IKJ elimination
// (Eq. 1; Eqs. lufactor2 and lufactor of Sec. 3.5), one warp per row.
//
// Row i is scattered from A onto F's pattern in the warp's shared-memory
// slice (fill positions +0.0).  For each h in L(i), ascending, the warp waits
// for row h to be final, forms the multiplier f_ih <- f_ih / f_hh (IEEE
// division) and applies f_ij <- f_ij - f_ih * f_hj (one rounding for the
// product, one for the difference) to every j > h of row h that row i also
// stores.  Lanes own distinct j, so each entry sees its updates in ascending
// h, exactly as the sequential algorithm does.  The finished row is written
// back and its ready flag released.
//
// The batched form runs `nbatch` value sets on the same pattern in the same
// persistent launch: tickets are handed out row-major over (row, set), so
// every set advances through the rows together and the sets' independent
// rows fill the GPU while each set's dependency chain is walked.
#include "internal.h"

namespace iluk {

constexpr int kNumThreads = 256;

__global__ void __launch_bounds__(kNumThreads)
k_numeric(int64_t n, int64_t nbatch, const int64_t *__restrict__ arp,
          const int32_t *__restrict__ a2f, const double *__restrict__ aval, int64_t astride,
          const int64_t *__restrict__ frp, const int32_t *__restrict__ fci,
          const int64_t *__restrict__ fdiag, double *fval, int64_t fstride, int *ready,
          unsigned long long *ticket, DevErr *errs, int cap, int64_t limit_ns,
          int64_t hold) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  double *svals = reinterpret_cast<double *>(smem) + (size_t)wib * cap;
  int32_t *scols = reinterpret_cast<int32_t *>(smem + (size_t)nwarps * cap * 8) + (size_t)wib * cap;
  const int64_t total = n * nbatch;

  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(ticket, 1ull);
    const int64_t t = (int64_t)__shfl_sync(FULL_MASK, tk, 0);
    if (t >= total) return;
    const int64_t row = t / nbatch;
    const int64_t set = t - row * nbatch;
    DevErr *err = errs + set;
    if (earlier_failed(err, row)) continue;
    double *fv = fval + set * fstride;
    int *rdy = ready + set * n;
    const double *av = aval + set * astride;

    const int64_t b0 = frp[row];
    const int m = (int)(frp[row + 1] - b0);
    const int dp = (int)(fdiag[row] - b0);
    const bool in_smem = m <= cap;
    const int32_t *rc = in_smem ? scols : fci + b0;
    double *rv = in_smem ? svals : fv + b0;
    if (in_smem) {
      for (int q = lane; q < m; q += 32) {
        scols[q] = fci[b0 + q];
        svals[q] = 0.0;
      }
    } else {
      for (int q = lane; q < m; q += 32) fv[b0 + q] = 0.0;
    }
    __syncwarp();
    bool bad = false;
    for (int64_t p = arp[row] + lane; p < arp[row + 1]; p += 32) {
      const double a = av[p];
      if (!isfinite(a)) bad = true;
      rv[a2f[p]] = a;
    }
    if (__any_sync(FULL_MASK, bad)) {
      if (lane == 0) set_err(err, row, ILUK_ENONFINITE);
      warp_publish(&rdy[row], lane);
      continue;
    }
    __syncwarp();

    bool ok = true;
    for (int q = 0; q < dp; ++q) {
      const int h = rc[q];
      if (!wait_flag(&rdy[h], err, row, limit_ns)) {
        ok = false;
        break;
      }
      const int64_t hd = fdiag[h];
      const double piv = *((volatile double *)&fv[hd]);
      const double fih = __ddiv_rn(rv[q], piv);
      __syncwarp();
      if (lane == 0) rv[q] = fih;
      const int64_t u1 = frp[h + 1];
      for (int64_t r = hd + 1 + lane; r < u1; r += 32) {
        const int32_t j = fci[r];
        const double fhj = *((volatile double *)&fv[r]);
        const int pos = lower_bound_i(rc, q + 1, m, j);
        if (pos < m && rc[pos] == j) rv[pos] = sub_prod(rv[pos], fih, fhj);
      }
      __syncwarp();
    }
    if (!__all_sync(FULL_MASK, ok)) {
      if (lane == 0 && !earlier_failed(err, row)) set_err(err, row, ILUK_ETIMEOUT);
      continue;
    }
    if (in_smem) {
      for (int q = lane; q < m; q += 32) fv[b0 + q] = svals[q];
    }
    __syncwarp();
    if (lane == 0 && rv[dp] == 0.0) set_err(err, row, ILUK_EZEROPIVOT);
    if (row != hold) warp_publish(&rdy[row], lane);
  }
}

static int numeric_cap(const iluk_sym *S, int *warps_out, size_t *smem_out) {
  // Per-warp slice: one row of F (double value + int32 column per entry).
  int cap = S->max_row;
  if (cap < 32) cap = 32;
  cap = (cap + 31) & ~31;
  int warps = kNumThreads / 32;
  const size_t budget = (size_t)max_smem_optin();
  while (warps > 1 && (size_t)cap * 12 * warps > budget) warps >>= 1;
  if ((size_t)cap * 12 * warps > budget) cap = (int)(budget / 12 / warps) & ~31;  // long rows in global
  *warps_out = warps;
  *smem_out = (size_t)cap * 12 * warps;
  return cap;
}

static cudaError_t launch_numeric_impl(const iluk_sym *S, int64_t nbatch, const double *avals,
                                       double *fvals, int *ready, unsigned long long *ticket,
                                       DevErr *errs, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_NUMERIC, s);
  int warps;
  size_t smem;
  const int cap = numeric_cap(S, &warps, &smem);
  cudaError_t e = cudaFuncSetAttribute(k_numeric, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_numeric, warps * 32, smem);
  if (bps < 1) bps = 1;
  int64_t grid = (int64_t)bps * num_sms();
  const int64_t want = (S->n * nbatch + warps - 1) / warps;
  if (grid > want) grid = want;
  if (grid < 1) grid = 1;
  k_numeric<<<(unsigned)grid, warps * 32, smem, s>>>(
      S->n, nbatch, S->arowptr, S->a2f, avals, S->nnzA, S->rowptr, S->colind, S->diag, fvals,
      S->nnz, ready, ticket, errs, cap, wait_limit(), hold_row());
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_numeric(const iluk_sym *S, const double *aval, double *fval, int *ready,
                           unsigned long long *ticket, DevErr *err, cudaStream_t s) {
  return launch_numeric_impl(S, 1, aval, fval, ready, ticket, err, s);
}

cudaError_t launch_numeric_batched(const iluk_sym *S, int64_t nbatch, const double *avals,
                                   double *fvals, int *ready, unsigned long long *ticket,
                                   DevErr *errs, cudaStream_t s) {
  return launch_numeric_impl(S, nbatch, avals, fvals, ready, ticket, errs, s);
}

}  // namespace iluk
