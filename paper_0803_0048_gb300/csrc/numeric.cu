// numeric.cu -- a3: numeric ILU(k) factorization, row-wise IKJ elimination
// (Eq. 1; Eqs. lufactor2 and lufactor of Sec. 3.5), one warp per row.
//
// Row i is scattered from A onto F's pattern in the warp's shared-memory
// slice (fill positions +0.0).  For each h in L(i), ascending, the warp finds
// where row h's entries j > h fall in row i (pattern only, before row h is
// final), waits for the values of row h, forms the multiplier
// f_ih <- f_ih / f_hh (IEEE division) and applies f_ij <- f_ij - f_ih * f_hj
// (one rounding for the product, one for the difference).  Lanes own
// distinct j, so each entry sees its updates in ascending h, exactly as the
// sequential algorithm does.  The finished row is then written back.
//
// The batched form runs `nbatch` value sets on the same pattern in the same
// persistent launch: tickets are handed out row-major over (row, set), so
// every set advances through the rows together and the sets' independent
// rows fill the GPU while each set's dependency chain is walked.
#include "internal.h"

namespace iluk {

constexpr int kNumThreads = 256;

// Factor values double as ready flags: the output array is filled with
// kPendingF before the launch, and a row's entries change from kPendingF to
// their final values when the row is written back.  A row that needs pivot
// row h reads f_hh and the f_hj directly, retrying while they are pending; no
// separate flag, fence or release store is needed.  The input values are
// checked to be finite, so no computed value can equal the marker (a
// signalling NaN).
constexpr unsigned long long kPendingF = 0x7FF0DEADBEEFCAFEull;

__device__ __forceinline__ bool pend_f(double v) {
  return (unsigned long long)__double_as_longlong(v) == kPendingF;
}

__device__ __forceinline__ double ld_gpu(const double *p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

// Warp-uniform wait until the lane's value at p (lanes with active == false
// pass) is no longer pending.  Returns false on time-out or when a row
// before `row` has failed.
__device__ __forceinline__ bool wait_vals(const double *p, bool active, double *val,
                                          const DevErr *err, int64_t row, int64_t limit_ns) {
  bool pend = active && pend_f(*val);
  if (!__any_sync(FULL_MASK, pend)) return true;
  const uint64_t t0 = globaltimer_ns();
  unsigned backoff = 32;
  for (unsigned it = 0;; ++it) {
    if (pend) {
      *val = ld_gpu(p);
      pend = pend_f(*val);
    }
    if (!__any_sync(FULL_MASK, pend)) return true;
    const bool stop = (it & 7u) == 7u &&
                      (earlier_failed(err, row) || (int64_t)(globaltimer_ns() - t0) > limit_ns);
    if (__any_sync(FULL_MASK, stop)) return false;  // the whole warp gives up together
    __nanosleep(backoff);
    if (backoff < 128u) backoff <<= 1;
  }
}

// What a warp needs from pivot row h before its values are final: where
// its first 64 entries j > h fall in the current row (pos, -1 if absent),
// and loads of those values and of f_hh already issued.
struct PivotPre {
  int64_t hd, u1;
  int pos0, pos1;
  double piv, f0, f1;
};

__device__ __forceinline__ void prefetch_pivot(PivotPre &pp, int q, const int32_t *rc, int m,
                                               const int64_t *__restrict__ fdiag,
                                               const int64_t *__restrict__ frp,
                                               const int32_t *__restrict__ fci, const double *fv,
                                               int lane) {
  const int h = rc[q];
  pp.hd = fdiag[h];
  pp.u1 = frp[h + 1];
  pp.piv = ld_gpu(&fv[pp.hd]);
  pp.pos0 = pp.pos1 = -1;
  pp.f0 = pp.f1 = 0.0;
  const int64_t r0 = pp.hd + 1 + lane, r1 = r0 + 32;
  if (r0 < pp.u1) {
    const int32_t j = fci[r0];
    const int ps = lower_bound_i(rc, q + 1, m, j);
    if (ps < m && rc[ps] == j) {
      pp.pos0 = ps;
      pp.f0 = ld_gpu(&fv[r0]);
    }
  }
  if (r1 < pp.u1) {
    const int32_t j = fci[r1];
    const int ps = lower_bound_i(rc, q + 1, m, j);
    if (ps < m && rc[ps] == j) {
      pp.pos1 = ps;
      pp.f1 = ld_gpu(&fv[r1]);
    }
  }
}

__global__ void k_fill_pending_f(int64_t n, double *x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = __longlong_as_double((long long)kPendingF);
}

__global__ void __launch_bounds__(kNumThreads)
k_numeric(int64_t n, int64_t nbatch, const int64_t *__restrict__ arp,
          const int32_t *__restrict__ a2f, const double *__restrict__ aval, int64_t astride,
          const int64_t *__restrict__ frp, const int32_t *__restrict__ fci,
          const int64_t *__restrict__ fdiag, double *fval, int64_t fstride,
          unsigned long long *ticket, DevErr *errs, int cap, int64_t limit_ns, int64_t hold) {
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
    const double *av = aval + set * astride;

    const int64_t b0 = frp[row];
    const int m = (int)(frp[row + 1] - b0);
    const int dp = (int)(fdiag[row] - b0);
    // The slice holds the whole row (numeric_cap sizes it for the longest
    // row of F): the output segment cannot serve as scratch, since other rows
    // read it as soon as an entry leaves the pending state.
    const int32_t *rc = scols;
    double *rv = svals;
    for (int q = lane; q < m; q += 32) {
      scols[q] = fci[b0 + q];
      svals[q] = 0.0;
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
      continue;
    }
    __syncwarp();

    // Pivots are software-pipelined: while the values of pivot q are awaited,
    // the pattern work and the value loads of pivot q+1 are already issued.
    // A prefetch covers the first 64 entries j > h of the pivot row (two per
    // lane); longer pivot rows finish their tail inline.
    bool ok = true;
    PivotPre cur, nxt;
    if (dp > 0) prefetch_pivot(cur, 0, rc, m, fdiag, frp, fci, fv, lane);
    for (int q = 0; q < dp && ok; ++q) {
      if (q + 1 < dp) prefetch_pivot(nxt, q + 1, rc, m, fdiag, frp, fci, fv, lane);
      if (!wait_vals(&fv[cur.hd], true, &cur.piv, err, row, limit_ns) ||
          !wait_vals(&fv[cur.hd + 1 + lane], cur.pos0 >= 0, &cur.f0, err, row, limit_ns) ||
          !wait_vals(&fv[cur.hd + 33 + lane], cur.pos1 >= 0, &cur.f1, err, row, limit_ns)) {
        ok = false;
        break;
      }
      const double fih = __ddiv_rn(rv[q], cur.piv);
      __syncwarp();
      if (lane == 0) rv[q] = fih;
      if (cur.pos0 >= 0) rv[cur.pos0] = sub_prod(rv[cur.pos0], fih, cur.f0);
      if (cur.pos1 >= 0) rv[cur.pos1] = sub_prod(rv[cur.pos1], fih, cur.f1);
      for (int64_t base = cur.hd + 65; base < cur.u1; base += 32) {  // long pivot rows
        const int64_t r = base + lane;
        int pos = -1;
        double fhj = 0.0;
        if (r < cur.u1) {
          const int32_t j = fci[r];
          const int ps = lower_bound_i(rc, q + 1, m, j);
          if (ps < m && rc[ps] == j) {
            pos = ps;
            fhj = ld_gpu(&fv[r]);
          }
        }
        if (!wait_vals(&fv[r], pos >= 0, &fhj, err, row, limit_ns)) {
          ok = false;
          break;
        }
        if (pos >= 0) rv[pos] = sub_prod(rv[pos], fih, fhj);
      }
      __syncwarp();
      cur = nxt;
    }
    if (!__all_sync(FULL_MASK, ok)) {
      if (lane == 0 && !earlier_failed(err, row)) set_err(err, row, ILUK_ETIMEOUT);
      continue;
    }
    if (lane == 0 && rv[dp] == 0.0) set_err(err, row, ILUK_EZEROPIVOT);
    if (row != hold)
      for (int q = lane; q < m; q += 32) fv[b0 + q] = svals[q];
    __syncwarp();
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
  if ((size_t)cap * 12 * warps > budget) return -1;  // a row of F exceeds shared memory
  *warps_out = warps;
  *smem_out = (size_t)cap * 12 * warps;
  return cap;
}

static cudaError_t launch_numeric_impl(const iluk_sym *S, int64_t nbatch, const double *avals,
                                       double *fvals, unsigned long long *ticket, DevErr *errs,
                                       cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_NUMERIC, s);
  int warps;
  size_t smem;
  const int cap = numeric_cap(S, &warps, &smem);
  if (cap < 0) return cudaErrorMemoryAllocation;
  {
    const int64_t nv = S->nnz * nbatch;
    int64_t b = (nv + 255) / 256;
    if (b > (int64_t)num_sms() * 8) b = (int64_t)num_sms() * 8;
    if (b < 1) b = 1;
    k_fill_pending_f<<<(unsigned)b, 256, 0, s>>>(nv, fvals);
    note_launch();
  }
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
      S->nnz, ticket, errs, cap, wait_limit(), hold_row());
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_numeric(const iluk_sym *S, const double *aval, double *fval,
                           unsigned long long *ticket, DevErr *err, cudaStream_t s) {
  return launch_numeric_impl(S, 1, aval, fval, ticket, err, s);
}

cudaError_t launch_numeric_batched(const iluk_sym *S, int64_t nbatch, const double *avals,
                                   double *fvals, unsigned long long *ticket, DevErr *errs,
                                   cudaStream_t s) {
  return launch_numeric_impl(S, nbatch, avals, fvals, ticket, errs, s);
}

}  // namespace iluk
