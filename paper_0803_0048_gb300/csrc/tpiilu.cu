// tpiilu.cu -- a5: the level-based incomplete inverse (TPIILU, Sec. 3.5).
//
// Lower part (Eq. inversedefine restricted to F's lower pattern):
//   beta_it = f_it - sum_{t<h<i} f_ih beta_ht,
// one warp per row, rows ascending: b_i. starts as the final multipliers of
// row i; for each h in L(i) ascending, once the values of row h are final,
// b_it <- b_it - f_ih * beta_ht for every t < h stored in both rows.
// The stored value is -beta (Eq. flipfactor), so a dependant reads
// beta_ht = -g_ht, an exact negation.
//
// Upper part, the mirror image (rows last to first, pivots right to left):
//   gamma_it = u^_it - sum_{i<h<t} u^_ih gamma_ht,  u^_it = u_it / u_ii,
// stored as -gamma; the diagonal position keeps u_ii.
//
// Apply: z_i = (sum_{t<i} g_it p_t + p_i) / u_ii, then
// y_i = sum_{t>i} g_it z_t + z_i; each sum runs left to right starting from
// its first product, the own term added last (Eq. forwardsubB).
#include <mutex>

#include "internal.h"

namespace iluk {

constexpr int kIiThreads = 256;

// The output g doubles as the ready flag of each row, as in the numeric
// phase: g is filled with kPendingG before the launch and a dependant reads
// the values it needs, retrying while they are pending.
constexpr unsigned long long kPendingG = 0x7FF0DEADBEEFCAFEull;

__device__ __forceinline__ bool pend_g(double v) {
  return (unsigned long long)__double_as_longlong(v) == kPendingG;
}

__device__ __forceinline__ double ld_gpu_g(const double *p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

__global__ void k_fill_pending_g(int64_t n, double *x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = __longlong_as_double((long long)kPendingG);
}

template <bool LOWER>
__global__ void __launch_bounds__(kIiThreads)
k_iiluk_build(int64_t n, const int64_t *__restrict__ frp, const int32_t *__restrict__ fci,
              const int64_t *__restrict__ fdiag, const double *__restrict__ fval, double *g,
              unsigned long long *ticket, DevErr *err, int cap, int64_t limit_ns) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  double *rv = reinterpret_cast<double *>(smem) + (size_t)wib * cap;
  int32_t *rc = reinterpret_cast<int32_t *>(smem + (size_t)nwarps * cap * 8) + (size_t)wib * cap;

  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(ticket, 1ull);
    const int64_t t = (int64_t)__shfl_sync(FULL_MASK, tk, 0);
    if (t >= n) return;
    if (earlier_failed(err, t)) continue;
    const int64_t row = LOWER ? t : n - 1 - t;
    const int64_t d = fdiag[row];
    const int64_t s0 = LOWER ? frp[row] : d + 1;  // segment of the row handled here
    const int m = (int)((LOWER ? d : frp[row + 1]) - s0);
    const double uii = fval[d];
    for (int q = lane; q < m; q += 32) {
      rc[q] = fci[s0 + q];
      rv[q] = LOWER ? fval[s0 + q] : __ddiv_rn(fval[s0 + q], uii);
    }
    __syncwarp();
    bool ok = true;
    for (int qq = 0; qq < m && ok; ++qq) {
      const int q = LOWER ? qq : m - 1 - qq;  // pivots ascending / descending
      const int h = rc[q];
      const double coef = LOWER ? fval[s0 + q] : __ddiv_rn(fval[s0 + q], uii);
      const int64_t hd = fdiag[h];
      const int64_t r0 = LOWER ? frp[h] : hd + 1;
      const int64_t r1 = LOWER ? hd : frp[h + 1];
      for (int64_t base = r0; base < r1; base += 32) {
        const int64_t r = base + lane;
        int pos = -1;
        double gv = 0.0;
        if (r < r1) {
          const int32_t col = fci[r];
          const int lo = LOWER ? 0 : q + 1, hi = LOWER ? q : m;
          const int ps = lower_bound_i(rc, lo, hi, col);
          if (ps < hi && rc[ps] == col) {
            pos = ps;
            gv = ld_gpu_g(&g[r]);
          }
        }
        bool pend = pos >= 0 && pend_g(gv);
        if (__any_sync(FULL_MASK, pend)) {
          const uint64_t t0 = globaltimer_ns();
          unsigned backoff = 32;
          for (unsigned it = 0;; ++it) {
            if (pend) {
              gv = ld_gpu_g(&g[r]);
              pend = pend_g(gv);
            }
            if (!__any_sync(FULL_MASK, pend)) break;
            const bool stop = (it & 7u) == 7u && (earlier_failed(err, t) ||
                                                  (int64_t)(globaltimer_ns() - t0) > limit_ns);
            if (__any_sync(FULL_MASK, stop)) {  // the whole warp gives up together
              ok = false;
              break;
            }
            __nanosleep(backoff);
            if (backoff < 256u) backoff <<= 1;
          }
          if (!__all_sync(FULL_MASK, ok)) break;
        }
        // beta_ht = -g_ht (or gamma_ht = -g_ht), an exact negation
        if (pos >= 0) rv[pos] = sub_prod(rv[pos], coef, -gv);
      }
      __syncwarp();
    }
    if (!__all_sync(FULL_MASK, ok)) {
      if (lane == 0 && !earlier_failed(err, t)) set_err(err, t, ILUK_ETIMEOUT);
      continue;
    }
    for (int q = lane; q < m; q += 32) g[s0 + q] = -rv[q];
    if (!LOWER && lane == 0) g[d] = uii;
    __syncwarp();
  }
}

cudaError_t launch_iiluk_build(const iluk_sym *S, const double *fval, double *g, int *sync,
                               DevErr *err, cudaStream_t s) {
  const int64_t n = S->n;
  if (n == 0) return cudaSuccess;
  int cap = S->max_row < 32 ? 32 : ((S->max_row + 31) & ~31);
  int warps = kIiThreads / 32;
  const size_t budget = (size_t)max_smem_optin();
  while (warps > 1 && (size_t)cap * 12 * warps > budget) warps >>= 1;
  if ((size_t)cap * 12 * warps > budget) return cudaErrorMemoryAllocation;
  const size_t smem = (size_t)cap * 12 * warps;
  unsigned long long *tick = reinterpret_cast<unsigned long long *>(sync);
  cudaError_t e = cudaMemsetAsync(sync, 0, 4 * sizeof(int), s);
  if (e != cudaSuccess) return e;
  {
    int64_t b = (S->nnz + 255) / 256;
    if (b > (int64_t)num_sms() * 8) b = (int64_t)num_sms() * 8;
    if (b < 1) b = 1;
    k_fill_pending_g<<<(unsigned)b, 256, 0, s>>>(S->nnz, g);
    note_launch();
  }
  int bps = 0;
  e = cudaFuncSetAttribute(k_iiluk_build<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_iiluk_build<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_iiluk_build<true>, warps * 32, smem);
  if (bps < 1) bps = 1;
  int64_t grid = (int64_t)bps * num_sms();
  const int64_t want = (n + warps - 1) / warps;
  if (grid > want) grid = want;
  {
    ProfScope prof_scope(ILUK_PROF_IILU_BUILD, s);
    k_iiluk_build<true><<<(unsigned)grid, warps * 32, smem, s>>>(
        n, S->rowptr, S->colind, S->diag, fval, g, tick, err, cap, wait_limit());
    note_launch();
  }
  {
    ProfScope prof_scope(ILUK_PROF_IILU_BUILD, s);
    k_iiluk_build<false><<<(unsigned)grid, warps * 32, smem, s>>>(
        n, S->rowptr, S->colind, S->diag, fval, g, tick + 1, err + 1, cap, wait_limit());
    note_launch();
  }
  return cudaGetLastError();
}

// Apply: warp per row, products in parallel, ordered left-to-right sum.
template <bool LOWER>
__global__ void __launch_bounds__(256)
k_iiluk_apply(int64_t n, const int64_t *__restrict__ frp, const int32_t *__restrict__ fci,
              const int64_t *__restrict__ fdiag, const double *__restrict__ g,
              const double *__restrict__ in, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += nw) {
    const int64_t d = fdiag[row];
    const int64_t b0 = LOWER ? frp[row] : d + 1;
    const int64_t b1 = LOWER ? d : frp[row + 1];
    double s = 0.0;
    bool first = true;
    for (int64_t base = b0; base < b1; base += 32) {
      const int64_t q = base + lane;
      double prod = 0.0;
      if (q < b1) prod = __dmul_rn(g[q], in[fci[q]]);
      const int cnt = (b1 - base) < 32 ? (int)(b1 - base) : 32;
      for (int l = 0; l < cnt; ++l) {
        const double pr = __shfl_sync(FULL_MASK, prod, l);
        s = first ? pr : __dadd_rn(s, pr);
        first = false;
      }
    }
    const double own = in[row];
    double x = (b1 > b0) ? __dadd_rn(s, own) : own;
    if (LOWER) x = __ddiv_rn(x, g[d]);
    if (lane == 0) out[row] = x;
  }
}

cudaError_t launch_iiluk_apply(const iluk_sym *S, const double *g, const double *p, double *tmp,
                               double *y, cudaStream_t s) {
  const int64_t n = S->n;
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n * 32 + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  {
    ProfScope prof_scope(ILUK_PROF_IILU_APPLY, s);
    k_iiluk_apply<true><<<(unsigned)blocks, 256, 0, s>>>(n, S->rowptr, S->colind, S->diag, g, p,
                                                       tmp);
    note_launch();
  }
  {
    ProfScope prof_scope(ILUK_PROF_IILU_APPLY, s);
    k_iiluk_apply<false><<<(unsigned)blocks, 256, 0, s>>>(n, S->rowptr, S->colind, S->diag, g, tmp,
                                                        y);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace iluk

// ---------------------------------------------------------------------------
// iiluk_apply_noalloc: the TPIILU apply for callers that cannot allocate device
// memory -- code whose memory belongs to another runtime or a pre-sized pool,
// or a solve loop where allocation is not allowed.  The caller passes every
// input and output; the intermediate vector between the two mat-vecs lives
// in this file-scope array instead of a cudaMalloc'd buffer.  Every device
// that loads the library holds the array (ILUK_NOALLOC_MAX_N doubles) until
// the process exits.
// ---------------------------------------------------------------------------
static __device__ __align__(256) double g_noalloc_z[ILUK_NOALLOC_MAX_N];

namespace {
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[64] = {};  // device address of g_noalloc_z, per device
}  // namespace

extern "C" int iiluk_apply_noalloc(int64_t n, const int64_t *rowptr, const int32_t *colind,
                                   const int64_t *diag, const double *g, const double *p,
                                   double *y, void *stream) {
  using namespace iluk;
  if (n < 0 || (n > 0 && (!rowptr || !colind || !diag || !g || !p || !y))) return ILUK_EINVAL;
  if (n > ILUK_NOALLOC_MAX_N) return ILUK_ENOMEM;  // larger than the static scratch
  if (n == 0) return ILUK_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ILUK_ECUDA;
  double *z = nullptr;
  {
    // Set-up, once per device, with that device current: the host-side name
    // of the array is only a stand-in, so ask the runtime for its address.
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      double *ptr = nullptr;
      if (cudaGetSymbolAddress((void **)&ptr, g_noalloc_z) != cudaSuccess || !ptr)
        return ILUK_ECUDA;
      g_noalloc_ptr[dev] = ptr;
    }
    z = g_noalloc_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  int64_t blocks = (n * 32 + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  // The lower pass writes every z_i before the upper pass reads it, so the
  // array needs no clearing between calls.
  k_iiluk_apply<true><<<(unsigned)blocks, 256, 0, s>>>(n, rowptr, colind, diag, g, p, z);
  note_launch();
  k_iiluk_apply<false><<<(unsigned)blocks, 256, 0, s>>>(n, rowptr, colind, diag, g, z, y);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? ILUK_OK : ILUK_ECUDA;
}
