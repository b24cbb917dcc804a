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

// Segment table: for a lower entry (i,h) of F, where row h's strictly lower
// part starts and how long it is; for an upper entry (i,h), h > i, the same
// for row h's strictly upper part (start << 24 | length).  Built once per
// pattern, so a warp reaches a pivot row's segment without dependent loads.
constexpr int kSegBits = 24;

__global__ void k_tpiilu_info(int64_t n, const int64_t *__restrict__ frp,
                              const int32_t *__restrict__ fci, const int64_t *__restrict__ fdiag,
                              int64_t *tinfo) {
  const int lane = threadIdx.x & 31;
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < n; row += nw) {
    const int64_t d = fdiag[row];
    for (int64_t p = frp[row] + lane; p < frp[row + 1]; p += 32) {
      const int32_t h = fci[p];
      const int64_t hd = fdiag[h];
      int64_t v = 0;
      if (p < d) v = (frp[h] << kSegBits) | (hd - frp[h]);
      else if (p > d) v = ((hd + 1) << kSegBits) | (frp[h + 1] - hd - 1);
      tinfo[p] = v;
    }
  }
}

cudaError_t launch_tpiilu_info(int64_t n, const int64_t *frp, const int32_t *fci,
                               const int64_t *fdiag, int64_t *tinfo, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n * 32 + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  k_tpiilu_info<<<(unsigned)blocks, 256, 0, s>>>(n, frp, fci, fdiag, tinfo);
  note_launch();
  return cudaGetLastError();
}

// One pivot h of the current row, staged like the numeric phase's pivots:
// stage A issues the column loads of the first kIiPre * 32 entries of row h's
// segment; stage B turns them into positions in the current row's segment and
// issues the loads of the matching g_ht; stage C waits for whatever is still
// pending and applies the pivot.
constexpr int kIiPre = 4;

struct IiStageA {
  int64_t start;
  int len;
  int32_t j[kIiPre];
};

struct IiStageB {
  int64_t start;
  int len;
  int pos[kIiPre];
  double gv[kIiPre];
};

struct IiIndex {  // position of a column in the current row's segment
  const int32_t *rc;
  const int16_t *map;
  int32_t c0;
  int span;
  bool use_map;
  __device__ __forceinline__ int find(int32_t j, int lo, int hi) const {
    if (use_map) {
      const int d = j - c0;
      return (d >= 0 && d < span) ? (int)map[d] : -1;
    }
    const int ps = lower_bound_i(rc, lo, hi, j);
    return (ps < hi && rc[ps] == j) ? ps : -1;
  }
};

__device__ __forceinline__ void ii_stage_a(IiStageA &a, int64_t info,
                                           const int32_t *__restrict__ fci, int lane) {
  a.start = info >> kSegBits;
  a.len = (int)(info & ((1ll << kSegBits) - 1));
#pragma unroll
  for (int c = 0; c < kIiPre; ++c) {
    const int e = lane + 32 * c;
    a.j[c] = e < a.len ? fci[a.start + e] : -1;
  }
}

template <bool LOWER>
__device__ __forceinline__ void ii_stage_b(IiStageB &b, const IiStageA &a, const IiIndex &ix,
                                           int q, int m, const double *g, int lane) {
  b.start = a.start;
  b.len = a.len;
  // row h's lower entries t < h can only match positions below q; its upper
  // entries t > h only positions above q
  int lo = LOWER ? 0 : q + 1;
  const int hi = LOWER ? q : m;
#pragma unroll
  for (int c = 0; c < kIiPre; ++c) {
    b.pos[c] = -1;
    b.gv[c] = 0.0;
    if (a.j[c] >= 0) {
      const int ps = ix.find(a.j[c], lo, hi);
      if (ps >= 0) {
        lo = ps;
        b.pos[c] = ps;
        b.gv[c] = ld_gpu_g(&g[b.start + lane + 32 * c]);
      }
    }
  }
}

__device__ __forceinline__ bool ii_pending(const IiStageB &b) {
  bool p = false;
#pragma unroll
  for (int c = 0; c < kIiPre; ++c) p |= b.pos[c] >= 0 && pend_g(b.gv[c]);
  return p;
}

__device__ __forceinline__ bool ii_wait(IiStageB &b, const double *g, int lane, const DevErr *err,
                                        int64_t key, int64_t limit_ns) {
  if (!__any_sync(FULL_MASK, ii_pending(b))) return true;
  const uint64_t t0 = globaltimer_ns();
  unsigned backoff = 16;
  for (unsigned it = 0;; ++it) {
#pragma unroll
    for (int c = 0; c < kIiPre; ++c)
      if (b.pos[c] >= 0 && pend_g(b.gv[c])) b.gv[c] = ld_gpu_g(&g[b.start + lane + 32 * c]);
    if (!__any_sync(FULL_MASK, ii_pending(b))) return true;
    const bool stop = (it & 31u) == 31u &&
                      (earlier_failed(err, key) || (int64_t)(globaltimer_ns() - t0) > limit_ns);
    if (__any_sync(FULL_MASK, stop)) return false;  // the whole warp gives up together
    if (it >= 4) {
      __nanosleep(backoff);
      if (backoff < 64u) backoff <<= 1;
    }
  }
}

// One row of one pass.  key orders the rows of the pass for error reports
// (row for the lower pass, n-1-row for the upper one, as processed by the
// sequential algorithm).
template <bool LOWER>
__device__ bool ii_row(int64_t n, int64_t row, const int64_t *__restrict__ frp,
                       const int32_t *__restrict__ fci, const int64_t *__restrict__ fdiag,
                       const double *__restrict__ fval, const DivPrep *__restrict__ rdiag,
                       const int64_t *__restrict__ tinfo, double *g, DevErr *err, double *rv,
                       int64_t *sinfo, int32_t *rc, int16_t *smap, int map_cap, int64_t limit_ns,
                       int lane) {
  const int64_t key = LOWER ? row : n - 1 - row;
  const int64_t d = fdiag[row];
  const int64_t s0 = LOWER ? frp[row] : d + 1;  // segment of the row handled here
  const int m = (int)((LOWER ? d : frp[row + 1]) - s0);
  const double uii = fval[d];
  const DivPrep rr = rdiag ? rdiag[row] : div_prep(uii);
  for (int q = lane; q < m; q += 32) {
    rc[q] = fci[s0 + q];
    sinfo[q] = tinfo[s0 + q];
    rv[q] = LOWER ? fval[s0 + q] : div_fin(fval[s0 + q], rr);  // u^_it = u_it / u_ii
  }
  __syncwarp();
  IiIndex ix;
  ix.rc = rc;
  ix.map = smap;
  ix.c0 = m > 0 ? rc[0] : 0;
  ix.span = m > 0 ? rc[m - 1] - ix.c0 + 1 : 0;
  ix.use_map = ix.span <= map_cap;
  if (ix.use_map && m > 0) {
    for (int dd = lane; dd < ix.span; dd += 32) smap[dd] = -1;
    __syncwarp();
    for (int q = lane; q < m; q += 32) smap[rc[q] - ix.c0] = (int16_t)q;
  }
  __syncwarp();
  // pivots ascending (lower pass) or descending (upper pass), k-th at qk(k)
  auto qk = [&](int k) { return LOWER ? k : m - 1 - k; };
  bool ok = true;
  IiStageA sa;
  IiStageB cur, nxt;
  if (m > 0) {
    ii_stage_a(sa, sinfo[qk(0)], fci, lane);
    ii_stage_b<LOWER>(cur, sa, ix, qk(0), m, g, lane);
  }
  if (m > 1) ii_stage_a(sa, sinfo[qk(1)], fci, lane);
  for (int k = 0; k < m && ok; ++k) {
    const int q = qk(k);
    if (k + 1 < m) ii_stage_b<LOWER>(nxt, sa, ix, qk(k + 1), m, g, lane);
    if (k + 2 < m) ii_stage_a(sa, sinfo[qk(k + 2)], fci, lane);
    if (!ii_wait(cur, g, lane, err, key, limit_ns)) {
      ok = false;
      break;
    }
    // the coefficient f_ih (lower) or u^_ih (upper): earlier pivots of this
    // pass never write position q, so rv[q] still holds it
    const double coef = rv[q];
    const int nch = (cur.len + 31) >> 5;
#pragma unroll
    for (int c = 0; c < kIiPre; ++c) {
      if (c >= nch) break;
      // beta_ht = -g_ht (or gamma_ht = -g_ht), an exact negation
      if (cur.pos[c] >= 0) rv[cur.pos[c]] = sub_prod(rv[cur.pos[c]], coef, -cur.gv[c]);
    }
    for (int base = 32 * kIiPre; base < cur.len; base += 32) {  // long segments
      const int e = base + lane;
      int pos = -1;
      double gv = 0.0;
      if (e < cur.len) {
        pos = ix.find(fci[cur.start + e], LOWER ? 0 : q + 1, LOWER ? q : m);
        if (pos >= 0) gv = ld_gpu_g(&g[cur.start + e]);
      }
      bool pend = pos >= 0 && pend_g(gv);
      if (__any_sync(FULL_MASK, pend)) {
        const uint64_t t0 = globaltimer_ns();
        for (unsigned it = 0;; ++it) {
          if (pend) {
            gv = ld_gpu_g(&g[cur.start + e]);
            pend = pend_g(gv);
          }
          if (!__any_sync(FULL_MASK, pend)) break;
          const bool stop = (it & 31u) == 31u && (earlier_failed(err, key) ||
                                                  (int64_t)(globaltimer_ns() - t0) > limit_ns);
          if (__any_sync(FULL_MASK, stop)) {
            ok = false;
            break;
          }
        }
        if (!ok) break;
      }
      if (pos >= 0) rv[pos] = sub_prod(rv[pos], coef, -gv);
    }
    __syncwarp();
    cur = nxt;
  }
  if (!__all_sync(FULL_MASK, ok)) {
    if (lane == 0 && !earlier_failed(err, key)) set_err(err, key, ILUK_ETIMEOUT);
    return false;
  }
  for (int q = lane; q < m; q += 32) g[s0 + q] = -rv[q];
  if (!LOWER && lane == 0) g[d] = uii;
  __syncwarp();
  return true;
}

// Both passes in one launch: even tickets take the next row of the lower
// pass (forward level order), odd tickets the next row of the upper pass
// (backward level order).  Each pass's rows depend only on rows of the same
// pass that sit at smaller tickets, so the launch cannot deadlock.
__global__ void __launch_bounds__(kIiThreads)
k_iiluk_build(int64_t n, const int64_t *__restrict__ frp, const int32_t *__restrict__ fci,
              const int64_t *__restrict__ fdiag, const double *__restrict__ fval,
              const DivPrep *__restrict__ rdiag, const int64_t *__restrict__ tinfo,
              const int32_t *__restrict__ lord, const int32_t *__restrict__ uord, double *g,
              unsigned long long *ticket, DevErr *err, int cap, int map_cap, int64_t limit_ns) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  double *rv = reinterpret_cast<double *>(smem) + (size_t)wib * cap;
  int64_t *sinfo = reinterpret_cast<int64_t *>(smem + (size_t)nwarps * cap * 8) + (size_t)wib * cap;
  int32_t *rc = reinterpret_cast<int32_t *>(smem + (size_t)nwarps * cap * 16) + (size_t)wib * cap;
  int16_t *smap =
      reinterpret_cast<int16_t *>(smem + (size_t)nwarps * cap * 20) + (size_t)wib * map_cap;
  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(ticket, 1ull);
    const int64_t t = (int64_t)__shfl_sync(FULL_MASK, tk, 0);
    if (t >= 2 * n) return;
    const int64_t idx = t >> 1;
    if ((t & 1) == 0) {
      const int64_t row = lord ? (int64_t)lord[idx] : idx;
      if (earlier_failed(err, row)) continue;
      ii_row<true>(n, row, frp, fci, fdiag, fval, rdiag, tinfo, g, err, rv, sinfo, rc, smap,
                   map_cap, limit_ns, lane);
    } else {
      const int64_t row = uord ? (int64_t)uord[idx] : n - 1 - idx;
      if (earlier_failed(err + 1, n - 1 - row)) continue;
      ii_row<false>(n, row, frp, fci, fdiag, fval, rdiag, tinfo, g, err + 1, rv, sinfo, rc,
                    smap, map_cap, limit_ns, lane);
    }
  }
}

cudaError_t launch_iiluk_build(const iluk_sym *S, const double *fval, const DivPrep *rdiag,
                               const int64_t *tinfo, double *g, int *sync, DevErr *err,
                               cudaStream_t s) {
  const int64_t n = S->n;
  if (n == 0) return cudaSuccess;
  int cap = S->max_row < 32 ? 32 : ((S->max_row + 31) & ~31);
  const size_t budget = (size_t)max_smem_optin();
  // on wide level orders more rows in flight matter more than the column
  // map, as in the numeric phase
  const bool wide = S->levels_built && n >= kWideLevelRows * (int64_t)S->lord.nlev;
  int warps = 0, map_cap = 0;
  for (int w : {8, 4, 2, 1}) {
    for (int mc : {8192, 4096, 0})
      if ((!wide || mc == 0) && ((size_t)cap * 20 + (size_t)mc * 2) * w <= budget) {
        warps = w;
        map_cap = mc;
        break;
      }
    if (warps) break;
  }
  if (!warps) return cudaErrorMemoryAllocation;
  const size_t smem = ((size_t)cap * 20 + (size_t)map_cap * 2) * warps;
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
  e = cudaFuncSetAttribute(k_iiluk_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_iiluk_build, warps * 32, smem);
  if (bps < 1) bps = 1;
  int64_t grid = (int64_t)bps * num_sms();
  const int64_t want = (2 * n + warps - 1) / warps;
  if (grid > want) grid = want;
  const int32_t *lord = S->levels_built ? S->lord.corder : nullptr;
  const int32_t *uord = S->levels_built ? S->uord.corder : nullptr;
  ProfScope prof_scope(ILUK_PROF_IILU_BUILD, s);
  k_iiluk_build<<<(unsigned)grid, warps * 32, smem, s>>>(n, S->rowptr, S->colind, S->diag, fval,
                                                         rdiag, tinfo, lord, uord, g, tick, err,
                                                         cap, map_cap, wait_limit());
  note_launch();
  return cudaGetLastError();
}

// Apply: one thread per row, each row summed left to right from its first
// product, the own term added last (Eq. forwardsubB); the sums are chains of
// dependent FP64 additions, so a warp advances 32 rows with each instruction.
template <bool LOWER>
__global__ void __launch_bounds__(256)
k_iiluk_apply(int64_t n, const int64_t *__restrict__ frp, const int32_t *__restrict__ fci,
              const int64_t *__restrict__ fdiag, const double *__restrict__ g,
              const double *__restrict__ in, double *__restrict__ out) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = fdiag[row];
    const int64_t b0 = LOWER ? frp[row] : d + 1;
    const int64_t b1 = LOWER ? d : frp[row + 1];
    const double own = in[row];
    double x = own;
    if (b1 > b0) {
      double s = __dmul_rn(g[b0], in[fci[b0]]);
#pragma unroll 4
      for (int64_t q = b0 + 1; q < b1; ++q) s = __dadd_rn(s, __dmul_rn(g[q], in[fci[q]]));
      x = __dadd_rn(s, own);
    }
    if (LOWER) x = __ddiv_rn(x, g[d]);
    out[row] = x;
  }
}

cudaError_t launch_iiluk_apply(const iluk_sym *S, const double *g, const double *p, double *tmp,
                               double *y, cudaStream_t s) {
  const int64_t n = S->n;
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
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
  // one thread per row, as in iiluk_apply
  const unsigned blocks = (unsigned)((n + 255) / 256);
  // The lower pass writes every z_i before the upper pass reads it, so the
  // array needs no clearing between calls.  cudaLaunchKernel reports the
  // error of each launch itself, not an earlier launch's pending one.
  const double *zin = z;
  void *lower[] = {(void *)&n, (void *)&rowptr, (void *)&colind, (void *)&diag, (void *)&g,
                   (void *)&p, (void *)&z};
  void *upper[] = {(void *)&n, (void *)&rowptr, (void *)&colind, (void *)&diag, (void *)&g,
                   (void *)&zin, (void *)&y};
  if (cudaLaunchKernel((const void *)k_iiluk_apply<true>, dim3(blocks), dim3(256), lower, 0, s) !=
      cudaSuccess)
    return ILUK_ECUDA;
  note_launch();
  if (cudaLaunchKernel((const void *)k_iiluk_apply<false>, dim3(blocks), dim3(256), upper, 0, s) !=
      cudaSuccess)
    return ILUK_ECUDA;
  note_launch();
  return ILUK_OK;
}
