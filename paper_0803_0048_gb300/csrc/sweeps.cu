// sweeps.cu -- a4: the triangular solve L~U~ y = p applied in every Krylov
// iteration (Eq. triangleSolve), and its transpose.
//
// Forward (Eq. forwardsubA): x_i = p_i - sum_{h<i} f_ih x_h, h ascending.
// Backward: y_i = (x_i - sum_{j>i} f_ij y_j) / f_ii, j ascending.
// Each row's subtraction chain keeps the sequential order: lanes form the
// products in parallel once the rows they read are final, then the warp runs
// the chain left to right (one rounding per product, one per difference).
//
// Two schedules of the same row task:
//  * FLAGS: persistent grid over all SMs, one warp per row, rows claimed by
//    an ascending ticket, per-row ready flags in global memory (release /
//    acquire at GPU scope).  Suits wide dependency DAGs.
//  * SINGLE_CTA: one 1024-thread block on one SM, ready bits in shared
//    memory and CTA-scope ordering, so a dependency is seen within tens of
//    cycles instead of an L2 round trip.  Suits deep, narrow DAGs, where the
//    chain of row-to-row hand-offs, not bandwidth, sets the time.
//
// The transposed solve (L~U~)^-T p runs the same kernels on an explicit CSR
// transpose T = F^T: forward with division by t_ii (U~^T), then backward with
// unit diagonal (L~^T).
#include "internal.h"

namespace iluk {

constexpr int kSweepThreads = 256;
constexpr int kCtaThreads = 1024;

// sync layout: [0] ticket fwd (u64), [2] ticket bwd (u64), [4..4+n) flags
// fwd, [4+n..4+2n) flags bwd.
size_t sweep_sync_ints(int64_t n) { return 4 + 2 * (size_t)n; }

template <bool FORWARD, bool DIVIDE>
__global__ void __launch_bounds__(kSweepThreads)
k_sweep_flags(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
              const int64_t *__restrict__ dg, const double *__restrict__ v,
              const double *in, double *out, int *flag, unsigned long long *ticket,
              DevErr *err, int64_t limit_ns) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(ticket, 1ull);
    const int64_t t = (int64_t)__shfl_sync(FULL_MASK, tk, 0);
    if (t >= n) return;
    const int64_t row = FORWARD ? t : n - 1 - t;
    const int64_t d = dg[row];
    const int64_t b0 = FORWARD ? rp[row] : d + 1;
    const int64_t b1 = FORWARD ? d : rp[row + 1];
    double s = in[row];
    bool ok = true;
    for (int64_t base = b0; base < b1; base += 32) {
      const int64_t q = base + lane;
      double prod = 0.0;
      if (q < b1) {
        const int32_t c = ci[q];
        const double f = v[q];
        if (wait_flag(&flag[c], err, t, limit_ns))
          prod = __dmul_rn(f, *((volatile double *)&out[c]));
        else
          ok = false;
      }
      if (!__all_sync(FULL_MASK, ok)) break;
      const int cnt = (b1 - base) < 32 ? (int)(b1 - base) : 32;
      for (int l = 0; l < cnt; ++l) s = __dsub_rn(s, __shfl_sync(FULL_MASK, prod, l));
    }
    if (!__all_sync(FULL_MASK, ok)) {
      if (lane == 0 && !earlier_failed(err, t)) set_err(err, t, ILUK_ETIMEOUT);
      return;
    }
    if (DIVIDE) s = __ddiv_rn(s, v[d]);
    if (lane == 0) out[row] = s;
    warp_publish(&flag[row], lane);
  }
}

// Shared-memory ready bits, CTA scope.
__device__ __forceinline__ bool cta_bit(const unsigned *bits, int64_t r) {
  return (((volatile const unsigned *)bits)[r >> 5] >> (r & 31)) & 1u;
}

__device__ __forceinline__ double ld_relaxed_cta(const double *p) {
  double v;
  asm volatile("ld.relaxed.cta.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_cta(double *p, double v) {
  asm volatile("st.relaxed.cta.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

template <bool FORWARD, bool DIVIDE>
__global__ void __launch_bounds__(kCtaThreads, 1)
k_sweep_cta(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
            const int64_t *__restrict__ dg, const double *__restrict__ v, const double *in,
            double *out, DevErr *err, int64_t limit_ns) {
  extern __shared__ unsigned bits[];
  __shared__ unsigned long long sticket;
  __shared__ int sfail;
  const int64_t words = (n + 31) >> 5;
  for (int64_t w = threadIdx.x; w < words; w += blockDim.x) bits[w] = 0u;
  if (threadIdx.x == 0) {
    sticket = 0;
    sfail = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(&sticket, 1ull);
    const int64_t t = (int64_t)__shfl_sync(FULL_MASK, tk, 0);
    if (t >= n) return;
    const int64_t row = FORWARD ? t : n - 1 - t;
    const int64_t d = dg[row];
    const int64_t b0 = FORWARD ? rp[row] : d + 1;
    const int64_t b1 = FORWARD ? d : rp[row + 1];
    double s = in[row];
    bool ok = true;
    for (int64_t base = b0; base < b1; base += 32) {
      const int64_t q = base + lane;
      double prod = 0.0;
      if (q < b1) {
        const int32_t c = ci[q];
        const double f = v[q];
        if (!cta_bit(bits, c)) {
          const uint64_t t0 = globaltimer_ns();
          while (!cta_bit(bits, c)) {
            if (*((volatile int *)&sfail)) { ok = false; break; }
            if ((int64_t)(globaltimer_ns() - t0) > limit_ns) { ok = false; break; }
          }
        }
        __threadfence_block();
        prod = __dmul_rn(f, ld_relaxed_cta(&out[c]));
      }
      if (!__all_sync(FULL_MASK, ok)) break;
      const int cnt = (b1 - base) < 32 ? (int)(b1 - base) : 32;
      for (int l = 0; l < cnt; ++l) s = __dsub_rn(s, __shfl_sync(FULL_MASK, prod, l));
    }
    if (!__all_sync(FULL_MASK, ok)) {
      if (lane == 0) {
        atomicExch(&sfail, 1);
        set_err(err, t, ILUK_ETIMEOUT);
      }
      return;
    }
    if (DIVIDE) s = __ddiv_rn(s, v[d]);
    if (lane == 0) {
      st_relaxed_cta(&out[row], s);
      __threadfence_block();
      atomicOr(&bits[row >> 5], 1u << (row & 31));
    }
    __syncwarp();
  }
}

static int64_t flags_grid(int64_t n) {
  int64_t g = (int64_t)num_sms() * (2048 / kSweepThreads);
  int64_t want = (n + (kSweepThreads / 32) - 1) / (kSweepThreads / 32);
  if (g > want) g = want;
  return g < 1 ? 1 : g;
}

template <bool FORWARD, bool DIVIDE>
static cudaError_t run_sweep(int64_t n, const int64_t *rp, const int32_t *ci, const int64_t *dg,
                             const double *v, const double *in, double *out, int *flag,
                             unsigned long long *ticket, int sched, DevErr *err, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (sched == ILUK_SCHED_SINGLE_CTA) {
    const size_t smem = (size_t)((n + 31) >> 5) * 4;
    cudaError_t e = cudaFuncSetAttribute(k_sweep_cta<FORWARD, DIVIDE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sweep_cta<FORWARD, DIVIDE><<<1, kCtaThreads, smem, s>>>(n, rp, ci, dg, v, in, out, err,
                                                              wait_limit());
  } else {
    k_sweep_flags<FORWARD, DIVIDE><<<(unsigned)flags_grid(n), kSweepThreads, 0, s>>>(
        n, rp, ci, dg, v, in, out, flag, ticket, err, wait_limit());
  }
  return cudaGetLastError();
}

// Largest n whose ready bits fit one block's shared memory.
static bool cta_fits(int64_t n) {
  return (size_t)((n + 31) >> 5) * 4 + 64 <= (size_t)max_smem_optin();
}

cudaError_t launch_apply(int64_t n, const int64_t *rp, const int32_t *ci, const int64_t *dg,
                         const double *v, const double *p, double *tmp, double *y, int *sync,
                         int transpose, int sched, DevErr *err, cudaStream_t s) {
  if (sched == ILUK_SCHED_SINGLE_CTA && !cta_fits(n)) sched = ILUK_SCHED_FLAGS;
  if (sched != ILUK_SCHED_SINGLE_CTA) sched = ILUK_SCHED_FLAGS;
  unsigned long long *tick = reinterpret_cast<unsigned long long *>(sync);
  int *fl_f = sync + 4, *fl_b = sync + 4 + n;
  cudaError_t e;
  if (sched == ILUK_SCHED_FLAGS) {
    e = cudaMemsetAsync(sync, 0, sweep_sync_ints(n) * sizeof(int), s);
    if (e != cudaSuccess) return e;
  }
  if (!transpose) {
    e = run_sweep<true, false>(n, rp, ci, dg, v, p, tmp, fl_f, tick, sched, err, s);
    if (e != cudaSuccess) return e;
    return run_sweep<false, true>(n, rp, ci, dg, v, tmp, y, fl_b, tick + 1, sched, err, s);
  }
  e = run_sweep<true, true>(n, rp, ci, dg, v, p, tmp, fl_f, tick, sched, err, s);
  if (e != cudaSuccess) return e;
  return run_sweep<false, false>(n, rp, ci, dg, v, tmp, y, fl_b, tick + 1, sched, err, s);
}

// ---------------------------------------------------------------------------
// CSR transpose: count, scan, scatter, then sort every row by source row so
// that row i of T lists column i of F top to bottom.
// ---------------------------------------------------------------------------
__global__ void k_count_cols(int64_t nnz, const int32_t *__restrict__ ci, int32_t *cnt) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
       p += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[ci[p]], 1);
}

__global__ void k_scatter_t(int64_t n, const int64_t *__restrict__ rp,
                            const int32_t *__restrict__ ci, const double *__restrict__ v,
                            const int64_t *__restrict__ trp, int32_t *cursor, int32_t *tci,
                            double *tv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int32_t c = ci[p];
      const int64_t dst = trp[c] + atomicAdd(&cursor[c], 1);
      tci[dst] = (int32_t)i;
      tv[dst] = v[p];
    }
  }
}

__global__ void k_sort_rows_t(int64_t n, const int64_t *__restrict__ trp, int32_t *tci,
                              double *tv, int64_t *tdiag) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = trp[r], e = trp[r + 1];
    for (int64_t p = b + 1; p < e; ++p) {  // insertion sort by source row
      const int32_t key = tci[p];
      const double val = tv[p];
      int64_t q = p - 1;
      while (q >= b && tci[q] > key) {
        tci[q + 1] = tci[q];
        tv[q + 1] = tv[q];
        --q;
      }
      tci[q + 1] = key;
      tv[q + 1] = val;
    }
    int64_t dpos = -1;
    for (int64_t p = b; p < e; ++p)
      if (tci[p] == r) dpos = p;
    if (tdiag) tdiag[r] = dpos;
  }
}

cudaError_t launch_transpose(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *ci,
                             const double *v, int64_t *trp, int32_t *tci, double *tv,
                             int64_t *tdiag, int32_t *cursor, int64_t *scan_tmp, cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(trp, 0, sizeof(int64_t), s);
  int64_t g = (int64_t)num_sms() * 8;
  cudaError_t e = cudaMemsetAsync(cursor, 0, (size_t)n * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  k_count_cols<<<(unsigned)g, 256, 0, s>>>(nnz, ci, cursor);
  e = launch_scan_lengths(n, cursor, trp, scan_tmp, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(cursor, 0, (size_t)n * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  k_scatter_t<<<(unsigned)g, 256, 0, s>>>(n, rp, ci, v, trp, cursor, tci, tv);
  k_sort_rows_t<<<(unsigned)g, 256, 0, s>>>(n, trp, tci, tv, tdiag);
  return cudaGetLastError();
}

}  // namespace iluk
