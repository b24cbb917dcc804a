// sweeps.cu -- a4: the triangular solve L~U~ y = p applied in every Krylov
// iteration (Eq. triangleSolve), and its transpose.
//
// Forward (Eq. forwardsubA): x_i = p_i - sum_{h<i} f_ih x_h, h ascending.
// Backward: y_i = (x_i - sum_{j>i} f_ij y_j) / f_ii, j descending (the mirror
// image: rows last to first, each row right to left).  Each row's
// subtraction chain keeps the sequential order (one rounding per product, one
// per difference); the division by f_ii runs on the integer pipes from the
// factor's fixed-point reciprocal of f_ii and gives IEEE's quotient
// (div_fin, common.cuh).
//
// Five schedules of the same row task, all bit-identical; the factor handle
// times them (the warp-per-row ones at several CTA widths) on its first
// application and keeps the fastest for each direction:
//  * WARP_CLUSTER: one warp per row in one 16-CTA thread-block cluster, x in
//    the cluster's distributed shared memory on the producer's SM; the warp
//    subtracts the longest ready prefix of its chain as values arrive, and
//    when only the last entry is missing, the lane that owns it finishes the
//    row alone (poll, multiply, subtract, divide, store).
//    Suits deep, narrow DAGs, where the hand-off latency sets the time.
//  * WARP_GRID: the same over all SMs with x in global memory (L2 hand-offs);
//    suits wide DAGs, which need many SMs in flight.
//  * FLAGS / SINGLE_CTA / CLUSTER: 32 rows of one level per warp in lockstep
//    (all SMs through L2, one SM, or one cluster); they pack the FP64 work
//    of 32 rows into each instruction but couple the rows of a warp.
// Rows are taken in level order (padded to warps for the lockstep kernels);
// every wait is bounded.
//
// The transposed solve (L~U~)^-T p runs the same kernels on an explicit CSR
// transpose T = F^T: forward with division by t_ii (U~^T), then backward with
// unit diagonal (L~^T).
#include <cstring>
#include <mutex>

#include "internal.h"

namespace iluk {

// Scratch ints kept per factor handle: the numeric phase's row ticket (rows
// hand their results over through the values themselves, so no flags).
size_t sweep_sync_ints(int64_t n) {
  (void)n;
  return 4;
}

constexpr int kCtaThreads = 1024;
constexpr int kGridThreads = 256;

// Sweep outputs double as their own ready flags: an entry holds kPending (a
// signalling NaN, which no arithmetic produces) until its row is final, so a
// row that reads x_c simply polls x_c.  No flag array, no fence, no memset.
constexpr unsigned long long kPending = 0x7FF0DEADBEEFCAFEull;
constexpr unsigned long long kQuietNaN = 0x7FF8000000000000ull;

template <bool GPU_SCOPE>
__device__ __forceinline__ double ld_val(const double *p) {
  double v;
  if (GPU_SCOPE)
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
  else
    asm volatile("ld.relaxed.cta.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

template <bool GPU_SCOPE>
__device__ __forceinline__ void st_val(double *p, double v) {
  if (GPU_SCOPE)
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
  else
    asm volatile("st.relaxed.cta.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ bool pending(double v) {
  return (unsigned long long)__double_as_longlong(v) == kPending;
}

// Wait for *p to leave the pending state; false on time-out or on a failure
// recorded by another thread.
// Rows of a sweep are taken 32 at a time from the level order (a warp's 32
// rows belong to one level, padding slots hold -1), and the warp walks the
// 32 subtraction chains in lockstep, a window of W entries at a time: it
// loads the W values each lane needs, waits (warp-uniformly) until none of
// them is pending, then forms the products and the differences with every
// lane active.  Keeping the FP64 instructions converged matters on GB300,
// where an FP64 warp instruction occupies the pipe for ~20 SM cycles however
// few lanes it serves.  Each chain still runs left to right in its own lane.
// `clear` (may alias `in`) gets kPending at position `row` once in[row] has
// been read, which re-arms the buffer the next sweep writes.
template <bool FORWARD, bool DIVIDE, bool GPU_SCOPE, int W>
__global__ void __launch_bounds__(GPU_SCOPE ? kGridThreads : kCtaThreads)
k_sweep(const int32_t *__restrict__ order, int64_t len, const int64_t *__restrict__ rp,
        const int32_t *__restrict__ ci, const int64_t *__restrict__ dg,
        const double *__restrict__ v, const DivPrep *__restrict__ rd, const double *in,
        double *out, double *clear, DevErr *err, int64_t limit_ns) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t slot0 = gw * 32; slot0 < len; slot0 += nw * 32) {
    const int64_t row = order[slot0 + lane];
    // Entry e (0-based, in subtraction order) of this row sits at
    // first + step * e: left to right in the forward sweep, right to left in
    // the backward sweep, so the nearest columns, whose rows finish last, are
    // always subtracted last.
    int64_t first = 0, d = 0;
    int mylen = 0;
    double s = 0.0;
    DivPrep rr{0ull, 1.0};
    if (row >= 0) {
      d = dg[row];
      if (DIVIDE) rr = rd[row];  // u_ii and its reciprocal, fetched off the chain
      if (FORWARD) {
        first = rp[row];
        mylen = (int)(d - first);
      } else {
        first = rp[row + 1] - 1;
        mylen = (int)(first - d);
      }
      s = in[row];
      if (clear) clear[row] = __longlong_as_double((long long)kPending);
    }
    constexpr int64_t step = FORWARD ? 1 : -1;
    const int maxlen = __reduce_max_sync(FULL_MASK, mylen);
    // Chains are right-aligned across the warp: lane entry e runs at lockstep
    // position e + (maxlen - mylen), so every lane's newest dependencies fall
    // in the last windows.
    const int off = maxlen - mylen;
    bool ok = true;
    for (int q0 = 0; q0 < maxlen; q0 += W) {
      int32_t c[W];
      double f[W], x[W];
      bool pend = false;
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int e = q0 + u - off;
        if (e >= 0 && e < mylen) {
          c[u] = ci[first + step * e];
          f[u] = v[first + step * e];
        }
      }
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int e = q0 + u - off;
        if (e >= 0 && e < mylen) {
          x[u] = ld_val<GPU_SCOPE>(&out[c[u]]);
          pend |= pending(x[u]);
        }
      }
      if (__any_sync(FULL_MASK, pend)) {
        // Re-read every still-pending value each round (they may arrive in any
        // order), sleeping briefly between rounds so that waiting warps leave
        // issue slots to the warps that can make progress.
        const uint64_t t0 = globaltimer_ns();
        unsigned backoff = 16;
        for (unsigned it = 0; __any_sync(FULL_MASK, pend); ++it) {
          pend = false;
#pragma unroll
          for (int u = 0; u < W; ++u) {
            const int e = q0 + u - off;
            if (e >= 0 && e < mylen && pending(x[u])) {
              x[u] = ld_val<GPU_SCOPE>(&out[c[u]]);
              pend |= pending(x[u]);
            }
          }
          // the decision to give up is taken by the whole warp at once
          const bool stop = (it & 15u) == 15u &&
                            (any_failed(err) || (int64_t)(globaltimer_ns() - t0) > limit_ns);
          if (__any_sync(FULL_MASK, stop)) {
            ok = false;
            break;
          }
          if (__any_sync(FULL_MASK, pend)) {
            __nanosleep(backoff);
            if (backoff < (GPU_SCOPE ? 256u : 128u)) backoff <<= 1;
          }
        }
        if (!__all_sync(FULL_MASK, ok)) break;
      }
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int e = q0 + u - off;
        if (e >= 0 && e < mylen) x[u] = __dmul_rn(f[u], x[u]);
      }
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int e = q0 + u - off;
        if (e >= 0 && e < mylen) s = __dsub_rn(s, x[u]);
      }
    }
    if (!__all_sync(FULL_MASK, ok)) {
      if (row >= 0) set_err(err, row, ILUK_ETIMEOUT);
      return;
    }
    if (DIVIDE && row >= 0) s = div_fin(s, rr);
    if (row >= 0) {
      if ((unsigned long long)__double_as_longlong(s) == kPending)
        s = __longlong_as_double((long long)kQuietNaN);
      st_val<GPU_SCOPE>(&out[row], s);
    }
  }
}

// ---------------------------------------------------------------------------
// Cluster schedule: one thread-block cluster of C CTAs (C up to 16, one per
// SM).  The sweep's output vector lives in the cluster's distributed shared
// memory -- x_i in the shared memory of CTA (i mod C), slot i / C -- so a
// dependency is handed from one SM to another through DSMEM (a few hundred
// cycles) instead of L2, while the FP64 work spreads over C SMs.  Values are
// again their own ready flags (kPending until written).  At the end each CTA
// copies its slice to the global output.  Every CTA reaches the final cluster
// barrier even after a failure, so no CTA leaves while others may still read
// its shared memory.
// ---------------------------------------------------------------------------
// The cluster width C is a power of two (lg = log2 C), so owner and slot
// are a mask and a shift: the address is computed once per value, off the
// polling loop.
__device__ __forceinline__ unsigned dsm_addr(unsigned base, int64_t i, int lg) {
  unsigned a;
  const unsigned rank = (unsigned)i & ((1u << lg) - 1u);
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(base), "r"(rank));
  return a + ((unsigned)(i >> lg) << 3);
}

__device__ __forceinline__ double ld_dsm(unsigned a) {
  unsigned long long v;
  asm volatile("ld.relaxed.cluster.shared::cluster.b64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
  return __longlong_as_double((long long)v);
}

__device__ __forceinline__ void st_dsm(unsigned a, double x) {
  asm volatile("st.relaxed.cluster.shared::cluster.b64 [%0], %1;" ::"r"(a),
               "l"((unsigned long long)__double_as_longlong(x))
               : "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

// The launch shape a cluster kernel finds, checked against the one its host
// side sized the shared memory for (cluster width, grid, dynamic shared
// memory): a launch that arrives otherwise records an error (row = width << 16
// | grid) and does nothing, rather than index past its shared memory.  The
// decision is the same in every CTA, so no CTA is left at a cluster barrier.
__device__ __forceinline__ bool cluster_launch_ok(unsigned C, int expect_c, int expect_grid,
                                                  uint64_t smem_need, DevErr *err) {
  unsigned dyn;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  const bool ok = (int)C == expect_c && (int)gridDim.x == expect_grid && smem_need <= dyn;
  if (!ok && threadIdx.x == 0 && blockIdx.x == 0)
    set_err(err, ((int64_t)C << 16) | (int64_t)gridDim.x, ILUK_ECUDA);
  return ok;
}

template <bool FORWARD, bool DIVIDE, int W>
__global__ void __launch_bounds__(kCtaThreads, 1)
k_sweep_cluster(const int32_t *__restrict__ order, int64_t len, int64_t n,
                const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                const int64_t *__restrict__ dg, const double *__restrict__ v,
                const DivPrep *__restrict__ rd, const double *in, double *out, double *clear,
                DevErr *err, int64_t limit_ns, int expect_c) {
  extern __shared__ __align__(16) double xs[];  // this CTA's slice of x
  __shared__ int sfail;
  unsigned rank, C;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(C));
  const int lg = __ffs((int)C) - 1;  // C is a power of two
  const int64_t slice = (n + C - 1) / C;
  if (!cluster_launch_ok(C, expect_c, expect_c, (uint64_t)slice * sizeof(double), err)) return;
  for (int64_t j = threadIdx.x; j < slice; j += blockDim.x)
    xs[j] = __longlong_as_double((long long)kPending);
  if (threadIdx.x == 0) sfail = 0;
  const unsigned base = (unsigned)__cvta_generic_to_shared(xs);
  cluster_sync_all();

  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)rank * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)C * (blockDim.x >> 5);
  bool ok = true;
  for (int64_t slot0 = gw * 32; slot0 < len && ok; slot0 += nw * 32) {
    const int64_t row = order[slot0 + lane];
    int64_t first = 0, d = 0;
    int mylen = 0;
    double s = 0.0;
    DivPrep rr{0ull, 1.0};
    if (row >= 0) {
      d = dg[row];
      if (DIVIDE) rr = rd[row];  // u_ii and its reciprocal, fetched off the chain
      if (FORWARD) {
        first = rp[row];
        mylen = (int)(d - first);
      } else {
        first = rp[row + 1] - 1;
        mylen = (int)(first - d);
      }
      s = in[row];
      if (clear) clear[row] = __longlong_as_double((long long)kPending);
    }
    constexpr int64_t step = FORWARD ? 1 : -1;
    const int maxlen = __reduce_max_sync(FULL_MASK, mylen);
    const int off = maxlen - mylen;
    for (int q0 = 0; q0 < maxlen; q0 += W) {
      unsigned a[W];
      double f[W], x[W];
      bool pend = false;
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int e = q0 + u - off;
        if (e >= 0 && e < mylen) {
          a[u] = dsm_addr(base, ci[first + step * e], lg);
          f[u] = v[first + step * e];
        }
      }
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int e = q0 + u - off;
        if (e >= 0 && e < mylen) {
          x[u] = ld_dsm(a[u]);
          pend |= pending(x[u]);
        }
      }
      if (__any_sync(FULL_MASK, pend)) {
        const uint64_t t0 = globaltimer_ns();
        unsigned backoff = 8;
        for (unsigned it = 0; __any_sync(FULL_MASK, pend); ++it) {
          pend = false;
#pragma unroll
          for (int u = 0; u < W; ++u) {
            const int e = q0 + u - off;
            if (e >= 0 && e < mylen && pending(x[u])) {
              x[u] = ld_dsm(a[u]);
              pend |= pending(x[u]);
            }
          }
          const bool stop = (it & 15u) == 15u &&
                            (*((volatile int *)&sfail) || any_failed(err) ||
                             (int64_t)(globaltimer_ns() - t0) > limit_ns);
          if (__any_sync(FULL_MASK, stop)) {
            ok = false;
            break;
          }
          if (__any_sync(FULL_MASK, pend) && it >= 2) {
            __nanosleep(backoff);
            if (backoff < 64u) backoff <<= 1;
          }
        }
        if (!__all_sync(FULL_MASK, ok)) {
          ok = false;
          break;
        }
      }
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int e = q0 + u - off;
        if (e >= 0 && e < mylen) x[u] = __dmul_rn(f[u], x[u]);
      }
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const int e = q0 + u - off;
        if (e >= 0 && e < mylen) s = __dsub_rn(s, x[u]);
      }
    }
    if (!ok) {
      if (lane == 0) {
        atomicExch(&sfail, 1);
        if (row >= 0) set_err(err, row, ILUK_ETIMEOUT);
        else set_err(err, n, ILUK_ETIMEOUT);
      }
      break;
    }
    if (DIVIDE && row >= 0) s = div_fin(s, rr);
    if (row >= 0) {
      if ((unsigned long long)__double_as_longlong(s) == kPending)
        s = __longlong_as_double((long long)kQuietNaN);
      st_dsm(dsm_addr(base, row, lg), s);
    }
  }
  // Every CTA arrives here, so no shared memory is released while read.
  cluster_sync_all();
  for (int64_t j = threadIdx.x; j < slice; j += blockDim.x) {
    const int64_t i = j * C + rank;
    if (i < n) out[i] = xs[j];
  }
}

// ---------------------------------------------------------------------------
// Warp-per-row schedules.  One warp owns one row (rows taken from the level
// order, so every dependency lies at an earlier position and is owned by a
// warp that is already running).  The lanes load and poll up to 32 entries at
// a time and form their products as soon as their values arrive; the warp
// then subtracts the longest ready prefix of the chain, in order, and goes
// back to polling only if the prefix stopped at a still-pending entry.  A row
// therefore pays, after its last dependency arrives, only for the rest of its
// own chain.  SCOPE 0: values in global memory, any number of SMs (a
// co-resident cooperative grid); SCOPE 1: values in the distributed shared
// memory of one thread-block cluster (as k_sweep_cluster).
// ---------------------------------------------------------------------------
template <int SCOPE>
__device__ __forceinline__ double wpr_load(const double *out, unsigned da, int64_t i) {
  if (SCOPE == 0) return ld_val<true>(&out[i]);
  return ld_dsm(da);
}

// Prefix helpers (ILUK_SCHED_WARP_CLUSTER_HELP).  The FP64 pipes of the
// cluster's SMs are kept busy by the rows' subtraction chains (one warp
// instruction per entry, however few lanes it serves), and that queueing
// delays the few FP64 operations on the critical path.  A second cluster of
// the same cooperative launch therefore takes most of each chain: its warps
// walk the slots in order, one row per warp, and for slot s, once the row at
// slot s - lag is final, subtract the products of the row's leading entries
// whose x is already final (read from a global copy of x that the row warps
// keep), stopping at the first one that is not, and publish the partial
// difference with the number of entries it covers.  The row's own warp,
// when it takes the row, starts from there.  Same products, same
// differences, same order: the result does not change.  A prefix is tagged
// with the launch's epoch (a device word the last CTA of the launch advances),
// so one left over from an earlier launch is never used; a row whose prefix
// is not published in time is simply done in full by its warp, which never
// waits for a helper.
template <bool FORWARD>
__device__ void sweep_prefixes(const int32_t *__restrict__ order, int64_t len,
                               const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               const int64_t *__restrict__ dg, const double *__restrict__ v,
                               const double *in, const double *xg, double *pre_s,
                               unsigned long long *pre_k, unsigned epoch, int64_t hid,
                               int64_t hp, int64_t lag, const DevErr *err, int64_t limit_ns,
                               int lane) {
  for (int64_t slot = hid; slot < len; slot += hp) {
    const int64_t ps = slot - lag;
    if (ps >= 0) {  // pace: start once the row at slot ps is final
      bool ok = true;
      if (lane == 0) {
        const double *pa = &xg[order[ps]];
        const uint64_t t0 = globaltimer_ns();
        for (unsigned it = 0;; ++it) {
          if (!pending(ld_val<true>(pa))) break;
          if ((it & 15u) == 15u &&
              (any_failed(err) || (int64_t)(globaltimer_ns() - t0) > limit_ns)) {
            ok = false;
            break;
          }
          __nanosleep(128);
        }
      }
      if (!__shfl_sync(FULL_MASK, ok ? 1 : 0, 0)) return;  // stop helping
    }
    const int64_t row = order[slot];
    if (!pending(ld_val<true>(&xg[row]))) continue;  // the row is done already
    const int64_t d = dg[row];
    const int64_t first = FORWARD ? rp[row] : rp[row + 1] - 1;
    const int mylen = (int)(FORWARD ? d - first : first - d);
    constexpr int64_t step = FORWARD ? 1 : -1;
    double s = in[row];
    int covered = 0;
    for (int b = 0; b < mylen; b += 32) {
      const int e = b + lane;
      const int cnt = mylen - b < 32 ? mylen - b : 32;
      double prod = 0.0;
      bool have = e >= mylen;
      if (e < mylen) {
        const double x = ld_val<true>(&xg[ci[first + step * e]]);
        if (!pending(x)) {
          prod = __dmul_rn(v[first + step * e], x);
          have = true;
        }
      }
      const unsigned ready = __ballot_sync(FULL_MASK, have);
      const int run = ready == FULL_MASK ? 32 : __ffs(~ready) - 1;
      const int upto = run < cnt ? run : cnt;
      for (int j = 0; j < upto; ++j) s = __dsub_rn(s, __shfl_sync(FULL_MASK, prod, j));
      covered += upto;
      if (upto < cnt) break;
    }
    if (covered > 0 && lane == 0) {
      pre_s[row] = s;
      __threadfence();  // the difference before the count that publishes it
      asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(pre_k + row),
                   "l"(((unsigned long long)epoch << 32) | (unsigned)covered)
                   : "memory");
    }
    __syncwarp();
  }
}

template <bool FORWARD, bool DIVIDE, int SCOPE>
__device__ __forceinline__ void
sweep_wpr_body(const int32_t *__restrict__ order, int64_t len, int64_t n,
               const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
               const int64_t *__restrict__ dg, const double *__restrict__ v,
               const DivPrep *__restrict__ rd, const double *in, double *out, double *clear,
               DevErr *err, int64_t limit_ns, const int32_t *__restrict__ owner, double *pre_s,
               unsigned long long *pre_k, unsigned *aux_words, int64_t lag, int expect_c,
               int expect_grid) {
  // SCOPE 1: x_i lives in the shared memory of the CTA whose warp computes
  // row i, at slot (k * wpc + warp) for the warp's k-th row; owner[i] holds
  // (rank << 26 | slot), so the producer's store stays on its own SM and only
  // the dependants' polls cross SMs.  With prefix helpers (pre_s non-null) the
  // launch holds a second cluster of helper CTAs (blockIdx.x >= C), and the
  // row warps also keep x in `out` (armed with kPending on entry) for them.
  extern __shared__ __align__(16) double xs[];
  unsigned rank = 0, C = 1, base = 0;
  const int wpc = blockDim.x >> 5;  // warps per CTA
  const bool help = SCOPE == 1 && pre_s != nullptr;
  const unsigned epoch = help ? *((volatile unsigned *)aux_words) : 0u;
  int64_t slice = 0;
  if (SCOPE == 1) {
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(C));
    const int64_t nwc = (int64_t)C * wpc;
    slice = (len + nwc - 1) / nwc * wpc;
    if (!cluster_launch_ok(C, expect_c, expect_grid, (uint64_t)slice * sizeof(double), err))
      return;
    for (int64_t j = threadIdx.x; j < slice; j += blockDim.x)
      xs[j] = __longlong_as_double((long long)kPending);
    base = (unsigned)__cvta_generic_to_shared(xs);
    cluster_sync_all();
  }
  const int lane = threadIdx.x & 31;
  const int64_t gw = SCOPE == 1 ? (int64_t)rank * wpc + (threadIdx.x >> 5)
                                : ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = SCOPE == 1 ? (int64_t)C * wpc : ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned own_slot = 0;  // SCOPE 1: the slot of this warp's current row
  unsigned own_base = 0;
  if (SCOPE == 1) asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(own_base) : "r"(base), "r"(rank));
  bool ok = true;
  if (help && blockIdx.x >= C) {  // a helper CTA: no rows of its own
    const int hw = (int)(blockDim.x >> 5);
    sweep_prefixes<FORWARD>(order, len, rp, ci, dg, v, in, out, pre_s, pre_k, epoch,
                            (int64_t)(blockIdx.x - C) * hw + (threadIdx.x >> 5),
                            (int64_t)(gridDim.x - C) * hw, lag, err, limit_ns, lane);
    ok = false;
  }
  for (int64_t slot = gw; slot < len && ok; slot += nw, own_slot += wpc) {
    const int64_t row = order[slot];
    if (row < 0) continue;
    const int64_t d = dg[row];
    DivPrep rr{0ull, 1.0};
    if (DIVIDE) rr = rd[row];  // u_ii and its reciprocal, fetched off the chain
    const int64_t first = FORWARD ? rp[row] : rp[row + 1] - 1;
    const int mylen = (int)(FORWARD ? d - first : first - d);
    constexpr int64_t step = FORWARD ? 1 : -1;
    double s = in[row];
    int k0 = 0;  // leading entries a helper has subtracted already
    if (help) {
      unsigned long long pk = 0;
      if (lane == 0)
        asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(pk) : "l"(pre_k + row));
      pk = __shfl_sync(FULL_MASK, pk, 0);
      if ((unsigned)(pk >> 32) == epoch) {
        __threadfence();  // the difference was written before the count
        k0 = (int)(pk & 0xffffffffu);
        s = ld_val<true>(&pre_s[row]);
      }
    }
    // where x_row goes: this CTA's slot for the warp's current row
    const unsigned sa = SCOPE == 1 ? own_base + ((own_slot + (threadIdx.x >> 5)) << 3) : 0u;
    if (clear && lane == 0) clear[row] = __longlong_as_double((long long)kPending);
    bool stored = false;  // the last-entry path below stored x_row already
    for (int b = k0; b < mylen && ok; b += 32) {
      const int e = b + lane;
      const bool act = e < mylen;
      const int cnt = (mylen - b) < 32 ? mylen - b : 32;
      const bool last_batch = b + 32 >= mylen;
      int32_t c = 0;
      unsigned da = 0;
      double f = 0.0, x = 0.0, prod = 0.0;
      bool have = !act;
      if (act) {
        c = ci[first + step * e];
        f = v[first + step * e];
        if (SCOPE == 1) {
          const unsigned oc = (unsigned)owner[c];
          unsigned a;
          asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(base), "r"(oc >> 26));
          da = a + ((oc & ((1u << 26) - 1u)) << 3);
        }
        x = wpr_load<SCOPE>(out, da, c);
        if (!pending(x)) {
          prod = __dmul_rn(f, x);
          have = true;
        }
      }
      int done = 0;
      const uint64_t t0 = globaltimer_ns();
      unsigned backoff = 8;
      for (unsigned it = 0;; ++it) {
        const unsigned ready = __ballot_sync(FULL_MASK, have);
        const unsigned rest = ~(ready >> done);  // first not-ready lane at or after `done`
        const int run = rest == 0u ? 32 - done : __ffs(rest) - 1;
        const int upto = done + run < cnt ? done + run : cnt;
        for (int j = done; j < upto; ++j) s = __dsub_rn(s, __shfl_sync(FULL_MASK, prod, j));
        done = upto;
        if (done >= cnt) break;
        if (last_batch && done == cnt - 1) {
          // Only the row's last entry is missing (most often the one from
          // the row that finished last): the lane that owns it polls alone,
          // then subtracts, divides and stores, with no warp vote or shuffle
          // between the value's arrival and the store.  Same operations,
          // same order.
          bool gave_up = false;
          if (lane == done) {
            for (unsigned jt = 0; !have; ++jt) {
              x = wpr_load<SCOPE>(out, da, c);
              if (!pending(x)) {
                prod = __dmul_rn(f, x);
                have = true;
              } else if ((jt & 15u) == 15u &&
                         (any_failed(err) || (int64_t)(globaltimer_ns() - t0) > limit_ns)) {
                gave_up = true;
                break;
              } else if (SCOPE == 0) {
                __nanosleep(backoff);
                if (backoff < 128u) backoff <<= 1;
              }
            }
            if (!gave_up) {
              double r = __dsub_rn(s, prod);
              if (DIVIDE) r = div_fin(r, rr);
              if ((unsigned long long)__double_as_longlong(r) == kPending)
                r = __longlong_as_double((long long)kQuietNaN);
              if (SCOPE == 0) {
                st_val<true>(&out[row], r);
              } else {
                st_dsm(sa, r);
                if (help) st_val<true>(&out[row], r);  // the helpers' copy
              }
            }
          }
          ok = __shfl_sync(FULL_MASK, gave_up ? 0 : 1, done) != 0;
          stored = ok;
          break;
        }
        const bool stop = (it & 15u) == 15u &&
                          (any_failed(err) || (int64_t)(globaltimer_ns() - t0) > limit_ns);
        if (__any_sync(FULL_MASK, stop)) {
          ok = false;
          break;
        }
        // grid: back off (L2 polls compete with the stores they wait for);
        // cluster: spin, a DSMEM poll is cheap and sleeping measured slower
        if (SCOPE == 0) {
          __nanosleep(backoff);
          if (backoff < 128u) backoff <<= 1;
        }
        if (!have) {
          x = wpr_load<SCOPE>(out, da, c);
          if (!pending(x)) {
            prod = __dmul_rn(f, x);
            have = true;
          }
        }
      }
    }
    if (!ok) {
      if (lane == 0) set_err(err, row, ILUK_ETIMEOUT);
      break;
    }
    if (stored) {
      __syncwarp();
      continue;
    }
    if (DIVIDE) s = div_fin(s, rr);
    if ((unsigned long long)__double_as_longlong(s) == kPending)
      s = __longlong_as_double((long long)kQuietNaN);
    if (lane == 0) {
      if (SCOPE == 0) {
        st_val<true>(&out[row], s);
      } else {
        st_dsm(sa, s);
        if (help) st_val<true>(&out[row], s);  // the helpers' copy
      }
    }
    __syncwarp();
  }
  if (SCOPE == 1) {
    cluster_sync_all();
    if (!help)  // with helpers every row already wrote its x to out
      for (int64_t j = threadIdx.x; j < slice; j += blockDim.x) {
        const int64_t pos = (j / wpc) * nw + (int64_t)rank * wpc + j % wpc;
        if (pos < len) out[order[pos]] = xs[j];
      }
    if (help) {
      // the last CTA to finish advances the epoch: every CTA read it at its
      // start and published its last prefix before arriving here
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&aux_words[1], 1u) == gridDim.x - 1) {
          aux_words[1] = 0u;
          __threadfence();
          aux_words[0] = epoch + 1u == 0xffffffffu ? 0u : epoch + 1u;
        }
      }
    }
  }
}

#define ILUK_WPR_PARAMS                                                                     \
  const int32_t *__restrict__ order, int64_t len, int64_t n, const int64_t *__restrict__ rp,  \
      const int32_t *__restrict__ ci, const int64_t *__restrict__ dg,                         \
      const double *__restrict__ v, const DivPrep *__restrict__ rd, const double *in,         \
      double *out, double *clear, DevErr *err, int64_t limit_ns,                              \
      const int32_t *__restrict__ owner, double *pre_s, unsigned long long *pre_k,            \
      unsigned *aux_words, int64_t lag, int expect_c, int expect_grid
#define ILUK_WPR_ARGS                                                                      \
  order, len, n, rp, ci, dg, v, rd, in, out, clear, err, limit_ns, owner, pre_s, pre_k,     \
      aux_words, lag, expect_c, expect_grid

// Warp-per-row sweeps: SCOPE 0 on a grid, SCOPE 1 on one cluster whose width
// the launch gives.
template <bool FORWARD, bool DIVIDE, int SCOPE>
__global__ void __launch_bounds__(kCtaThreads, 1) k_sweep_wpr(ILUK_WPR_PARAMS) {
  sweep_wpr_body<FORWARD, DIVIDE, SCOPE>(ILUK_WPR_ARGS);
}

// The helped form: a cooperative launch of two clusters of kHelpCluster CTAs,
// the sweep's and the helpers'.  The cluster width is part of the kernel
// (not an attribute of the launch), so every path that launches it gets it.
constexpr int kHelpCluster = 16;
template <bool FORWARD, bool DIVIDE>
__global__ void __cluster_dims__(kHelpCluster, 1, 1) __launch_bounds__(kCtaThreads, 1)
    k_sweep_wpr_help(ILUK_WPR_PARAMS) {
  sweep_wpr_body<FORWARD, DIVIDE, 1>(ILUK_WPR_ARGS);
}
#undef ILUK_WPR_PARAMS
#undef ILUK_WPR_ARGS

// owner[order[pos]] = (rank << 26 | slot) for the CTA layout above.
__global__ void k_owner_codes(const int32_t *__restrict__ order, int64_t len, int C, int wpc,
                              int32_t *owner) {
  const int64_t nw = (int64_t)C * wpc;
  for (int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < len;
       pos += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = pos % nw;
    const int64_t slot = (pos / nw) * wpc + g % wpc;
    owner[order[pos]] = (int32_t)(((g / wpc) << 26) | slot);
  }
}

// The (cached) owner codes of a level order for one cluster and CTA width.
static std::mutex g_owner_mu;
static const int32_t *owner_codes(const LevelOrder &lo_c, int64_t n, int C, int threads,
                                  cudaStream_t s) {
  LevelOrder &lo = const_cast<LevelOrder &>(lo_c);  // a cache of the order
  std::lock_guard<std::mutex> lk(g_owner_mu);
  for (OwnerCode &oc : lo.owner)
    if (oc.code && oc.C == C && oc.threads == threads) return oc.code;
  OwnerCode *slot = nullptr;
  for (OwnerCode &oc : lo.owner)
    if (!oc.code) {
      slot = &oc;
      break;
    }
  if (!slot) {  // full: reuse the first entry (stream order keeps its users safe)
    slot = &lo.owner[0];
    cudaFreeAsync(slot->code, s);
    slot->code = nullptr;
  }
  if (cudaMallocAsync((void **)&slot->code, (size_t)(n > 0 ? n : 1) * sizeof(int32_t), s) !=
      cudaSuccess) {
    slot->code = nullptr;
    return nullptr;
  }
  int64_t b = (lo.clen + 255) / 256;
  if (b > (int64_t)num_sms() * 8) b = (int64_t)num_sms() * 8;
  if (b < 1) b = 1;
  k_owner_codes<<<(unsigned)b, 256, 0, s>>>(lo.corder, lo.clen, C, threads / 32, slot->code);
  note_launch();
  slot->C = C;
  slot->threads = threads;
  return slot->code;
}

__global__ void k_fill_pending(int64_t n, double *x, unsigned long long bits) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = __longlong_as_double((long long)bits);
}

static cudaError_t fill_bits(int64_t n, double *x, unsigned long long bits, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (b > cap) b = cap;
  k_fill_pending<<<(unsigned)b, 256, 0, s>>>(n, x, bits);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_fill_pending(int64_t n, double *x, cudaStream_t s) {
  return fill_bits(n, x, kPending, s);
}

cudaError_t launch_fill_value(int64_t n, double *x, double v, cudaStream_t s) {
  unsigned long long bits;
  std::memcpy(&bits, &v, sizeof bits);
  return fill_bits(n, x, bits, s);
}

// q_i = a_i / b_i through div_prep + div_fin, the division of the numeric
// phase's multipliers and of the sweeps.
__global__ void k_div_check(int64_t n, const double *__restrict__ a,
                            const double *__restrict__ b, double *__restrict__ q) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    q[i] = div_int(a[i], b[i]);
}

cudaError_t launch_div_check(int64_t n, const double *a, const double *b, double *q,
                             cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t g = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (g > cap) g = cap;
  k_div_check<<<(unsigned)g, 256, 0, s>>>(n, a, b, q);
  note_launch();
  return cudaGetLastError();
}

// Cluster width for n rows: the largest of 16, 8, 4, 2 whose slices fit in
// one CTA's shared memory and that the device can schedule (0 when none).
template <typename K>
static int cluster_width(int64_t n, K kern) {
  static int cached[64][2] = {};
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t budget = (size_t)max_smem_optin() - 1024;
  for (int C : {16, 8, 4, 2}) {
    const size_t smem = (size_t)((n + C - 1) / C) * sizeof(double);
    if (smem > budget) continue;
    {
      std::lock_guard<std::mutex> lk(mu);
      // schedulable widths do not depend on n beyond the shared memory size
      if (dev < 64 && cached[dev][0] == C && (size_t)cached[dev][1] >= smem) return C;
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kCtaThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 1) {
      std::lock_guard<std::mutex> lk(mu);
      if (dev < 64) {
        cached[dev][0] = C;
        cached[dev][1] = (int)smem;
      }
      return C;
    }
    cudaGetLastError();
  }
  return 0;
}

int cluster_size_for(int64_t n) { return cluster_width(n, k_sweep_cluster<true, false, 4>); }

template <typename K, typename... Args>
static cudaError_t launch_on_cluster(K kern, int C, int threads, size_t smem, cudaStream_t s,
                                     Args... args) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, args...);
  note_launch();
  return e;
}

// The helped sweep: two clusters (width from the kernel), launched
// cooperatively, so every CTA is resident at once or the launch fails: the
// helper CTAs wait on the sweep's.
template <typename K, typename... Args>
static cudaError_t launch_help(K kern, int threads, size_t smem, cudaStream_t s, Args... args) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * kHelpCluster));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, args...);
  note_launch();
  return e;
}

// Slots beyond the row warps' own span at which a prefix helper starts a row
// (it waits until the row `lag` slots earlier is final): late enough that
// most of the row's leading entries are final, early enough to publish before
// the row's warp takes the row.  Measured on the random band matrix with
// n = 160,000, k = 2: forward best at 384-512, backward at 256.
constexpr int64_t kHelpLagFwd = 448;
constexpr int64_t kHelpLagBwd = 256;

template <bool FORWARD, bool DIVIDE>
static cudaError_t run_sweep(int64_t n, const LevelOrder &lo, const int64_t *rp, const int32_t *ci,
                             const int64_t *dg, const double *v, const DivPrep *rd,
                             const double *in, double *out, double *clear, int sched, DevErr *err,
                             const SweepAux *aux, cudaStream_t s) {
  ProfScope prof_scope(FORWARD ? ILUK_PROF_SWEEP : ILUK_PROF_SWEEP_BWD, s);
  // an empty order: nothing to sweep (n = 0, or a direction the caller skips)
  if (n == 0 || (!lo.order && !lo.corder)) return cudaSuccess;
  // the helped kind needs its scratch; without it, the plain cluster kind
  if ((sched & 0xf) == ILUK_SCHED_WARP_CLUSTER_HELP && (!aux || !aux->pre_s || aux->n < n))
    sched = (sched & ~0xf) | ILUK_SCHED_WARP_CLUSTER;
  const bool helped = (sched & 0xf) == ILUK_SCHED_WARP_CLUSTER_HELP;
  if (helped) sched = (sched & ~0xf) | ILUK_SCHED_WARP_CLUSTER;
  // the lockstep kinds walk the padded level order; an index order (a
  // factorization that has not built its level orders) has only the plain one
  const int kind0 = sched & 0xf;
  const bool padded = kind0 != ILUK_SCHED_WARP_GRID && kind0 != ILUK_SCHED_WARP_CLUSTER;
  if (padded && !lo.order) return cudaErrorInvalidValue;
  if (!padded && !lo.corder) return cudaErrorInvalidValue;
  int64_t limit = wait_limit();
  const int32_t *order = lo.order;
  int64_t len = lo.len;
  const int w = (sched >> 4) & 0xf;  // CTA width / 128 of the warp-per-row kinds
  const int threads = w ? w * 128 : kCtaThreads;
  sched &= 0xf;
  if (sched == ILUK_SCHED_SINGLE_CTA) {
    k_sweep<FORWARD, DIVIDE, false, 4><<<1, kCtaThreads, 0, s>>>(order, len, rp, ci, dg, v, rd,
                                                                in, out, clear, err, limit);
    note_launch();
    return cudaGetLastError();
  }
  if (sched == ILUK_SCHED_WARP_GRID || sched == ILUK_SCHED_WARP_CLUSTER) {
    // one warp per row needs no warp-aligned levels: the unpadded order keeps
    // every warp's next row further ahead and wastes no slot loads
    order = lo.corder;
    len = lo.clen;
  }
  if (sched == ILUK_SCHED_CLUSTER || sched == ILUK_SCHED_WARP_CLUSTER) {
    const bool wpr = sched == ILUK_SCHED_WARP_CLUSTER;
    const int C = wpr ? cluster_width(n, k_sweep_wpr<FORWARD, DIVIDE, 1>)
                      : cluster_width(n, k_sweep_cluster<FORWARD, DIVIDE, 4>);
    if (C == 0) return cudaErrorInvalidConfiguration;
    if (wpr) {
      const int wpc = threads / 32;
      const int64_t nwc = (int64_t)C * wpc;
      const size_t wsmem = (size_t)((len + nwc - 1) / nwc * wpc) * sizeof(double);
      if (wsmem > (size_t)max_smem_optin()) return cudaErrorInvalidConfiguration;
      const int32_t *owner = owner_codes(lo, n, C, threads, s);
      if (!owner) return cudaErrorMemoryAllocation;
      double *no_ps = nullptr;
      unsigned long long *no_pk = nullptr;
      unsigned *no_words = nullptr;
      if (helped && C == kHelpCluster) {  // a second cluster of prefix helpers
        const int64_t lag = (FORWARD ? kHelpLagFwd : kHelpLagBwd) + nwc;
        const cudaError_t e =
            launch_help(k_sweep_wpr_help<FORWARD, DIVIDE>, threads, wsmem, s, order, len, n, rp,
                        ci, dg, v, rd, in, out, clear, err, limit, owner, aux->pre_s, aux->pre_k,
                        aux->words, lag, C, 2 * C);
        if (e == cudaSuccess) return e;
        cudaGetLastError();  // cannot hold both clusters at once: the plain kind
      }
      return launch_on_cluster(k_sweep_wpr<FORWARD, DIVIDE, 1>, C, threads, wsmem, s, order, len,
                               n, rp, ci, dg, v, rd, in, out, clear, err, limit, owner, no_ps,
                               no_pk, no_words, (int64_t)0, C, C);
    }
    const size_t smem = (size_t)((n + C - 1) / C) * sizeof(double);
    return launch_on_cluster(k_sweep_cluster<FORWARD, DIVIDE, 4>, C, kCtaThreads, smem, s, order,
                             len, n, rp, ci, dg, v, rd, in, out, clear, err, limit, C);
  }
  if (sched == ILUK_SCHED_WARP_GRID) {
    auto kern = k_sweep_wpr<FORWARD, DIVIDE, 0>;
    int bps = 1;  // an explicit width means one CTA of that width per SM
    if (w == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kCtaThreads, 0);
    if (bps < 1) bps = 1;
    int64_t grid = (int64_t)bps * num_sms();
    const int64_t want = (len + (threads / 32) - 1) / (threads / 32);
    if (grid > want) grid = want;
    const int64_t nn = n;
    const int32_t *no_owner = nullptr;
    double *no_ps = nullptr;
    unsigned long long *no_pk = nullptr;
    unsigned *no_words = nullptr;
    int64_t no_lag = 0;
    int no_c = 0;
    void *args[] = {(void *)&order, (void *)&len, (void *)&nn, (void *)&rp, (void *)&ci,
                    (void *)&dg, (void *)&v, (void *)&rd, (void *)&in, (void *)&out,
                    (void *)&clear, (void *)&err, (void *)&limit, (void *)&no_owner,
                    (void *)&no_ps, (void *)&no_pk, (void *)&no_words, (void *)&no_lag,
                    (void *)&no_c, (void *)&no_c};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)grid),
                                                dim3((unsigned)threads), args, 0, s);
    note_launch();
    return e;
  }
  // Multi-SM: every block must be resident (rows wait on rows of other
  // blocks), so the grid is launched cooperatively and sized by occupancy.
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_sweep<FORWARD, DIVIDE, true, 8>,
                                                kGridThreads, 0);
  if (bps > 2) bps = 2;
  if (bps < 1) bps = 1;
  int64_t grid = (int64_t)bps * num_sms();
  const int64_t want = (len + kGridThreads - 1) / kGridThreads;  // one warp per 32 slots
  if (grid > want) grid = want;
  void *args[] = {(void *)&order, (void *)&len, (void *)&rp, (void *)&ci, (void *)&dg,
                  (void *)&v, (void *)&rd, (void *)&in, (void *)&out, (void *)&clear,
                  (void *)&err, (void *)&limit};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_sweep<FORWARD, DIVIDE, true, 8>,
                                              dim3((unsigned)grid), dim3(kGridThreads), args, 0, s);
  note_launch();
  return e;
}

// One schedule byte made usable for n rows: an unknown kind becomes the
// warp-per-row grid, a cluster kind without a usable cluster likewise, and a
// width only stays with the warp-per-row kinds (256..1024 threads).
static int usable_sched(int64_t n, int sc) {
  int kind = sc & 0xf, w = (sc >> 4) & 0xf;
  if (kind < ILUK_SCHED_FLAGS || kind > ILUK_SCHED_WARP_CLUSTER_HELP) kind = ILUK_SCHED_WARP_GRID;
  const bool clustered = kind == ILUK_SCHED_CLUSTER || kind == ILUK_SCHED_WARP_CLUSTER ||
                         kind == ILUK_SCHED_WARP_CLUSTER_HELP;
  if (clustered && cluster_size_for(n) == 0) kind = ILUK_SCHED_WARP_GRID;
  const bool per_row = kind == ILUK_SCHED_WARP_GRID || kind == ILUK_SCHED_WARP_CLUSTER ||
                       kind == ILUK_SCHED_WARP_CLUSTER_HELP;
  if (!per_row || w < 2 || w > 8) w = 0;
  return kind | (w << 4);
}

cudaError_t launch_apply_backward(int64_t n, const int64_t *rp, const int32_t *ci,
                                  const int64_t *dg, const double *v, const DivPrep *rd,
                                  const LevelOrder &bwd, double *tmp, double *y, int sched,
                                  DevErr *err, const SweepAux *aux, cudaStream_t s) {
  // tmp already holds L^-1 p; y is armed here as the forward sweep would
  // have armed it, and the backward sweep re-arms tmp as usual
  int sb = (sched >> 8) & 0xff;
  if (sb == 0) sb = sched & 0xff;
  cudaError_t e = launch_fill_pending(n, y, s);
  if (e != cudaSuccess) return e;
  return run_sweep<false, true>(n, bwd, rp, ci, dg, v, rd, tmp, y, tmp, usable_sched(n, sb), err,
                                aux, s);
}

cudaError_t launch_apply(int64_t n, const int64_t *rp, const int32_t *ci, const int64_t *dg,
                         const double *v, const DivPrep *rd, const LevelOrder &fwd,
                         const LevelOrder &bwd,
                         const double *p, double *tmp, double *y, int transpose, int sched,
                         DevErr *err, const SweepAux *aux, cudaStream_t s) {
  // sched packs the forward schedule in bits 0-7 and the backward one in 8-15
  // (a single value applies to both).
  int sf = sched & 0xff, sb = (sched >> 8) & 0xff;
  if (sb == 0) sb = sf;
  sf = usable_sched(n, sf);
  sb = usable_sched(n, sb);
  cudaError_t e;
  // tmp is pending on entry (left so by the previous backward sweep); the
  // forward sweep re-arms y, the backward sweep re-arms tmp.
  if (!transpose) {
    e = run_sweep<true, false>(n, fwd, rp, ci, dg, v, rd, p, tmp, y, sf, err, aux, s);
    if (e != cudaSuccess) return e;
    return run_sweep<false, true>(n, bwd, rp, ci, dg, v, rd, tmp, y, tmp, sb, err, aux, s);
  }
  e = run_sweep<true, true>(n, fwd, rp, ci, dg, v, rd, p, tmp, y, sf, err, aux, s);
  if (e != cudaSuccess) return e;
  return run_sweep<false, false>(n, bwd, rp, ci, dg, v, rd, tmp, y, tmp, sb, err, aux, s);
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
  ProfScope prof_scope(ILUK_PROF_TRANSPOSE, s);
  if (n == 0) return cudaMemsetAsync(trp, 0, sizeof(int64_t), s);
  int64_t g = (int64_t)num_sms() * 8;
  cudaError_t e = cudaMemsetAsync(cursor, 0, (size_t)n * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  k_count_cols<<<(unsigned)g, 256, 0, s>>>(nnz, ci, cursor);
  note_launch();
  e = launch_scan_lengths(n, cursor, trp, scan_tmp, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(cursor, 0, (size_t)n * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  k_scatter_t<<<(unsigned)g, 256, 0, s>>>(n, rp, ci, v, trp, cursor, tci, tv);
  note_launch();
  k_sort_rows_t<<<(unsigned)g, 256, 0, s>>>(n, trp, tci, tv, tdiag);
  note_launch();
  return cudaGetLastError();
}

}  // namespace iluk
