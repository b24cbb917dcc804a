// batched.cu -- a7: many systems, numerically factored and solved in one
// persistent launch.
//
// Each CTA of a persistent grid takes the next instance (an atomic ticket) and
// runs its whole pipeline alone: ILU(k) numeric factorization, then
// right-preconditioned GMRES(m) with the ILU sweeps, exactly the algorithm of
// the single-instance path.  Inside a CTA there is no waiting on flags: the
// factorization and both sweeps walk the instance's level sets (built by the
// symbolic phase) with a __syncthreads between levels, and the warps walk the
// rows of a level with converged FP64 instructions.  Inner products follow the
// same 4096-partial fixed tree as the single-instance path, so every instance
// is bit-identical to solving it on its own.  Instances may have different
// patterns and sizes (uneven grids); those sharing one symbolic handle share
// its pattern arrays.  The work is enqueued asynchronously with no host
// round trip, so a stream capture records it as a graph.
#include "internal.h"

namespace iluk {

constexpr int kBMaxRestart = 64;

struct BatchItemDev {
  int64_t n, nnzA, nnzF;
  const int64_t *arp;
  const int32_t *aci;
  const double *aval;
  const int64_t *frp;
  const int32_t *fci;
  const int64_t *fdiag;
  const int64_t *farp;  // A row pointers as stored by the symbolic phase
  const int32_t *a2f;
  const int32_t *lord;
  const int64_t *lstart;
  int32_t nlev_l;
  const int32_t *uord;
  const int64_t *ustart;
  int32_t nlev_u;
  const double *b;
  double *x;
};

struct BatchResultDev {
  int32_t status, iters, cycles, pad;
  int64_t row;
  double relres;
};

struct BatchWork {
  // z: the m preconditioned basis vectors of a cycle; u: the reciprocals of
  // the diagonal the numeric phase publishes (div_prep, one 64-bit word a row)
  double *fval, *V, *w, *z, *u, *tmp;
  int64_t ldv;  // stride between basis vectors
};

// --- in-CTA building blocks -------------------------------------------------

// Fixed-shape inner product (same shape as k_dot): partial p sums i = p,
// p + 4096, ... from +0.0; pairwise tree.  If `upd` is set, first applies
// w_i <- w_i - h * v_i to the indices the partial owns.  Result broadcast.
// A thread owns kDotP / NT partials and advances four of them side by side,
// one element each per round: all loads of a round are issued before its
// arithmetic and stores (a store to w could otherwise alias the next
// partial's loads and serialise them), and the four chains are independent.
// Each partial still sums its own elements in order.
template <int NT>
__device__ double cta_dot(int64_t n, double *w, const double *v, double h, bool upd,
                          const double *y, double *sh, bool take_sqrt) {
  constexpr int kPer = kDotP / NT;
  constexpr int kG = kPer < 4 ? kPer : 4;
  static_assert(kPer % kG == 0, "partials per thread");
  for (int k0 = 0; k0 < kPer; k0 += kG) {
    double s[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) s[g] = 0.0;
    for (int64_t i0 = threadIdx.x + (int64_t)k0 * NT; i0 < n; i0 += kDotP) {
      double wv[kG], vv[kG], yv[kG];
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        const int64_t i = i0 + (int64_t)g * NT;
        wv[g] = vv[g] = yv[g] = 0.0;
        if (i < n) {
          wv[g] = w[i];
          if (upd) vv[g] = v[i];
          if (y != nullptr) yv[g] = y[i];
        }
      }
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        const int64_t i = i0 + (int64_t)g * NT;
        if (i < n) {
          double wi = wv[g];
          if (upd) {
            wi = __dsub_rn(wi, __dmul_rn(h, vv[g]));
            w[i] = wi;
          }
          s[g] = __dadd_rn(s[g], __dmul_rn(wi, y == nullptr ? wi : yv[g]));
        }
      }
    }
#pragma unroll
    for (int g = 0; g < kG; ++g) sh[threadIdx.x + (k0 + g) * NT] = s[g];
  }
  __syncthreads();
  for (int wdt = kDotP / 2; wdt >= 1; wdt >>= 1) {
    for (int p = threadIdx.x; p < wdt; p += NT) sh[p] = __dadd_rn(sh[p], sh[p + wdt]);
    __syncthreads();
  }
  const double r = take_sqrt ? __dsqrt_rn(sh[0]) : sh[0];
  __syncthreads();
  return r;
}

// y = A x (bm == nullptr) or y = bm - A x; rows summed left to right from 0.
template <int NT>
__device__ void cta_spmv(const BatchItemDev &it, const double *x, double *y, const double *bm) {
  for (int64_t row = threadIdx.x; row < it.n; row += NT) {
    double s = 0.0;
    for (int64_t p = it.arp[row]; p < it.arp[row + 1]; ++p)
      s = __dadd_rn(s, __dmul_rn(it.aval[p], x[it.aci[p]]));
    y[row] = bm ? __dsub_rn(bm[row], s) : s;
  }
  __syncthreads();
}

// One sweep, level by level; the 32 rows a warp takes from a level run their
// chains in lockstep, forward left to right, backward right to left, each row
// exactly in the order of the single-instance kernels.  Nothing a row's chain
// reads from F depends on the level before, so a warp loads its next level's
// rows (position, right-hand side, the first kSweepPf coefficients and their
// columns) before the barrier that ends the current level; after it, only the
// gather of the values just computed is left.  The backward division uses the
// reciprocal of u_ii published by the numeric phase (rdx).
constexpr int kSweepPf = 4;

struct SweepChunk {
  int64_t first;      // position of the chain's first coefficient
  int32_t row, len;   // row (-1: padding) and chain length
  double s;           // right-hand side entry
  double cv[kSweepPf];
  int32_t ci[kSweepPf];
};

// `active` false (no chunk for this warp): an empty chunk, every field set,
// so that nothing of an earlier chunk stays live.
template <bool FORWARD>
__device__ __forceinline__ void sweep_chunk_load(const BatchItemDev &it, const double *fv,
                                                 const int32_t *order, int64_t slot, bool active,
                                                 const double *in, SweepChunk &c) {
  c.row = active ? order[slot] : -1;
  c.len = 0;
  c.first = 0;
  c.s = 0.0;
  if (c.row >= 0) {
    const int64_t d = it.fdiag[c.row];
    if (FORWARD) {
      c.first = it.frp[c.row];
      c.len = (int)(d - c.first);
    } else {
      c.first = it.frp[c.row + 1] - 1;
      c.len = (int)(c.first - d);
    }
    c.s = in[c.row];
  }
#pragma unroll
  for (int q = 0; q < kSweepPf; ++q) {
    c.cv[q] = 0.0;
    c.ci[q] = 0;
    if (q < c.len) {
      const int64_t pq = FORWARD ? c.first + q : c.first - q;
      c.cv[q] = fv[pq];
      c.ci[q] = it.fci[pq];
    }
  }
}

template <bool FORWARD>
__device__ __forceinline__ void sweep_chunk_run(const BatchItemDev &it, const double *fv,
                                                const unsigned long long *rdx,
                                                const SweepChunk &c, double *out) {
  const int maxlen = __reduce_max_sync(FULL_MASK, c.len);
  double xv[kSweepPf];
#pragma unroll
  for (int q = 0; q < kSweepPf; ++q)
    if (q < c.len) xv[q] = out[c.ci[q]];
  double sacc = c.s;
#pragma unroll
  for (int q = 0; q < kSweepPf; ++q)
    if (q < c.len) sacc = __dsub_rn(sacc, __dmul_rn(c.cv[q], xv[q]));
  for (int q = kSweepPf; q < maxlen; ++q) {
    if (q < c.len) {
      const int64_t pq = FORWARD ? c.first + q : c.first - q;
      sacc = __dsub_rn(sacc, __dmul_rn(fv[pq], out[it.fci[pq]]));
    }
  }
  if (c.row >= 0) {
    if (FORWARD) {
      out[c.row] = sacc;
    } else {
      const int64_t d = c.first - c.len;
      out[c.row] = div_fin(sacc, DivPrep{rdx[c.row], fv[d]});
    }
  }
}

template <int NT, bool FORWARD>
__device__ void cta_sweep(const BatchItemDev &it, const double *fv, const unsigned long long *rdx,
                          const double *in, double *out) {
  const int32_t *order = FORWARD ? it.lord : it.uord;
  const int64_t *start = FORWARD ? it.lstart : it.ustart;
  const int nlev = FORWARD ? it.nlev_l : it.nlev_u;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  SweepChunk nx;
  int64_t lbeg = nlev > 0 ? start[0] : 0;
  int64_t lend = nlev > 0 ? start[1] : 0;
  sweep_chunk_load<FORWARD>(it, fv, order, lbeg + wid * 32 + lane, lbeg + wid * 32 < lend, in,
                            nx);
  for (int l = 0; l < nlev; ++l) {
    const int64_t nend = l + 1 < nlev ? start[l + 2] : 0;
    if (lbeg + wid * 32 < lend) sweep_chunk_run<FORWARD>(it, fv, rdx, nx, out);
    for (int64_t s0 = lbeg + (int64_t)wid * 32 + NT; s0 < lend; s0 += NT) {  // wide levels
      SweepChunk c;
      sweep_chunk_load<FORWARD>(it, fv, order, s0 + lane, true, in, c);
      sweep_chunk_run<FORWARD>(it, fv, rdx, c, out);
    }
    // the next level's first chunk of this warp, before the barrier
    sweep_chunk_load<FORWARD>(it, fv, order, lend + wid * 32 + lane, lend + wid * 32 < nend, in,
                              nx);
    lbeg = lend;
    lend = nend;
    __syncthreads();
  }
}

// The same sweep without level barriers: the output starts as a pending
// marker (a signalling-NaN pattern no arithmetic produces) and each warp,
// taking its 32 rows from the level order, polls the values its lanes need
// with CTA-scope loads, so a row starts as soon as its own inputs are final.
// Each chain keeps the level form's order, so the results are identical.
// Bounded: false when a wait runs out.
constexpr unsigned long long kSpinPending = 0x7FF0DEADBEEFCAFEull;

__device__ __forceinline__ double ld_cta_f64(const double *p) {
  double v;
  asm volatile("ld.relaxed.cta.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ void st_cta_f64(double *p, double v) {
  asm volatile("st.relaxed.cta.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ bool spin_pending(double v) {
  return (unsigned long long)__double_as_longlong(v) == kSpinPending;
}

// A warp's chunk of the spinning sweep: position of its rows' chains and
// right-hand sides, loaded while the chunk before waits for its inputs.
struct SpinMeta {
  int64_t first;     // position of the chain's first coefficient
  int32_t row, len;  // row (-1: padding) and chain length
  double s;          // right-hand side entry
};

template <bool FORWARD>
__device__ __forceinline__ void spin_meta_load(const BatchItemDev &it, const int32_t *order,
                                               int64_t slot, bool active, const double *in,
                                               SpinMeta &m) {
  m.row = active ? order[slot] : -1;
  m.len = 0;
  m.first = 0;
  m.s = 0.0;
  if (m.row >= 0) {
    const int64_t d = it.fdiag[m.row];
    if (FORWARD) {
      m.first = it.frp[m.row];
      m.len = (int)(d - m.first);
    } else {
      m.first = it.frp[m.row + 1] - 1;
      m.len = (int)(m.first - d);
    }
    m.s = in[m.row];
  }
}

// Per chunk: the first kSpinPf coefficients, their columns and (backward)
// the divisor are loaded at once, and so are the next chunk's rows; then the
// inputs are gathered together and only those still pending are polled
// again.  Longer chains finish one coefficient at a time.
constexpr int kSpinPf = 6;

template <int NT, bool FORWARD>
__device__ bool cta_sweep_spin(const BatchItemDev &it, const double *fv,
                               const unsigned long long *rdx, const double *in, double *out,
                               int64_t limit_ns) {
  const int32_t *order = FORWARD ? it.lord : it.uord;
  const int64_t len = FORWARD ? it.lstart[it.nlev_l] : it.ustart[it.nlev_u];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = 0;
  for (int64_t i = threadIdx.x; i < it.n; i += NT)
    out[i] = __longlong_as_double((long long)kSpinPending);
  __syncthreads();
  bool ok = true;
  SpinMeta cur;
  spin_meta_load<FORWARD>(it, order, (int64_t)wid * 32 + lane, (int64_t)wid * 32 < len, in, cur);
  for (int64_t s0 = (int64_t)wid * 32; s0 < len; s0 += NT) {
    double cv[kSpinPf];
    int32_t ci[kSpinPf];
#pragma unroll
    for (int q = 0; q < kSpinPf; ++q) {
      cv[q] = 0.0;
      ci[q] = 0;
      if (q < cur.len) {
        const int64_t pq = FORWARD ? cur.first + q : cur.first - q;
        cv[q] = fv[pq];
        ci[q] = it.fci[pq];
      }
    }
    unsigned long long rx = 0;
    double diag = 0.0;
    if (!FORWARD && cur.row >= 0) {
      rx = rdx[cur.row];
      diag = fv[cur.first - cur.len];
    }
    SpinMeta nxt;
    spin_meta_load<FORWARD>(it, order, s0 + NT + lane, s0 + NT < len, in, nxt);
    double xv[kSpinPf];
    unsigned pend = 0;
#pragma unroll
    for (int q = 0; q < kSpinPf; ++q) {
      xv[q] = 0.0;
      if (q < cur.len) {
        xv[q] = ld_cta_f64(&out[ci[q]]);
        if (spin_pending(xv[q])) pend |= 1u << q;
      }
    }
    if (__any_sync(FULL_MASK, pend != 0)) {
      const uint64_t t0 = globaltimer_ns();
      for (unsigned k = 0; __any_sync(FULL_MASK, pend != 0); ++k) {
#pragma unroll
        for (int q = 0; q < kSpinPf; ++q) {
          if ((pend >> q) & 1u) {
            xv[q] = ld_cta_f64(&out[ci[q]]);
            if (!spin_pending(xv[q])) pend &= ~(1u << q);
          }
        }
        const bool stop = (k & 31u) == 31u &&
                          (*((volatile int *)&s_fail) ||
                           (int64_t)(globaltimer_ns() - t0) > limit_ns);
        if (__any_sync(FULL_MASK, stop)) {  // the whole warp gives up together
          ok = false;
          break;
        }
      }
    }
    if (!ok) break;
    double sacc = cur.s;
#pragma unroll
    for (int q = 0; q < kSpinPf; ++q)
      if (q < cur.len) sacc = __dsub_rn(sacc, __dmul_rn(cv[q], xv[q]));
    const int maxlen = __reduce_max_sync(FULL_MASK, cur.len);
    for (int q = kSpinPf; q < maxlen; ++q) {
      const bool act = q < cur.len;
      int64_t pq = 0;
      double x = 0.0;
      if (act) {
        pq = FORWARD ? cur.first + q : cur.first - q;
        x = ld_cta_f64(&out[it.fci[pq]]);
      }
      bool pq_pend = act && spin_pending(x);
      if (__any_sync(FULL_MASK, pq_pend)) {
        const uint64_t t0 = globaltimer_ns();
        for (unsigned k = 0; __any_sync(FULL_MASK, pq_pend); ++k) {
          if (pq_pend) {
            x = ld_cta_f64(&out[it.fci[pq]]);
            pq_pend = spin_pending(x);
          }
          const bool stop = (k & 31u) == 31u &&
                            (*((volatile int *)&s_fail) ||
                             (int64_t)(globaltimer_ns() - t0) > limit_ns);
          if (__any_sync(FULL_MASK, stop)) {
            ok = false;
            break;
          }
        }
        if (!ok) break;
      }
      if (act) sacc = __dsub_rn(sacc, __dmul_rn(fv[pq], x));
    }
    if (!ok) break;
    if (cur.row >= 0) {
      double y = FORWARD ? sacc : div_fin(sacc, DivPrep{rx, diag});
      if ((unsigned long long)__double_as_longlong(y) == kSpinPending)
        y = __longlong_as_double(0x7FF8000000000000ll);  // never the marker
      st_cta_f64(&out[cur.row], y);
    }
    cur = nxt;
  }
  if (!ok && lane == 0) atomicExch(&s_fail, 1);
  __syncthreads();
  return s_fail == 0;
}

// Numeric factorization, level by level over the forward level sets; one
// warp per row, the row in the warp's shared slice, pivots ascending (the IKJ
// order of Eq. lufactor2).  Under the level schedule every pivot row of a
// row is final before the row starts, so the warp first stages all of them at
// once: for each pivot h its diagonal f_hh and the reciprocal published when
// row h finished (rdx[h], see div_prep), and for each entry f_hj, j > h, its
// value and the position of column j in row i (-1 when (i, j) is not in the
// pattern).  The loads of all pivots overlap, and the pivot loop is left with
// the multiplier (div_fin) and the row's updates, all from shared memory.
// Rows with more pivots or pivot entries than a warp's staging area holds
// load each pivot row in turn.  A finished row publishes the reciprocal of
// its diagonal for the rows and backward sweeps after it.  The staging areas
// take the inner-product partials' shared memory, idle during this phase.
template <int NT>
struct WarpStage {
  static constexpr int kBytes = 8 * kDotP / (NT / 32);    // one warp's share of the partials
  static constexpr int kPiv = kBytes >= 2048 ? 32 : 16;   // pivots staged
  static constexpr int kPairs = (kBytes - 24 * kPiv - 4 * (kPiv + 1)) / 12;  // pivot entries
  static_assert(8 * kPairs + 24 * kPiv + 4 * kPairs + 4 * (kPiv + 1) <= kBytes, "stage size");
  double *v;                // f_hj of the staged entries
  unsigned long long *x;    // rdx[h]
  double *piv;              // f_hh
  int64_t *hd;              // position of f_hh
  int32_t *pos;             // position of column j in the row, or -1
  int32_t *off;             // first staged entry of each pivot, then the total
  __device__ explicit WarpStage(double *base)
      : v(base),
        x(reinterpret_cast<unsigned long long *>(base + kPairs)),
        piv(reinterpret_cast<double *>(x + kPiv)),
        hd(reinterpret_cast<int64_t *>(piv + kPiv)),
        pos(reinterpret_cast<int32_t *>(hd + kPiv)),
        off(pos + kPairs) {}
};

__device__ __forceinline__ void numeric_report(int *s_bad, long long *s_badrow, int code,
                                               int64_t row) {
  atomicCAS(s_bad, 0, code);
  atomicMin(s_badrow, (long long)row);
}

// One row by the whole warp.
template <int NT>
__device__ __forceinline__ void numeric_row_warp(const BatchItemDev &it, double *fv,
                                                 unsigned long long *rdx, double *rv, int32_t *rc,
                                                 const WarpStage<NT> &st, int64_t row, int lane,
                                                 int *s_bad, long long *s_badrow) {
  constexpr int kStagePiv = WarpStage<NT>::kPiv, kStagePairs = WarpStage<NT>::kPairs;
  const int64_t b0 = it.frp[row];
  const int m = (int)(it.frp[row + 1] - b0);
  const int dp = (int)(it.fdiag[row] - b0);
  for (int q = lane; q < m; q += 32) {
    rc[q] = it.fci[b0 + q];
    rv[q] = 0.0;
  }
  __syncwarp();
  bool bad = false;
  for (int64_t p = it.farp[row] + lane; p < it.farp[row + 1]; p += 32) {
    const double a = it.aval[p];
    if (!isfinite(a)) bad = true;
    rv[it.a2f[p]] = a;
  }
  if (__any_sync(FULL_MASK, bad) && lane == 0) numeric_report(s_bad, s_badrow, ILUK_ENONFINITE, row);
  // stage the pivots: lane q takes pivot q
  int len = 0;
  if (dp <= kStagePiv && lane < dp) {
    const int h = rc[lane];
    const int64_t hd = it.fdiag[h];
    len = (int)(it.frp[h + 1] - hd - 1);
    st.hd[lane] = hd;
    st.x[lane] = rdx[h];
    st.piv[lane] = fv[hd];
  }
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(FULL_MASK, incl, o);
    if (lane >= o) incl += t;
  }
  const int total = __shfl_sync(FULL_MASK, incl, 31);
  if (dp <= kStagePiv && total <= kStagePairs) {
    if (lane < dp) st.off[lane] = incl - len;
    if (lane == 0) st.off[dp] = total;
    __syncwarp();
    for (int t = lane; t < total; t += 32) {
      int q = 0;  // the pivot of entry t: the last q with off[q] <= t
      for (int lo = 0, hi = dp; lo < hi;) {
        const int mid = (lo + hi) >> 1;
        if (st.off[mid] <= t) { q = mid; lo = mid + 1; } else { hi = mid; }
      }
      const int64_t r = st.hd[q] + 1 + (t - st.off[q]);
      const int32_t j = it.fci[r];
      st.v[t] = fv[r];
      const int pos = lower_bound_i(rc, q + 1, m, j);
      st.pos[t] = (pos < m && rc[pos] == j) ? pos : -1;
    }
    __syncwarp();
    for (int q = 0; q < dp; ++q) {
      const double fih = div_fin(rv[q], DivPrep{st.x[q], st.piv[q]});
      for (int t = st.off[q] + lane; t < st.off[q + 1]; t += 32) {
        const int pos = st.pos[t];
        if (pos >= 0) rv[pos] = sub_prod(rv[pos], fih, st.v[t]);
      }
      __syncwarp();  // every lane has read rv[q] and applied this pivot
      if (lane == 0) rv[q] = fih;
    }
  } else {
    for (int q = 0; q < dp; ++q) {
      const int h = rc[q];
      const int64_t hd = it.fdiag[h];
      const double fih = div_fin(rv[q], DivPrep{rdx[h], fv[hd]});
      __syncwarp();
      if (lane == 0) rv[q] = fih;
      __syncwarp();
      for (int64_t r = hd + 1 + lane; r < it.frp[h + 1]; r += 32) {
        const int32_t j = it.fci[r];
        const int pos = lower_bound_i(rc, q + 1, m, j);
        if (pos < m && rc[pos] == j) rv[pos] = sub_prod(rv[pos], fih, fv[r]);
      }
      __syncwarp();
    }
  }
  __syncwarp();
  for (int q = lane; q < m; q += 32) fv[b0 + q] = rv[q];
  if (lane == 0) {
    const double d = rv[dp];
    rdx[row] = div_prep(d).x;
    if (d == 0.0) numeric_report(s_bad, s_badrow, ILUK_EZEROPIVOT, row);
  }
  __syncwarp();
}

// Two rows of a level side by side, one per half-warp (lanes 0-15 take rowA,
// 16-31 rowB; -1: none), each with half of the warp's row slice and staging
// area: the two rows' load and division latencies overlap, and one FP64
// instruction applies both rows' updates.  Each row keeps the whole-warp
// path's order of operations.  Returns false, having changed nothing the
// whole-warp path relies on, when a row has more than 16 entries or does not
// fit half a staging area.
template <int NT>
__device__ __forceinline__ bool numeric_rows_half(const BatchItemDev &it, double *fv,
                                                  unsigned long long *rdx, double *rv_w,
                                                  int32_t *rc_w, const WarpStage<NT> &st,
                                                  int64_t rowA, int64_t rowB, int lane,
                                                  int *s_bad, long long *s_badrow) {
  constexpr int kHalfPiv = WarpStage<NT>::kPiv / 2;     // staged pivots per half, plus one offset
  constexpr int kHalfPairs = WarpStage<NT>::kPairs / 2;  // staged entries per half
  const int half = lane >> 4, hl = lane & 15;
  const int64_t row = half ? rowB : rowA;
  int64_t b0 = 0;
  int m = 0, dp = 0;
  if (row >= 0) {
    b0 = it.frp[row];
    m = (int)(it.frp[row + 1] - b0);
    dp = (int)(it.fdiag[row] - b0);
  }
  if (!__all_sync(FULL_MASK, m <= 16 && dp < kHalfPiv)) return false;
  double *rv = rv_w + half * 16;
  int32_t *rc = rc_w + half * 16;
  double *sv = st.v + half * kHalfPairs;
  int32_t *spos = st.pos + half * kHalfPairs;
  unsigned long long *sx = st.x + half * kHalfPiv;
  double *spiv = st.piv + half * kHalfPiv;
  int64_t *shd = st.hd + half * kHalfPiv;
  int32_t *soff = st.off + half * kHalfPiv;
  if (hl < m) {
    rc[hl] = it.fci[b0 + hl];
    rv[hl] = 0.0;
  }
  __syncwarp();
  bool bad = false;
  if (row >= 0) {
    for (int64_t p = it.farp[row] + hl; p < it.farp[row + 1]; p += 16) {
      const double a = it.aval[p];
      if (!isfinite(a)) bad = true;
      rv[it.a2f[p]] = a;
    }
  }
  const unsigned badm = __ballot_sync(FULL_MASK, bad);
  if (hl == 0 && ((badm >> (16 * half)) & 0xffffu))
    numeric_report(s_bad, s_badrow, ILUK_ENONFINITE, row);
  int len = 0;
  if (hl < dp) {
    const int h = rc[hl];
    const int64_t hd = it.fdiag[h];
    len = (int)(it.frp[h + 1] - hd - 1);
    shd[hl] = hd;
    sx[hl] = rdx[h];
    spiv[hl] = fv[hd];
  }
  int incl = len;
#pragma unroll
  for (int o = 1; o < 16; o <<= 1) {
    const int t = __shfl_up_sync(FULL_MASK, incl, o, 16);
    if (hl >= o) incl += t;
  }
  const int total = __shfl_sync(FULL_MASK, incl, 15, 16);
  if (!__all_sync(FULL_MASK, total <= kHalfPairs)) {
    __syncwarp();
    return false;
  }
  if (hl < dp) soff[hl] = incl - len;
  if (hl == 0) soff[dp] = total;
  __syncwarp();
  for (int t = hl; t < total; t += 16) {
    int q = 0;  // the pivot of entry t: the last q with off[q] <= t
    for (int lo = 0, hi = dp; lo < hi;) {
      const int mid = (lo + hi) >> 1;
      if (soff[mid] <= t) { q = mid; lo = mid + 1; } else { hi = mid; }
    }
    const int64_t r = shd[q] + 1 + (t - soff[q]);
    const int32_t j = it.fci[r];
    sv[t] = fv[r];
    const int pos = lower_bound_i(rc, q + 1, m, j);
    spos[t] = (pos < m && rc[pos] == j) ? pos : -1;
  }
  __syncwarp();
  const int dmax = __reduce_max_sync(FULL_MASK, dp);
  for (int q = 0; q < dmax; ++q) {
    double fih = 0.0;
    if (q < dp) {
      fih = div_fin(rv[q], DivPrep{sx[q], spiv[q]});
      for (int t = soff[q] + hl; t < soff[q + 1]; t += 16) {
        const int pos = spos[t];
        if (pos >= 0) rv[pos] = sub_prod(rv[pos], fih, sv[t]);
      }
    }
    __syncwarp();  // every lane has read rv[q] and applied this pivot
    if (q < dp && hl == 0) rv[q] = fih;
  }
  __syncwarp();
  if (hl < m) fv[b0 + hl] = rv[hl];
  if (hl == 0 && row >= 0) {
    const double d = rv[dp];
    rdx[row] = div_prep(d).x;
    if (d == 0.0) numeric_report(s_bad, s_badrow, ILUK_EZEROPIVOT, row);
  }
  __syncwarp();
  return true;
}

template <int NT>
__device__ bool cta_numeric(const BatchItemDev &it, double *fv, unsigned long long *rdx,
                            double *svals, int32_t *scols, double *stage_base, int cap,
                            BatchResultDev *res) {
  constexpr int kBWarps = NT / 32;
  // half-warp pairs where half a staging area holds a 7-point ILU(1) row
  constexpr bool kPairs = WarpStage<NT>::kPairs / 2 >= 40;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double *rv = svals + (size_t)wid * cap;
  int32_t *rc = scols + (size_t)wid * cap;
  const WarpStage<NT> st(stage_base + (size_t)wid * (kDotP / kBWarps));
  __shared__ int s_bad;
  __shared__ long long s_badrow;
  if (threadIdx.x == 0) {
    s_bad = 0;
    s_badrow = 0x7fffffffffffffffLL;
  }
  __syncthreads();
  for (int l = 0; l < it.nlev_l; ++l) {
    const int64_t lb = it.lstart[l], le = it.lstart[l + 1];
    if (kPairs) {
      for (int64_t sp = lb + 2 * wid; sp < le; sp += 2 * kBWarps) {
        const int64_t rowA = it.lord[sp];
        const int64_t rowB = sp + 1 < le ? it.lord[sp + 1] : -1;
        if (!numeric_rows_half<NT>(it, fv, rdx, rv, rc, st, rowA, rowB, lane, &s_bad,
                                   &s_badrow)) {
          if (rowA >= 0) numeric_row_warp<NT>(it, fv, rdx, rv, rc, st, rowA, lane, &s_bad, &s_badrow);
          if (rowB >= 0) numeric_row_warp<NT>(it, fv, rdx, rv, rc, st, rowB, lane, &s_bad, &s_badrow);
        }
      }
    } else {
      for (int64_t slot = lb + wid; slot < le; slot += kBWarps) {
        const int64_t row = it.lord[slot];
        if (row >= 0) numeric_row_warp<NT>(it, fv, rdx, rv, rc, st, row, lane, &s_bad, &s_badrow);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && s_bad) {
    res->status = s_bad;
    res->row = s_badrow;
  }
  __syncthreads();
  return s_bad == 0;
}

template <int NT, bool SPIN>
__device__ bool cta_apply(const BatchItemDev &it, const double *fv, const unsigned long long *rdx,
                          const double *p, double *tmp, double *y, int64_t limit_ns) {
  if (SPIN)
    return cta_sweep_spin<NT, true>(it, fv, rdx, p, tmp, limit_ns) &&
           cta_sweep_spin<NT, false>(it, fv, rdx, tmp, y, limit_ns);
  cta_sweep<NT, true>(it, fv, rdx, p, tmp);
  cta_sweep<NT, false>(it, fv, rdx, tmp, y);
  return true;
}

template <int NT>
__device__ void cta_vec_div(int64_t n, const double *x, double den, double *y) {
  if (den != 0.0) {
    const DivPrep pd = div_prep(den);  // one reciprocal, n quotients
    for (int64_t i = threadIdx.x; i < n; i += NT) y[i] = div_fin(x[i], pd);
  }
  __syncthreads();
}

// --- the persistent kernel ---------------------------------------------------

template <int NT, bool SPIN>
__global__ void __launch_bounds__(NT, 1024 / NT)
k_batch_solve(const BatchItemDev *items, int64_t nitems, BatchResultDev *results,
              BatchWork *work, unsigned long long *ticket, int m, double rtol, int maxit,
              int cap, int64_t limit_ns) {
  constexpr int kBWarps = NT / 32;
  // dynamic shared memory: the inner-product partials, the Hessenberg matrix
  // and rotations of a cycle (sized by m), then each warp's row slice
  extern __shared__ __align__(16) unsigned char smem[];
  double *sh = reinterpret_cast<double *>(smem);                 // kDotP doubles
  double *H = sh + kDotP;                                        // (m + 1) * m
  double *cs = H + (size_t)(m + 1) * m;                          // m
  double *sn = cs + m;                                           // m
  double *gv = sn + m;                                           // m + 1
  double *yv = gv + m + 1;                                       // m
  double *svals = yv + m;                                        // kBWarps * cap
  int32_t *scols = reinterpret_cast<int32_t *>(svals + (size_t)kBWarps * cap);
  // the published reciprocals of the diagonal (div_prep), one per row
  unsigned long long *rdx = reinterpret_cast<unsigned long long *>(work[blockIdx.x].u);
  __shared__ unsigned long long s_item;
  __shared__ int s_stop;
  const BatchWork wk = work[blockIdx.x];

  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(ticket, 1ull);
    __syncthreads();
    const unsigned long long id = s_item;
    __syncthreads();
    if (id >= (unsigned long long)nitems) return;
    const BatchItemDev it = items[id];
    BatchResultDev *res = results + id;
    const int64_t n = it.n;
    if (threadIdx.x == 0) {
      res->status = ILUK_OK;
      res->row = -1;
      res->iters = 0;
      res->cycles = 0;
      res->relres = 0.0;
    }
    if (!cta_numeric<NT>(it, wk.fval, rdx, svals, scols, sh, cap, res)) continue;

    // GMRES(m): the same steps, in the same order, as gmres_solve.
    const double bnorm = cta_dot<NT>(n, const_cast<double *>(it.b), nullptr, 0.0, false, nullptr,
                                     sh, true);
    for (int64_t i = threadIdx.x; i < n; i += NT) it.x[i] = 0.0;
    __syncthreads();
    int iters = 0, cycles = 0;
    double relres = 0.0;
    int status = ILUK_ENOCONV;
    if (bnorm == 0.0) status = ILUK_OK;
    while (bnorm != 0.0) {
      cta_spmv<NT>(it, it.x, wk.w, it.b);
      const double beta = cta_dot<NT>(n, wk.w, nullptr, 0.0, false, nullptr, sh, true);
      relres = beta / bnorm;
      if (relres <= rtol) { status = ILUK_OK; break; }
      if (iters >= maxit) { status = ILUK_ENOCONV; break; }
      ++cycles;
      cta_vec_div<NT>(n, wk.w, beta, wk.V);
      if (threadIdx.x == 0) gv[0] = beta;
      int jend = -1;
      for (int j = 0; j < m; ++j) {
        double *vj = wk.V + (size_t)j * wk.ldv;
        double *zj = wk.z + (size_t)j * wk.ldv;
        if (!cta_apply<NT, SPIN>(it, wk.fval, rdx, vj, wk.tmp, zj, limit_ns)) {
          if (threadIdx.x == 0) s_stop = 3;  // a bounded wait ran out
          __syncthreads();
          break;
        }
        cta_spmv<NT>(it, zj, wk.w, nullptr);
        double hval = cta_dot<NT>(n, wk.w, nullptr, 0.0, false, wk.V, sh, false);
        if (threadIdx.x == 0) H[0 * m + j] = hval;
        for (int i = 0; i <= j; ++i) {
          const double *vi = wk.V + (size_t)i * wk.ldv;
          const double *vn = (i < j) ? wk.V + (size_t)(i + 1) * wk.ldv : nullptr;
          hval = cta_dot<NT>(n, wk.w, vi, hval, true, vn, sh, i == j);
          if (threadIdx.x == 0) H[(i + 1) * m + j] = hval;
        }
        const double hn = hval;
        cta_vec_div<NT>(n, wk.w, hn, wk.V + (size_t)(j + 1) * wk.ldv);
        if (threadIdx.x == 0) {
          s_stop = 0;
          for (int i = 0; i < j; ++i) {
            const double a = H[i * m + j], c = H[(i + 1) * m + j];
            const double t1 = __dmul_rn(cs[i], a), t2 = __dmul_rn(sn[i], c);
            const double t3 = __dmul_rn(sn[i], a), t4 = __dmul_rn(cs[i], c);
            H[i * m + j] = __dadd_rn(t1, t2);
            H[(i + 1) * m + j] = __dsub_rn(t4, t3);
          }
          const double a = H[j * m + j], c = H[(j + 1) * m + j];
          const double rr = __dsqrt_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(c, c)));
          if (rr == 0.0) {
            s_stop = 2;
          } else {
            cs[j] = __ddiv_rn(a, rr);
            sn[j] = __ddiv_rn(c, rr);
            H[j * m + j] = rr;
            H[(j + 1) * m + j] = 0.0;
            gv[j + 1] = -__dmul_rn(sn[j], gv[j]);
            gv[j] = __dmul_rn(cs[j], gv[j]);
            const bool conv = __ddiv_rn(fabs(gv[j + 1]), bnorm) <= rtol;
            if (conv || iters + 1 >= maxit || hn == 0.0) s_stop = 1;
          }
        }
        __syncthreads();
        if (s_stop == 2) break;
        ++iters;
        jend = j;
        if (s_stop == 1) break;
      }
      if (s_stop == 2) { status = ILUK_EINVAL; break; }
      if (s_stop == 3) { status = ILUK_ETIMEOUT; break; }
      if (threadIdx.x == 0) {
        for (int i = jend; i >= 0; --i) {
          double sacc = gv[i];
          for (int l = i + 1; l <= jend; ++l) sacc = __dsub_rn(sacc, __dmul_rn(H[i * m + l], yv[l]));
          yv[i] = __ddiv_rn(sacc, H[i * m + i]);
        }
      }
      __syncthreads();
      // x += Z y, each entry summed over j in order from +0.0
      for (int64_t q = threadIdx.x; q < n; q += NT) {
        double sacc = 0.0;
        for (int jj = 0; jj <= jend; ++jj)
          sacc = __dadd_rn(sacc, __dmul_rn(yv[jj], wk.z[(size_t)jj * wk.ldv + q]));
        it.x[q] = __dadd_rn(it.x[q], sacc);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      res->status = status;
      res->iters = iters;
      res->cycles = cycles;
      res->relres = relres;
    }
    __syncthreads();
  }
}

size_t batch_smem_bytes(int nt, int cap, int m) {
  return (size_t)kDotP * 8 + ((size_t)(m + 1) * m + 4 * (size_t)m + 1) * 8 +
         (size_t)(nt / 32) * cap * 12;
}

int batch_max_restart() { return kBMaxRestart; }

template <int NT>
static cudaError_t launch_bs(const void *items, int64_t nitems, void *results, void *work,
                             int64_t nwork, unsigned long long *ticket, int m, double rtol,
                             int maxit, int cap, bool spin, cudaStream_t s) {
  const size_t smem = batch_smem_bytes(NT, cap, m);
  auto kern = spin ? k_batch_solve<NT, true> : k_batch_solve<NT, false>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // as many CTAs as fit on the GPU at once, within the work slots
  int bps = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, NT, smem);
  if (e != cudaSuccess) return e;
  if (bps < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)bps * num_sms();
  if (grid > nwork) grid = nwork;
  kern<<<(unsigned)grid, NT, smem, s>>>((const BatchItemDev *)items, nitems,
                                         (BatchResultDev *)results, (BatchWork *)work, ticket, m,
                                         rtol, maxit, cap, wait_limit());
  note_launch();
  return cudaGetLastError();
}

// nt = threads per instance (256, 512 or 1024); at most nwork CTAs (the work
// slots), as many as fit on the GPU at once.
cudaError_t launch_batch_solve(int nt, bool spin, const void *items, int64_t nitems,
                               void *results, void *work, int64_t nwork,
                               unsigned long long *ticket, int m, double rtol, int maxit, int cap,
                               cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_BATCH, s);
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (nt == 256)
    return launch_bs<256>(items, nitems, results, work, nwork, ticket, m, rtol, maxit, cap, spin,
                          s);
  if (nt == 512)
    return launch_bs<512>(items, nitems, results, work, nwork, ticket, m, rtol, maxit, cap, spin,
                          s);
  return launch_bs<1024>(items, nitems, results, work, nwork, ticket, m, rtol, maxit, cap, spin,
                         s);
}

size_t batch_item_bytes() { return sizeof(BatchItemDev); }
size_t batch_result_bytes() { return sizeof(BatchResultDev); }
size_t batch_work_bytes() { return sizeof(BatchWork); }

// Host-side packing of descriptors (layouts are private to this file).
void batch_pack_item(void *dst, const iluk_sym *S, const int64_t *arp, const int32_t *aci,
                     const double *aval, const double *b, double *x) {
  BatchItemDev d;
  d.n = S->n;
  d.nnzA = S->nnzA;
  d.nnzF = S->nnz;
  d.arp = arp;
  d.aci = aci;
  d.aval = aval;
  d.frp = S->rowptr;
  d.fci = S->colind;
  d.fdiag = S->diag;
  d.farp = S->arowptr;
  d.a2f = S->a2f;
  d.lord = S->lord.order;
  d.lstart = S->lord.lstart;
  d.nlev_l = S->lord.nlev;
  d.uord = S->uord.order;
  d.ustart = S->uord.lstart;
  d.nlev_u = S->uord.nlev;
  d.b = b;
  d.x = x;
  *reinterpret_cast<BatchItemDev *>(dst) = d;
}

void batch_pack_work(void *dst, double *fval, double *V, double *w, double *z, double *u,
                     double *tmp, int64_t ldv) {
  BatchWork d{fval, V, w, z, u, tmp, ldv};
  *reinterpret_cast<BatchWork *>(dst) = d;
}

void batch_unpack_result(const void *src, int32_t *status, int32_t *iters, int32_t *cycles,
                         int64_t *row, double *relres) {
  const BatchResultDev &r = *reinterpret_cast<const BatchResultDev *>(src);
  *status = r.status;
  *iters = r.iters;
  *cycles = r.cycles;
  *row = r.row;
  *relres = r.relres;
}

}  // namespace iluk
