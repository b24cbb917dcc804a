// numeric.cu -- a3: numeric ILU(k) factorization, row-wise IKJ elimination
// (Eq. 1; Eqs. lufactor2 and lufactor of Sec. 3.5), one warp per row.
//
// Row i is scattered from A onto F's pattern in the warp's shared-memory
// slice (fill positions +0.0).  For each h in L(i), ascending, the warp finds
// where row h's entries j > h fall in row i (pattern only, before row h is
// final), waits for the values of row h, forms the multiplier f_ih / f_hh by
// IEEE division and applies f_ij <- f_ij - f_ih * f_hj (one rounding for the
// product, one for the difference).  Lanes own distinct j, so each
// entry sees its updates in ascending h, exactly as the sequential algorithm
// does.  The finished row is written back, diagonal and upper part first.
// Pivots are pipelined three deep (see PivotA); rows are claimed in index
// order, or in forward level order once that is known.
//
// The batched form runs `nbatch` value sets on the same pattern in the same
// persistent launch: tickets are handed out row-major over (row, set), so
// every set advances through the rows together and the sets' independent
// rows fill the GPU while each set's dependency chain is walked.
//
// k_factor_fused runs this phase beside the symbolic one in one launch, each
// row starting as soon as its pattern is final (see the section below).
#include "internal.h"
#include "symbolic_body.cuh"

namespace iluk {

constexpr int kNumThreads = 256;
// Static shared memory of the numeric kernels (apply_pivots' per-warp
// bitmaps), left out of the dynamic shared memory's budget.
constexpr int kTouchedWords = 16;  // bitmap words per warp: rows of up to 512 entries
constexpr size_t kStaticSmem = (kNumThreads / 32) * kTouchedWords * sizeof(unsigned);
// Average entries per row of F from which the refactorization publishes
// entries early (random band, k = 2, 119 a row: 30.6 -> 25.8 ms; grids of 9 to
// 61 a row lost 5-10 %).
constexpr int64_t kEarlyRowLen = 80;
// Entries of L per forward level below which the refactorization publishes
// early whatever the row length (band matrices: 560-830 a level; 3D grids:
// 4,000-19,000).
constexpr int64_t kEarlyLevelEntries = 2000;
// Sixteenths of the fused factorization's CTAs that run the symbolic walk:
// few with the level-map walk, which keeps ahead of the numeric rows easily;
// more with the sorted-list walk of wide matrices, which is slower per row.
// (On the 7-point 3D 64^3 grid, k = 2: 58 ms at 3/16, 23 ms at 8/16, 37 ms
// at 12/16.)  With the level map, how far ahead the walk must run depends on
// how long the numeric rows take: where A has long rows (they fill in to
// long rows of F, each numeric row is slow) a smaller share leaves more SMs
// to the numeric rows (random band, n = 160,000, 10 entries a row, k = 2:
// 30.3 ms at 4/16, 29.1 ms at 3/16 and 2/16); where rows are short the walk
// needs its 4/16 (2D 256^2 grid, 5 a row: 32.5 ms at 4/16, 40.6 at 3/16,
// 50.5 at 2/16).
constexpr int kFusedSymPartMap = 4;
constexpr int kFusedSymPartMapLongRows = 3;
constexpr int64_t kLongRowsOfA = 8;  // entries per row of A, on average
constexpr int kFusedSymPartList = 8;

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

// Pivot row h, as the warp stages it before its values are final.  Stage A
// issues the loads of f_hh and of the columns j of the first kPre * 32
// entries j > h; stage B, one pivot later,
// turns those columns into positions in the current row (pos, -1 if absent)
// and issues the loads of the matching f_hj; stage C, one more pivot later,
// waits for whatever is still pending and applies the pivot.  The per-entry
// pivot facts (where row h's diagonal sits, how long its U part is) come from
// a table built with the pattern, so no stage waits on a dependent load.
constexpr int kPre = 4;
constexpr unsigned kPollSleepMax = 64;
constexpr int kUlenBits = 24;  // pivot info = diag position << 24 | U length

struct PivotA {
  int64_t hd;
  int ulen;
  int32_t j[kPre];
  double piv;
  unsigned long long xr;  // the pivot row's published reciprocal of f_hh, or ~0
};

struct PivotPre {
  int64_t hd;
  int ulen;
  int pos[kPre];
  double piv, f[kPre];
  unsigned long long xr;
};

// Where column j sits in the current row: a dense map over the row's column
// span when it fits in shared memory, else a binary search from `lo`.
struct RowIndex {
  const int32_t *rc;
  const int16_t *map;
  int32_t c0;
  int span, m;
  bool use_map;
  __device__ __forceinline__ int find(int32_t j, int lo) const {
    if (use_map) {
      const int d = j - c0;
      return (d >= 0 && d < span) ? (int)map[d] : -1;
    }
    const int ps = lower_bound_i(rc, lo, m, j);
    return (ps < m && rc[ps] == j) ? ps : -1;
  }
};

__device__ __forceinline__ void stage_a(PivotA &a, int64_t pinfo, const int32_t *__restrict__ fci,
                                        const double *fv, int lane, const DivPrep *rdp, int32_t h) {
  a.hd = pinfo >> kUlenBits;
  a.ulen = (int)(pinfo & ((1ll << kUlenBits) - 1));
  a.piv = ld_gpu(&fv[a.hd]);
  a.xr = ~0ull;
  if (rdp) asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(a.xr) : "l"(&rdp[h].x));
#pragma unroll
  for (int c = 0; c < kPre; ++c) {
    const int e = lane + 32 * c;
    a.j[c] = e < a.ulen ? fci[a.hd + 1 + e] : -1;
  }
}

__device__ __forceinline__ void stage_b(PivotPre &pp, const PivotA &a, const RowIndex &ri, int q,
                                        const double *fv, int lane) {
  pp.hd = a.hd;
  pp.ulen = a.ulen;
  pp.piv = a.piv;
  pp.xr = a.xr;
  int lo = q + 1;  // a lane's columns increase with c: each search starts where the last ended
#pragma unroll
  for (int c = 0; c < kPre; ++c) {
    pp.pos[c] = -1;
    pp.f[c] = 0.0;
    if (a.j[c] >= 0) {
      const int ps = ri.find(a.j[c], lo);
      if (ps >= 0) {
        lo = ps;
        pp.pos[c] = ps;
        pp.f[c] = ld_gpu(&fv[pp.hd + 1 + lane + 32 * c]);
      }
    }
  }
}

// Re-issue the loads of the values of a staged pivot that are still pending.
// The loads are independent, so they travel together: one round trip
// refreshes the whole pivot.
__device__ __forceinline__ void refresh_pivot(PivotPre &pp, const double *fv, int lane) {
  if (pend_f(pp.piv)) pp.piv = ld_gpu(&fv[pp.hd]);
#pragma unroll
  for (int c = 0; c < kPre; ++c)
    if (pp.pos[c] >= 0 && pend_f(pp.f[c])) pp.f[c] = ld_gpu(&fv[pp.hd + 1 + lane + 32 * c]);
}

__device__ __forceinline__ bool pivot_pending(const PivotPre &pp) {
  bool p = pend_f(pp.piv);
#pragma unroll
  for (int c = 0; c < kPre; ++c) p |= pp.pos[c] >= 0 && pend_f(pp.f[c]);
  return p;
}

// Warp-uniform wait until f_hh and every staged f_hj of the pivot are final,
// polling all of them at once.  False on time-out or when a row before `row`
// has failed.
__device__ __forceinline__ bool wait_pivot(PivotPre &pp, const double *fv, int lane,
                                           const DevErr *err, int64_t row, int64_t limit_ns) {
  if (!__any_sync(FULL_MASK, pivot_pending(pp))) return true;
  const uint64_t t0 = globaltimer_ns();
  unsigned backoff = 16;
  for (unsigned it = 0;; ++it) {
    refresh_pivot(pp, fv, lane);
    if (!__any_sync(FULL_MASK, pivot_pending(pp))) return true;
    const bool stop = (it & 31u) == 31u &&
                      (earlier_failed(err, row) || (int64_t)(globaltimer_ns() - t0) > limit_ns);
    if (__any_sync(FULL_MASK, stop)) return false;  // the whole warp gives up together
    if (it >= 4) {  // a short spin first, then a bounded back-off
      __nanosleep(backoff);
      if (backoff < kPollSleepMax) backoff <<= 1;
    }
  }
}

// The row's diagonal with its fixed-point reciprocal, for the later rows
// that divide by it (the x word, ~0 until written, is what they look for)
// and for the sweeps.
__device__ __forceinline__ void publish_recip(DivPrep *d, double fii) {
  const DivPrep p = div_prep(fii);
  d->b = p.b;
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(&d->x), "l"(p.x) : "memory");
}

// The row's depth in the forward DAG (Sec. 3.6's level sets): 1 + the
// deepest of its pivot rows (cols[0..dp)), written once the row is written
// back.  Those rows are written back already and set their own depth right
// after, so each wait is short; depth 0 means not yet.  maxdepth collects
// the DAG's depth, from which the factorization judges the DAG's width.
// Warp-uniform; gives up (no depth) on time-out or an earlier row's failure.
__device__ __forceinline__ void note_depth(int64_t row, int dp, const int32_t *cols,
                                           int32_t *depth, unsigned *maxdepth, const DevErr *err,
                                           int64_t limit_ns, int lane) {
  int dm = 0;
  bool ok = true;
  for (int q = lane; q < dp; q += 32) {
    const int32_t *p = &depth[cols[q]];
    int d;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(d) : "l"(p));
    if (d == 0) {
      const uint64_t t0 = globaltimer_ns();
      for (unsigned it = 0; d == 0; ++it) {
        __nanosleep(64);
        asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(d) : "l"(p));
        if ((it & 15u) == 15u &&
            (earlier_failed(err, row) || (int64_t)(globaltimer_ns() - t0) > limit_ns)) {
          ok = false;
          break;
        }
      }
    }
    if (d > dm) dm = d;
  }
  dm = __reduce_max_sync(FULL_MASK, dm) + 1;
  if (__all_sync(FULL_MASK, ok) && lane == 0) {
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(depth + row), "r"(dm) : "memory");
    atomicMax(maxdepth, (unsigned)dm);
  }
}

// Where the row's finished entries go (position q of the row, diagonal at
// dp): out[at(q)].  `out` null: nowhere, the caller writes the row back.
struct CsrOut {
  double *out;
  int64_t b0;
  __device__ __forceinline__ int64_t at(int q) const { return b0 + q; }
};
struct ArenaOut {  // a slot: diagonal, upper part, end marker, lower part
  double *out;
  int64_t slot;
  int dp, mu;
  __device__ __forceinline__ int64_t at(int q) const {
    return q < dp ? slot + mu + 2 + q : slot + (q - dp);
  }
};

// Row i's pivots, ascending: the staged pipeline (see PivotA) applied to the
// row in shared memory.  fci and fv hold the pivot rows' columns and values
// at their diagonal position hd and the upper part after it (CSR, or a slot of
// the factorization arena); spinfo[q] = hd << 24 | |U(h)| for the row's q-th
// lower entry h.  Warp-uniform; false on time-out or an earlier row's failure.
//
// The diagonal and upper part are what later rows wait for, so they leave as
// soon as they are final.  The last pivot's positions in the row are known
// (stage B) before its values arrive: every diagonal/upper entry it does not
// touch is final already and goes out before the wait (`touched`, a 16-word
// per-warp bitmap over the row's positions); the entries it does touch go
// out from registers as each update completes.  Then *upper_sent is true and
// the caller writes only the lower part.  (A row longer than the bitmap, or a
// last pivot row longer than the staged chunks, leaves it all to the caller.)
template <bool EARLY, typename Out>
__device__ __forceinline__ bool apply_pivots(int dp, double *rv, const int64_t *spinfo,
                                             const RowIndex &ri, const int32_t *__restrict__ fci,
                                             const double *fv, const DevErr *err, int64_t row,
                                             int64_t limit_ns, int lane, const Out &out, int m,
                                             unsigned *touched, bool *upper_sent,
                                             const DivPrep *rdp) {
  // Pivots go through the three stages (see PivotA): in iteration q the
  // warp applies pivot q, finds the positions of pivot q+1 and issues the
  // loads of pivot q+2, so the latencies of the later stages overlap the
  // work and the waits of the earlier ones.
  bool ok = true;
  PivotA pa;
  PivotPre cur, nxt;
  if (dp > 0) {
    stage_a(pa, spinfo[0], fci, fv, lane, rdp, ri.rc[0]);
    stage_b(cur, pa, ri, 0, fv, lane);
  }
  if (dp > 1) stage_a(pa, spinfo[1], fci, fv, lane, rdp, ri.rc[1]);
  for (int q = 0; q < dp && ok; ++q) {
    if (q + 1 < dp) stage_b(nxt, pa, ri, q + 1, fv, lane);
    if (q + 2 < dp) stage_a(pa, spinfo[q + 2], fci, fv, lane, rdp, ri.rc[q + 2]);
    const bool early = EARLY && out.out != nullptr && q + 1 == dp && cur.ulen <= 32 * kPre &&
                       m <= 32 * kTouchedWords;
    if (early) {
      if (lane < kTouchedWords) touched[lane] = 0u;
      __syncwarp();
#pragma unroll
      for (int c = 0; c < kPre; ++c)
        if (cur.pos[c] >= 0) atomicOr(&touched[cur.pos[c] >> 5], 1u << (cur.pos[c] & 31));
      __syncwarp();
      for (int t = dp + lane; t < m; t += 32)
        if (!((touched[t >> 5] >> (t & 31)) & 1u)) out.out[out.at(t)] = rv[t];
      *upper_sent = true;
    }
    if (!wait_pivot(cur, fv, lane, err, row, limit_ns)) {
      ok = false;
      break;
    }
    // The multiplier f_ih / f_hh, correctly rounded, on the integer pipes
    // (div_int): a fraction of the latency of an FP64 division, and it
    // leaves the FP64 pipe to the updates.  A pivot row publishes the
    // fixed-point reciprocal of its diagonal (rdp[h].x) once it has written
    // itself back; when that is already there at staging, only the remainder
    // half of the division is left (div_fin).  Same quotient either way.
    const unsigned long long xr = __shfl_sync(FULL_MASK, cur.xr, 0);
    const double fih =
        xr != ~0ull ? div_fin(rv[q], DivPrep{xr, cur.piv}) : div_int(rv[q], cur.piv);
    __syncwarp();
    if (lane == 0) rv[q] = fih;
    // only the chunks the pivot row has: an FP64 instruction costs its
    // pipe time even with every lane predicated off
    const int nch = (cur.ulen + 31) >> 5;
#pragma unroll
    for (int c = 0; c < kPre; ++c) {
      if (c >= nch) break;
      if (cur.pos[c] >= 0) {
        const double nv = sub_prod(rv[cur.pos[c]], fih, cur.f[c]);
        rv[cur.pos[c]] = nv;
        if (early && cur.pos[c] >= dp) out.out[out.at(cur.pos[c])] = nv;  // final: out now
      }
    }
    const int64_t u1 = cur.hd + 1 + cur.ulen;
    for (int64_t base = cur.hd + 1 + 32 * kPre; base < u1; base += 32) {  // long rows
      const int64_t r = base + lane;
      int pos = -1;
      double fhj = 0.0;
      if (r < u1) {
        pos = ri.find(fci[r], q + 1);
        if (pos >= 0) fhj = ld_gpu(&fv[r]);
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
  return __all_sync(FULL_MASK, ok);
}

// Pivot facts per lower entry (i, h) of F: position of row h's diagonal and
// the length of its strictly upper part, packed for the numeric phase.
__global__ void k_pivot_info(int64_t n, const int64_t *__restrict__ frp,
                             const int32_t *__restrict__ fci, const int64_t *__restrict__ fdiag,
                             int64_t *pinfo) {
  const int lane = threadIdx.x & 31;
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < n; row += nw)
    for (int64_t p = frp[row] + lane; p < fdiag[row]; p += 32) {
      const int32_t h = fci[p];
      const int64_t hd = fdiag[h];
      pinfo[p] = (hd << kUlenBits) | (frp[h + 1] - hd - 1);
    }
}

cudaError_t launch_pivot_info(int64_t n, const int64_t *frp, const int32_t *fci,
                              const int64_t *fdiag, int64_t *pinfo, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_COMPACT, s);  // pattern post-processing
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n * 32 + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  k_pivot_info<<<(unsigned)blocks, 256, 0, s>>>(n, frp, fci, fdiag, pinfo);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_fill_pending_f(int64_t n, double *x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = __longlong_as_double((long long)kPendingF);
}

template <bool EARLY>
__global__ void __launch_bounds__(kNumThreads)
k_numeric(int64_t n, int64_t nbatch, const int64_t *__restrict__ arp,
          const int32_t *__restrict__ a2f, const double *__restrict__ aval, int64_t astride,
          const int64_t *__restrict__ frp, const int32_t *__restrict__ fci,
          const int64_t *__restrict__ fdiag, const int64_t *__restrict__ pinfo, double *fval,
          int64_t fstride, const int32_t *__restrict__ order,
          unsigned long long *ticket, DevErr *errs, int cap, int map_cap, int64_t limit_ns,
          int64_t hold, DivPrep *rdiag, int32_t *depth, unsigned *maxdepth) {
  // per warp: values, pivot infos (cap each), columns, then the column map
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  double *svals = reinterpret_cast<double *>(smem) + (size_t)wib * cap;
  int64_t *spinfo = reinterpret_cast<int64_t *>(smem + (size_t)nwarps * cap * 8) + (size_t)wib * cap;
  int32_t *scols =
      reinterpret_cast<int32_t *>(smem + (size_t)nwarps * cap * 16) + (size_t)wib * cap;
  int16_t *smap =
      reinterpret_cast<int16_t *>(smem + (size_t)nwarps * cap * 20) + (size_t)wib * map_cap;
  unsigned *touched_w = nullptr;  // see apply_pivots
  if constexpr (EARLY) {
    __shared__ unsigned touched[kNumThreads / 32][kTouchedWords];
    touched_w = touched[wib];
  }
  const int64_t total = n * nbatch;

  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(ticket, 1ull);
    const int64_t t = (int64_t)__shfl_sync(FULL_MASK, tk, 0);
    if (t >= total) return;
    // tickets walk the rows in level order when it is known (every row's
    // pivots then lie at earlier tickets, as in index order), else in index
    // order
    const int64_t slot = t / nbatch;
    const int64_t set = t - slot * nbatch;
    const int64_t row = order ? (int64_t)order[slot] : slot;
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
    for (int q = lane; q < dp; q += 32) spinfo[q] = pinfo[b0 + q];
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
    RowIndex ri;
    ri.rc = rc;
    ri.map = smap;
    ri.m = m;
    ri.c0 = rc[0];
    ri.span = rc[m - 1] - ri.c0 + 1;
    ri.use_map = ri.span <= map_cap;
    if (ri.use_map) {
      for (int d = lane; d < ri.span; d += 32) smap[d] = -1;
      __syncwarp();
      for (int q = lane; q < m; q += 32) smap[rc[q] - ri.c0] = (int16_t)q;
    }
    __syncwarp();

    bool upper_sent = false;
    const CsrOut out{row != hold ? fv : nullptr, b0};
    const bool ok = apply_pivots<EARLY>(dp, rv, spinfo, ri, fci, fv, err, row, limit_ns, lane,
                                        out, m, touched_w, &upper_sent, rdiag);
    if (!ok) {
      if (lane == 0 && !earlier_failed(err, row)) set_err(err, row, ILUK_ETIMEOUT);
      continue;
    }
    if (lane == 0 && rv[dp] == 0.0) set_err(err, row, ILUK_EZEROPIVOT);
    // the rest of the row: the diagonal and U part first (what later rows
    // wait for) unless they are out already, then the lower part
    if (row != hold) {
      if (upper_sent) {
        for (int q = lane; q < dp; q += 32) fv[b0 + q] = svals[q];
      } else {
        for (int t = lane; t < m; t += 32) {
          const int q = t + dp < m ? t + dp : t + dp - m;
          fv[b0 + q] = svals[q];
        }
      }
      if (rdiag && lane == 0) publish_recip(&rdiag[row], svals[dp]);
      if (depth) note_depth(row, dp, rc, depth, maxdepth, err, limit_ns, lane);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Symbolic and numeric phases in one launch (k >= 2).  The CTAs below g_sym
// run the symbolic row walk; the others factor rows as soon as the walk has
// finished them.  A numeric row waits for its own pattern (the symbolic row
// publishes (length << 32 | upper start) in rinfo once its slot is written)
// and for the values of its pivot rows, which live in a value arena laid out
// like the column arena: row h's slot holds the diagonal, the strictly upper
// part, an end marker and the strictly lower part, so the pivot pipeline above
// reads a pivot row at its slot exactly as it reads a CSR row at its diagonal
// position.  Both phases only wait for rows that come earlier in their own
// order (index order), and every CTA of the cooperative launch is resident,
// so the numeric CTAs' waits on the symbolic ones always end.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_u64_gpu(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

// Warp-uniform wait until *p is no longer ~0; false on time-out or failure.
__device__ __forceinline__ bool wait_word(const unsigned long long *p, unsigned long long *out,
                                          const DevErr *err, int64_t row, int64_t limit_ns) {
  unsigned long long v = ld_u64_gpu(p);
  if (v != ~0ull) {
    *out = v;
    return true;
  }
  const uint64_t t0 = globaltimer_ns();
  unsigned backoff = 16;
  for (unsigned it = 0;; ++it) {
    v = ld_u64_gpu(p);
    if (v != ~0ull) {
      *out = v;
      return true;
    }
    const bool stop = (it & 31u) == 31u &&
                      (earlier_failed(err, row) || (int64_t)(globaltimer_ns() - t0) > limit_ns);
    if (stop) return false;
    if (it >= 4) {
      __nanosleep(backoff);
      if (backoff < kPollSleepMax) backoff <<= 1;
    }
  }
}

// The forward substitution L x = v0 (L unit lower triangular, its strictly
// lower part the multipliers f_ih of Eq. 1) for one row, taken by the warp that
// has just factored that row: x_i = v0_i - sum over h in L(i), ascending, of
// f_ih * x_h, each product and each difference rounded once, in the order of
// the stand-alone forward sweep, so the result is bit for bit the sweep's.
// The row's multipliers and columns are still in the warp's shared memory.
// x lives in global memory, filled with kPendingF before the launch; x_h is
// polled until it leaves that state (the rows that own x_h were claimed
// earlier and are resident, so every wait ends).  A value that would equal
// the marker is stored as a quiet NaN, as the sweep does.  Warp-uniform;
// false on time-out or when a row before `row` has failed.
__device__ __forceinline__ bool forward_entry(int64_t row, int dp, const double *lmul,
                                              const int32_t *lcol, const double *v0, double *x,
                                              const DevErr *err, int64_t limit_ns, int lane) {
  double s = v0[row];
  for (int b = 0; b < dp; b += 32) {
    const int e = b + lane;
    const bool act = e < dp;
    const int cnt = dp - b < 32 ? dp - b : 32;
    double f = 0.0, prod = 0.0;
    int32_t c = 0;
    bool have = !act;
    if (act) {
      c = lcol[e];
      f = lmul[e];
      const double xh = ld_gpu(&x[c]);
      if (!pend_f(xh)) {
        prod = __dmul_rn(f, xh);
        have = true;
      }
    }
    int done = 0;
    const uint64_t t0 = globaltimer_ns();
    unsigned backoff = 16;
    for (unsigned it = 0;; ++it) {
      // subtract the ready products in order, up to the first missing one
      const unsigned ready = __ballot_sync(FULL_MASK, have);
      const unsigned rest = ~(ready >> done);
      const int run = rest == 0u ? 32 - done : __ffs(rest) - 1;
      const int upto = done + run < cnt ? done + run : cnt;
      for (int j = done; j < upto; ++j) s = __dsub_rn(s, __shfl_sync(FULL_MASK, prod, j));
      done = upto;
      if (done >= cnt) break;
      const bool stop = (it & 15u) == 15u &&
                        (earlier_failed(err, row) || (int64_t)(globaltimer_ns() - t0) > limit_ns);
      if (__any_sync(FULL_MASK, stop)) return false;
      __nanosleep(backoff);
      if (backoff < 128u) backoff <<= 1;
      if (!have) {
        const double xh = ld_gpu(&x[c]);
        if (!pend_f(xh)) {
          prod = __dmul_rn(f, xh);
          have = true;
        }
      }
    }
  }
  if ((unsigned long long)__double_as_longlong(s) == kPendingF)
    s = __longlong_as_double((long long)0x7FF8000000000000ll);
  if (lane == 0) asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(x + row), "d"(s) : "memory");
  return true;
}

__device__ void numeric_arena_rows(int64_t n, const int64_t *__restrict__ arp,
                                   const int32_t *__restrict__ aci,
                                   const double *__restrict__ aval, const int32_t *acol,
                                   double *vals, const unsigned long long *meta,
                                   const unsigned long long *rinfo, unsigned long long *ticket,
                                   DevErr *err, int cap, int map_cap, int64_t limit_ns,
                                   const double *v0, double *xf, DivPrep *rdiag,
                                   int32_t *depth, unsigned *maxdepth, unsigned char *smem) {
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  double *svals = reinterpret_cast<double *>(smem) + (size_t)wib * cap;
  int64_t *spinfo = reinterpret_cast<int64_t *>(smem + (size_t)nwarps * cap * 8) + (size_t)wib * cap;
  int32_t *scols =
      reinterpret_cast<int32_t *>(smem + (size_t)nwarps * cap * 16) + (size_t)wib * cap;
  int16_t *smap =
      reinterpret_cast<int16_t *>(smem + (size_t)nwarps * cap * 20) + (size_t)wib * map_cap;
  __shared__ unsigned touched[kNumThreads / 32][kTouchedWords];  // see apply_pivots
  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(ticket, 1ull);
    const int64_t row = (int64_t)__shfl_sync(FULL_MASK, tk, 0);
    if (row >= n) return;
    if (earlier_failed(err, row)) continue;
    // the row's pattern, once the symbolic walk has written it
    unsigned long long ri_w = 0;
    bool ok = lane == 0 ? wait_word(&rinfo[row], &ri_w, err, row, limit_ns) : true;
    ok = __shfl_sync(FULL_MASK, ok ? 1 : 0, 0) != 0;
    ri_w = __shfl_sync(FULL_MASK, ri_w, 0);
    if (!ok) {
      if (lane == 0 && !earlier_failed(err, row)) set_err(err, row, ILUK_ETIMEOUT);
      continue;
    }
    __threadfence();  // the row's slot entries were written before rinfo
    const int m = (int)(ri_w >> 32), ust = (int)(ri_w & 0xffffffffu);
    const int mu = m - ust, dp = ust - 1;
    if (m > cap) {  // longer than this launch's numeric slice: the host redoes it apart
      if (lane == 0) {
        set_err(err, row, ILUK_ENOMEM);
        atomicMax(&err->need, (unsigned long long)m);
      }
      continue;
    }
    const int64_t slot = (int64_t)ld_u64_gpu(&meta[row]);
    // columns in CSR order: lower part, diagonal, upper part
    for (int q = lane; q < m; q += 32) {
      const int64_t src = q < dp ? slot + mu + 2 + q : slot + (q - dp);
      int32_t c;
      asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(c) : "l"(acol + src));
      scols[q] = c;
      svals[q] = 0.0;
    }
    __syncwarp();
    // pivot facts: row h's slot (its diagonal) and upper length
    for (int q = lane; q < dp; q += 32) {
      const int32_t h = scols[q];
      unsigned long long rh = 0;
      if (!wait_word(&rinfo[h], &rh, err, row, limit_ns)) {
        ok = false;
      } else {
        const int64_t sh = (int64_t)ld_u64_gpu(&meta[h]);
        const int64_t muh = (int64_t)(rh >> 32) - (int64_t)(rh & 0xffffffffu);
        spinfo[q] = (sh << kUlenBits) | muh;
      }
    }
    if (!__all_sync(FULL_MASK, ok)) {
      if (lane == 0 && !earlier_failed(err, row)) set_err(err, row, ILUK_ETIMEOUT);
      continue;
    }
    __threadfence();  // the pivot rows' slot columns were written before their rinfo
    // A's row onto the pattern (A's columns are a subset of the row's)
    bool bad = false;
    for (int64_t p = arp[row] + lane; p < arp[row + 1]; p += 32) {
      const double a = aval[p];
      if (!isfinite(a)) bad = true;
      svals[lower_bound_i(scols, 0, m, aci[p])] = a;
    }
    if (__any_sync(FULL_MASK, bad)) {
      if (lane == 0) set_err(err, row, ILUK_ENONFINITE);
      continue;
    }
    RowIndex ri;
    ri.rc = scols;
    ri.map = smap;
    ri.m = m;
    ri.c0 = scols[0];
    ri.span = scols[m - 1] - ri.c0 + 1;
    ri.use_map = ri.span <= map_cap;
    if (ri.use_map) {
      for (int d = lane; d < ri.span; d += 32) smap[d] = -1;
      __syncwarp();
      for (int q = lane; q < m; q += 32) smap[scols[q] - ri.c0] = (int16_t)q;
    }
    __syncwarp();
    bool upper_sent = false;
    const ArenaOut out{vals, slot, dp, mu};
    if (!apply_pivots<true>(dp, svals, spinfo, ri, acol, vals, err, row, limit_ns, lane, out, m,
                            touched[wib], &upper_sent, rdiag)) {
      if (lane == 0 && !earlier_failed(err, row)) set_err(err, row, ILUK_ETIMEOUT);
      continue;
    }
    if (lane == 0 && svals[dp] == 0.0) set_err(err, row, ILUK_EZEROPIVOT);
    // the rest of the row into its slot: the diagonal and upper part first
    // (what later rows wait for) unless they are out already, then the lower
    // part
    if (upper_sent) {
      for (int q = lane; q < dp; q += 32) vals[out.at(q)] = svals[q];
    } else {
      for (int t = lane; t < m; t += 32) {
        const int q = t + dp < m ? t + dp : t + dp - m;
        vals[out.at(q)] = svals[q];
      }
    }
    if (rdiag && lane == 0) publish_recip(&rdiag[row], svals[dp]);
    __syncwarp();
    // the row's entry of L x = v0, when the launch carries the first
    // right-hand side
    if (xf && !forward_entry(row, dp, svals, scols, v0, xf, err, limit_ns, lane)) {
      if (lane == 0 && !earlier_failed(err, row)) set_err(err, row, ILUK_ETIMEOUT);
    }
    if (depth) note_depth(row, dp, scols, depth, maxdepth, err, limit_ns, lane);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kNumThreads)
k_factor_fused(int64_t n, const int64_t *__restrict__ arp, const int32_t *__restrict__ aci,
               const double *__restrict__ aval, int k, int32_t *arena_col, uint8_t *arena_lev,
               double *arena_val, int64_t arena_cap, unsigned long long *arena_top,
               int64_t *row_off, int32_t *row_len, int32_t *row_ust, unsigned long long *meta,
               unsigned long long *rinfo, unsigned long long *sym_ticket,
               unsigned long long *num_ticket, DevErr *err, int scap, int mapw, int64_t chunk,
               int ncap, int nmap, int g_sym, int64_t limit_ns, const double *v0, double *xf,
               DivPrep *rdiag, int32_t *depth, unsigned *maxdepth) {
  extern __shared__ __align__(16) unsigned char smem[];
  if ((int)blockIdx.x < g_sym)
    symbolic_rows_body<false, true>(n, arp, aci, k, arena_col, arena_lev, arena_cap, arena_top,
                                    row_off, row_len, row_ust, meta, sym_ticket, err, scap, mapw,
                                    chunk, limit_ns, rinfo, smem);
  else
    numeric_arena_rows(n, arp, aci, aval, arena_col, arena_val, meta, rinfo, num_ticket, err,
                       ncap, nmap, limit_ns, v0, xf, rdiag, depth, maxdepth, smem);
}

// Shared memory per warp: a row of F (value, pivot info, column: 20 bytes per
// entry) and a column map of map_cap int16.  The largest map that lets 8,
// then 4, 2, 1 warps share a CTA; rows whose column span exceeds the map
// fall back to binary search.
// kWideLevelRows (internal.h): on level orders this wide the numeric phase
// goes without the column map: the map's shared memory holds the launch to
// one CTA per SM, and here more rows in flight matter more than the map
// (refactorization of the 27-point 90^3 grid, 1,168 rows a level: 10.1 ->
// 5.9 ms; C3, 378 a level: 3.46 -> 2.71 ms; 196 and 64 a level lost 2-3 %).

static int numeric_cap(const iluk_sym *S, size_t static_smem, bool wide, int *warps_out,
                       int *map_out, size_t *smem_out) {
  int cap = S->max_row;
  if (cap < 32) cap = 32;
  cap = (cap + 31) & ~31;
  const size_t budget = (size_t)max_smem_optin() - static_smem;
  for (int warps : {8, 4, 2, 1})
    for (int map : {8192, 4096, 0}) {
      if (wide && map) continue;
      const size_t need = ((size_t)cap * 20 + (size_t)map * 2) * warps;
      if (need <= budget) {
        *warps_out = warps;
        *map_out = map;
        *smem_out = need;
        return cap;
      }
    }
  return -1;  // a row of F exceeds shared memory
}

static cudaError_t launch_numeric_impl(const iluk_sym *S, int64_t nbatch, const double *avals,
                                       double *fvals, DivPrep *rdiag, unsigned long long *ticket,
                                       DevErr *errs, int32_t *depth, unsigned *maxdepth,
                                       cudaStream_t s) {
  // the forward level order, once built, is a valid and better-spread order
  const int32_t *order = S->levels_built ? S->lord.corder : nullptr;
  ProfScope prof_scope(ILUK_PROF_NUMERIC, s);
  const bool wide = order != nullptr && S->n >= kWideLevelRows * (int64_t)S->lord.nlev;
  // rows publish their entries as soon as final (see apply_pivots) where F's
  // rows are long, or where a level holds few entries of L (fewer than
  // kEarlyLevelEntries: the band matrices at k <= 1 gain 15-35 %), or before
  // the level orders exist; on grids, whose levels hold thousands of short
  // rows' entries (3D 7- and 27-point stencils), it measured 5-10 % slower
  const bool early = S->nnz >= kEarlyRowLen * S->n || order == nullptr ||
                     (S->nnz - S->n) / 2 < kEarlyLevelEntries * (int64_t)S->lord.nlev;
  const auto kern = early ? k_numeric<true> : k_numeric<false>;
  int warps, map_cap;
  size_t smem;
  const int cap = numeric_cap(S, early ? kStaticSmem : 0, wide, &warps, &map_cap, &smem);
  if (cap < 0) return cudaErrorMemoryAllocation;
  {
    const int64_t nv = S->nnz * nbatch;
    int64_t b = (nv + 255) / 256;
    if (b > (int64_t)num_sms() * 8) b = (int64_t)num_sms() * 8;
    if (b < 1) b = 1;
    k_fill_pending_f<<<(unsigned)b, 256, 0, s>>>(nv, fvals);
    note_launch();
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, warps * 32, smem);
  if (bps < 1) bps = 1;
  int64_t grid = (int64_t)bps * num_sms();
  const int64_t want = (S->n * nbatch + warps - 1) / warps;
  if (grid > want) grid = want;
  if (grid < 1) grid = 1;
  if (rdiag) {  // every row writes its own entry; ~0 marks the ones not written yet
    e = cudaMemsetAsync(rdiag, 0xff, (size_t)S->n * sizeof(DivPrep), s);
    if (e != cudaSuccess) return e;
  }
  kern<<<(unsigned)grid, warps * 32, smem, s>>>(
      S->n, nbatch, S->arowptr, S->a2f, avals, S->nnzA, S->rowptr, S->colind, S->diag, S->pinfo,
      fvals, S->nnz, order, ticket, errs, cap, map_cap, wait_limit(), hold_row(), rdiag, depth,
      maxdepth);
  note_launch();
  return cudaGetLastError();
}

// Symbolic (k >= 2) and numeric phases in one cooperative launch.  The symbolic
// CTAs use the symbolic kernel's per-warp layout (scap, mapw); the numeric
// CTAs hold rows of at most ncap entries.  Fails (cudaErrorInvalidConfiguration)
// when the two layouts do not fit one CTA's shared memory or the grid has room
// for fewer than two CTAs.
cudaError_t launch_factor_fused(int64_t n, int64_t nnz_a, const int64_t *arp,
                                const int32_t *aci, const double *aval, int k, const SymArena &ar,
                                double *arena_val, unsigned long long *rinfo,
                                unsigned long long *num_ticket, DevErr *err, int scap, int mapw,
                                int ncap, const double *v0, double *xf, DivPrep *rdiag,
                                int32_t *depth, unsigned *maxdepth, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_FACTOR, s);
  const int warps = kNumThreads / 32;
  const size_t sym_smem = (symbolic_smem_per_warp(scap) + symbolic_map_per_warp(mapw)) * warps;
  int nmap = 0;
  size_t num_smem = 0;
  for (int map : {8192, 4096, 0}) {
    num_smem = ((size_t)ncap * 20 + (size_t)map * 2) * warps;
    nmap = map;
    if (num_smem + kStaticSmem <= (size_t)max_smem_optin()) break;
  }
  const size_t smem = sym_smem > num_smem ? sym_smem : num_smem;
  if (smem + kStaticSmem > (size_t)max_smem_optin()) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_factor_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int bps = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_factor_fused, kNumThreads, smem);
  if (bps < 1) return cudaErrorInvalidConfiguration;
  int grid = bps * num_sms();
  if (grid < 2) return cudaErrorInvalidConfiguration;
  // the symbolic walk runs ahead of the numeric one with far fewer warps
  const int part = !mapw ? kFusedSymPartList
                   : nnz_a >= kLongRowsOfA * n ? kFusedSymPartMapLongRows
                                                : kFusedSymPartMap;
  int g_sym = (int)((int64_t)grid * part / 16);
  if (g_sym < 1) g_sym = 1;
  if (g_sym > grid - 1) g_sym = grid - 1;
  const int64_t chunk = symbolic_chunk(k, scap);
  int64_t limit = wait_limit();
  int kk = k, sc = scap, mw = mapw, nc = ncap, nm = nmap, gs = g_sym;
  int64_t nn = n, acap = ar.cap, ch = chunk;
  void *args[] = {(void *)&nn, (void *)&arp, (void *)&aci, (void *)&aval, (void *)&kk,
                  (void *)&ar.col, (void *)&ar.lev, (void *)&arena_val, (void *)&acap,
                  (void *)&ar.top, (void *)&ar.row_off, (void *)&ar.row_len, (void *)&ar.row_ust,
                  (void *)&ar.meta, (void *)&rinfo, (void *)&ar.ticket, (void *)&num_ticket,
                  (void *)&err, (void *)&sc, (void *)&mw, (void *)&ch, (void *)&nc, (void *)&nm,
                  (void *)&gs, (void *)&limit, (void *)&v0, (void *)&xf, (void *)&rdiag,
                  (void *)&depth, (void *)&maxdepth};
  e = cudaLaunchCooperativeKernel((const void *)k_factor_fused, dim3((unsigned)grid),
                                  dim3(kNumThreads), args, smem, s);
  note_launch();
  return e;
}

cudaError_t launch_numeric(const iluk_sym *S, const double *aval, double *fval, DivPrep *rdiag,
                           unsigned long long *ticket, DevErr *err, int32_t *depth,
                           unsigned *maxdepth, cudaStream_t s) {
  return launch_numeric_impl(S, 1, aval, fval, rdiag, ticket, err, depth, maxdepth, s);
}

cudaError_t launch_numeric_batched(const iluk_sym *S, int64_t nbatch, const double *avals,
                                   double *fvals, unsigned long long *ticket, DevErr *errs,
                                   cudaStream_t s) {
  return launch_numeric_impl(S, nbatch, avals, fvals, nullptr, ticket, errs, nullptr, nullptr, s);
}

}  // namespace iluk
