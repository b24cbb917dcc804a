// symbolic.cu -- a2: symbolic ILU(k) factorization (Algorithm 1, Sec. 2.2)
// with the level of fill of Def. 2.3, one warp per row.
//
// Row j's permitted set starts as A's row (level 0).  Its entries below the
// diagonal are walked in ascending order, including those inserted during
// the walk; for each such i with level(j,i) < k the warp waits for row i to be
// final, then merges row i's entries t > i: weight = level(j,i) + level(i,t)
// + 1, a min-update when t is present, an insertion when weight <= k.
// Entries with level(j,i) >= k, or with weight > k, cannot change anything
// and are skipped.  For k >= 2 the row is kept as a level map over a window
// of columns in shared memory (one byte per column plus presence and pivot
// bitmaps); a row that leaves the window, and every row of a matrix too wide
// for one, is kept as a sorted list with parallel insertion instead.
// Rows go to an arena carved into per-warp chunks (the device analogue of the
// paper's thread-private allocation arenas, Sec. 3.3).  A warp that claims a
// row fixes the row's slot at once (its chunk always has room for the longest
// row) and announces the slot; the finished row is written upper part first,
// closed by an end marker, so a row that needs it polls those entries
// directly, one round trip after they land.  Rows are compacted into CSR
// afterwards (Sec. 3.4).
//
// With k <= 1 rows are independent (Sec. 3.3: only level-0 entries can cause
// fill), so the warp reads the pivot rows straight from A and never waits.
#include <climits>

#include "internal.h"

namespace iluk {

constexpr int kSymThreads = 256;

// Hand-off between rows without fences.  The arena is filled with pending
// markers (column -1, level 255: levels never exceed k <= 250) before the
// launch, and each entry is written once, so a reader simply retries while it
// sees a marker.  A claimed row announces its arena slot in one 64-bit word
// (kMetaPending until then).  The slot holds the row's strictly upper part in
// ascending order, then an entry with column kEndCol, then the lower part and
// the diagonal.
constexpr unsigned long long kMetaPending = ~0ull;
constexpr int32_t kEndCol = INT_MAX;

__device__ __forceinline__ unsigned long long ld_meta(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ int32_t ld_col(const int32_t *p) {
  int32_t v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ int ld_lev(const uint8_t *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u8 %0, [%1];" : "=r"(v) : "l"(p));
  return (int)v;
}

// Warp-uniform poll of a row's announcement; false on time-out or when a
// row before `row` failed.
__device__ __forceinline__ bool wait_meta(const unsigned long long *p, unsigned long long *out,
                                          const DevErr *err, int64_t row, int64_t limit_ns) {
  unsigned long long v = ld_meta(p);
  if (__all_sync(FULL_MASK, v != kMetaPending)) {
    *out = __shfl_sync(FULL_MASK, v, 0);
    return true;
  }
  const uint64_t t0 = globaltimer_ns();
  unsigned backoff = 16;
  for (unsigned it = 0;; ++it) {
    v = ld_meta(p);
    if (__all_sync(FULL_MASK, v != kMetaPending)) {
      *out = __shfl_sync(FULL_MASK, v, 0);
      return true;
    }
    const bool stop = (it & 31u) == 31u &&
                      (earlier_failed(err, row) || (int64_t)(globaltimer_ns() - t0) > limit_ns);
    if (__any_sync(FULL_MASK, stop)) return false;
    if (it >= 4) {
      __nanosleep(backoff);
      if (backoff < 64u) backoff <<= 1;
    }
  }
}

// Loads entry b0 + lane of the upper part of the row whose slot starts at
// `slot` into (t, lt) and waits until every entry of this chunk up to the end
// marker is visible (entries past the marker are not waited for).  Returns how
// many entries of the chunk belong to the upper part (32 when the marker lies
// beyond the chunk), or -1 on time-out or an earlier row's failure.
__device__ __forceinline__ int load_upper_chunk(const int32_t *acol, const uint8_t *alev,
                                                int64_t arena_cap, int64_t slot, int b0,
                                                int lane, int &t, int &lt, const DevErr *err,
                                                int64_t row, int64_t limit_ns) {
  const int64_t a = slot + b0 + lane;
  const bool in = a < arena_cap;  // the row ends before the arena does
  t = kEndCol;
  lt = 0;
  if (in) {
    t = ld_col(&acol[a]);
    lt = ld_lev(&alev[a]);
  }
  bool pend = t < 0 || lt == 255;
  uint64_t t0 = 0;
  unsigned backoff = 16;
  for (unsigned it = 0;; ++it) {
    const unsigned endm = __ballot_sync(FULL_MASK, !pend && t == kEndCol);
    const unsigned pm = __ballot_sync(FULL_MASK, pend);
    const int e = endm ? __ffs(endm) - 1 : 32;  // first visible end marker
    const unsigned before = e >= 32 ? ~0u : ((1u << e) - 1u);
    if ((pm & before) == 0u) return e;
    if (it == 0) t0 = globaltimer_ns();
    const bool stop = (it & 31u) == 31u &&
                      (earlier_failed(err, row) || (int64_t)(globaltimer_ns() - t0) > limit_ns);
    if (__any_sync(FULL_MASK, stop)) return -1;
    if (it >= 4) {  // a row far from finishing: poll gently
      __nanosleep(backoff);
      if (backoff < 64u) backoff <<= 1;
    }
    if (pend) {
      t = ld_col(&acol[a]);
      lt = ld_lev(&alev[a]);
      pend = t < 0 || lt == 255;
    }
  }
}

// Level map of the row being built (k >= 2): one byte per column over a window
// that starts at the row's first column of A.  Every column of the final row
// lies at or above that column: a fill column t comes from the upper part of
// a pivot i that is itself a column of the row, so t > i >= the first column.
// Only the upper end can leave the window; a row that does falls back to the
// sorted list.
// The window width (a power of two, mapw columns) is chosen per call from the
// widest row of A: twice its span, at most kMaxMapCols; 0 selects the list.
// The cap is also an occupancy choice: rows are claimed in index order before
// any level information exists, so a matrix with wide wavefronts (a 3D grid)
// needs many warps in flight, which larger maps would crowd out.
constexpr int kMaxMapCols = 8192;

size_t symbolic_smem_per_warp(int cap) { return (size_t)cap * 5; }
// per warp: the level bytes, then a presence bitmap and a pivot bitmap (level < k)
size_t symbolic_map_per_warp(int mapw) { return (size_t)mapw + (size_t)mapw / 4; }

// Window for the level map: twice the widest column span of a row of A,
// rounded up to a power of two (at least 1024); 0 when that exceeds
// kMaxMapCols.  Synchronous.
__global__ void k_row_span(int64_t n, const int64_t *__restrict__ arp,
                           const int32_t *__restrict__ aci, int32_t *span) {
  int32_t mx = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (arp[i + 1] > arp[i]) {
      const int32_t w = aci[arp[i + 1] - 1] - aci[arp[i]] + 1;
      if (w > mx) mx = w;
    }
  mx = __reduce_max_sync(FULL_MASK, mx);
  if ((threadIdx.x & 31) == 0 && mx > 0) atomicMax(span, mx);
}

int symbolic_map_width(int64_t n, const int64_t *arp, const int32_t *aci, int k,
                       cudaStream_t s) {
  if (k < 2 || n == 0) return 0;
  int32_t *d = nullptr;
  if (cudaMallocAsync((void **)&d, sizeof(int32_t), s) != cudaSuccess) return 0;
  int32_t span = 0;
  cudaMemsetAsync(d, 0, sizeof(int32_t), s);
  int64_t b = (n + 255) / 256;
  if (b > (int64_t)num_sms() * 8) b = (int64_t)num_sms() * 8;
  k_row_span<<<(unsigned)b, 256, 0, s>>>(n, arp, aci, d);
  note_launch();
  cudaMemcpyAsync(&span, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return 0;
  int64_t w = 1024;
  while (w < 2 * (int64_t)span) w <<= 1;
  return w <= kMaxMapCols ? (int)w : 0;
}

template <bool INDEP>
__global__ void __launch_bounds__(kSymThreads)
k_symbolic_rows(int64_t n, const int64_t *__restrict__ arp, const int32_t *__restrict__ aci,
                int k, int32_t *arena_col, uint8_t *arena_lev, int64_t arena_cap,
                unsigned long long *arena_top, int64_t *row_off, int32_t *row_len,
                int32_t *row_ust, unsigned long long *meta, unsigned long long *ticket, DevErr *err,
                int cap, int mapw, int64_t chunk, int64_t limit_ns) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  int32_t *cols = reinterpret_cast<int32_t *>(smem) + (size_t)wib * cap;
  uint8_t *lev = smem + (size_t)nwarps * cap * 4 + (size_t)wib * cap;
  uint8_t *map = mapw ? smem + (size_t)nwarps * cap * 5 + (size_t)wib * (mapw + mapw / 4)
                      : nullptr;
  uint32_t *pres = mapw ? reinterpret_cast<uint32_t *>(map + mapw) : nullptr;
  uint32_t *piv = mapw ? pres + mapw / 32 : nullptr;
  // this warp's arena chunk [ch_off, ch_end) (warp-uniform)
  unsigned long long ch_off = 0, ch_end = 0;

  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(ticket, 1ull);
    const int64_t row = (int64_t)__shfl_sync(FULL_MASK, tk, 0);
    if (row >= n) return;
    if (earlier_failed(err, row)) return;

    // The row's slot: k >= 2 rows announce it now; the warp's chunk always
    // has room for cap + 1 entries here.
    unsigned long long slot = 0;
    if (!INDEP && chunk > 0) {
      if (ch_end - ch_off < (unsigned long long)cap + 1) {  // first row of the warp
        unsigned long long c0 = 0;
        if (lane == 0) c0 = atomicAdd(arena_top, (unsigned long long)chunk);
        ch_off = __shfl_sync(FULL_MASK, c0, 0);
        ch_end = ch_off + (unsigned long long)chunk;
      }
      slot = ch_off;
      if (lane == 0)
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(&meta[row]), "l"(slot) : "memory");
    }
    const int64_t a0 = arp[row], a1 = arp[row + 1];
    int m = (int)(a1 - a0);
    if (a1 - a0 > cap) {
      if (lane == 0) {
        set_err(err, row, ILUK_ENOMEM);
        atomicMax(&err->need, (unsigned long long)(a1 - a0));
      }
      return;
    }
    for (int q = lane; q < m; q += 32) {
      cols[q] = aci[a0 + q];
      lev[q] = 0;
    }
    __syncwarp();

    bool ok = true;
    bool built = false;  // row finished by the level map (k >= 2)
    if (!INDEP && mapw) {
      // Level-map form of the same walk: map[c - base] = level of column c,
      // valid where the presence bit is set; a second bitmap marks possible
      // pivots (level < k).  A candidate is one min-update, the next pivot a
      // scan of 32 bitmap words at a time, the finished row a popcount
      // compaction.  The result is the sorted-list walk's: candidates are
      // distinct columns, each changes only its own entry, and pivots are
      // still taken in ascending order, inserted ones included.
      const int32_t base = cols[0];
      int hi = cols[m - 1] - base;  // highest occupied offset
      bool fits = hi < mapw;
      if (fits) {
        for (int w = lane; w < mapw / 32; w += 32) {
          pres[w] = 0u;
          piv[w] = 0u;
        }
        __syncwarp();
        for (int q = lane; q < m; q += 32) {  // A's entries: level 0 < k
          const int d = cols[q] - base;
          map[d] = 0;
          atomicOr(&pres[d >> 5], 1u << (d & 31));
          atomicOr(&piv[d >> 5], 1u << (d & 31));
        }
        __syncwarp();
        const int jlim = (int)(row - base);  // pivots lie at offsets below the diagonal
        const int jw = (jlim + 31) >> 5;     // bitmap words holding such offsets
        int cur = -1;
        // the slot of the pivot expected next, loaded one pivot ahead (a fill
        // inserted in between only wastes the load)
        int pf_i = -1;
        unsigned long long pf_slot = kMetaPending;
        for (;;) {
          int nxt = -1, nxt2 = -1;
          const int from = cur + 1;
          for (int w0 = from >> 5; w0 < jw; w0 += 32) {
            const int wi = w0 + lane;
            uint32_t bits = 0u;
            if (wi < jw) {
              bits = piv[wi];
              if (wi == (from >> 5)) bits &= ~0u << (from & 31);
              const int room = jlim - wi * 32;  // offsets at or beyond jlim are not pivots
              if (room < 32) bits &= (1u << room) - 1u;
            }
            const unsigned b = __ballot_sync(FULL_MASK, bits != 0u);
            if (b) {
              const int l = __ffs(b) - 1;
              const uint32_t wb = __shfl_sync(FULL_MASK, bits, l);
              nxt = (w0 + l) * 32 + __ffs(wb) - 1;
              // and the pivot after it, if this window shows it
              const uint32_t wb2 = wb & (wb - 1u);
              const unsigned b2 = b & ~((2u << l) - 1u);
              if (wb2) {
                nxt2 = (w0 + l) * 32 + __ffs(wb2) - 1;
              } else if (b2) {
                const int l2 = __ffs(b2) - 1;
                nxt2 = (w0 + l2) * 32 + __ffs(__shfl_sync(FULL_MASK, bits, l2)) - 1;
              }
              break;
            }
          }
          if (nxt < 0) break;
          cur = nxt;
          const int i = base + nxt;
          const int lji = map[nxt];
          unsigned long long islot = 0;
          if (pf_i == i && __all_sync(FULL_MASK, pf_slot != kMetaPending)) {
            islot = pf_slot;
          } else if (!wait_meta(&meta[i], &islot, err, row, limit_ns)) {
            if (lane == 0 && !earlier_failed(err, row)) set_err(err, row, ILUK_ETIMEOUT);
            ok = false;
            break;
          }
          pf_i = nxt2 >= 0 ? base + nxt2 : -1;
          pf_slot = nxt2 >= 0 ? ld_meta(&meta[pf_i]) : kMetaPending;
          const int limit = k - 1 - lji;
          for (int b0 = 0;; b0 += 32) {
            int t, lt;
            const int cnt = load_upper_chunk(arena_col, arena_lev, arena_cap, (int64_t)islot, b0,
                                             lane, t, lt, err, row, limit_ns);
            if (cnt < 0) {
              if (lane == 0 && !earlier_failed(err, row)) set_err(err, row, ILUK_ETIMEOUT);
              ok = false;
              break;
            }
            if (lane < cnt && lt <= limit) {
              const int d = t - base;
              if (d >= mapw) {
                fits = false;
              } else {
                const int w = lji + lt + 1;  // <= k
                const uint32_t bit = 1u << (d & 31);
                if (!(pres[d >> 5] & bit)) {  // insertion
                  map[d] = (uint8_t)w;
                  atomicOr(&pres[d >> 5], bit);
                  if (w < k) atomicOr(&piv[d >> 5], bit);
                  if (d > hi) hi = d;
                } else if (w < (int)map[d]) {  // lower level
                  if ((int)map[d] >= k && w < k) atomicOr(&piv[d >> 5], bit);
                  map[d] = (uint8_t)w;
                }
              }
            }
            __syncwarp();
            if (cnt < 32) break;
          }
          if (!ok) break;
          if (!__all_sync(FULL_MASK, fits)) {
            fits = false;
            break;
          }
        }
        if (!ok) return;
      }
      if (fits) {
        hi = __reduce_max_sync(FULL_MASK, hi);
        const int nw = (hi >> 5) + 1;
        int mm = 0;
        for (int w0 = 0; w0 < nw; w0 += 32) {
          const int wi = w0 + lane;
          uint32_t bits = wi < nw ? pres[wi] : 0u;
          const int c = __popc(bits);
          int incl = c;  // inclusive prefix of the counts over the lanes
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += y;
          }
          int pos = mm + incl - c;
          while (bits) {
            const int d = wi * 32 + __ffs(bits) - 1;
            bits &= bits - 1u;
            if (pos < cap) {
              cols[pos] = base + d;
              lev[pos] = map[d];
            }
            ++pos;
          }
          mm += __shfl_sync(FULL_MASK, incl, 31);
        }
        if (mm > cap) {
          if (lane == 0) {
            set_err(err, row, ILUK_ENOMEM);
            atomicMax(&err->need, (unsigned long long)mm);
          }
          return;
        }
        m = mm;
        built = true;
        __syncwarp();
      }
      // else: the row left the window; cols/lev still hold A's row
    }

    for (int p = 0; p < m && !built; ++p) {
      const int i = cols[p];
      if (i >= row) break;
      const int lji = lev[p];
      if (lji >= k) continue;  // weight would exceed k for every t
      // row i's upper part: from A (k <= 1), else from row i's arena slot,
      // a chunk of 32 at a time up to its end marker
      const int32_t *ucol = nullptr;
      int ulen = INT_MAX;
      unsigned long long islot = 0;
      if (INDEP) {
        const int64_t b0 = arp[i], b1 = arp[i + 1];
        const int64_t s = lower_bound_l(aci, b0, b1, (int32_t)(i + 1));
        ucol = aci + s;
        ulen = (int)(b1 - s);
      } else if (!wait_meta(&meta[i], &islot, err, row, limit_ns)) {
        if (lane == 0 && !earlier_failed(err, row)) set_err(err, row, ILUK_ETIMEOUT);
        ok = false;
        break;
      }
      const int limit = k - 1 - lji;  // level(i,t) must not exceed this
      for (int base = 0; base < ulen; base += 32) {
        const int q = base + lane;
        int t = INT_MAX, lt = 255;
        int cnt = 32;  // entries of this chunk in row i's upper part
        if (INDEP) {
          if (q < ulen) {
            t = ucol[q];
            lt = 0;
          }
          cnt = ulen - base < 32 ? ulen - base : 32;
        } else {
          cnt = load_upper_chunk(arena_col, arena_lev, arena_cap, (int64_t)islot, base, lane, t,
                                 lt, err, row, limit_ns);
          if (cnt < 0) {
            if (lane == 0 && !earlier_failed(err, row)) set_err(err, row, ILUK_ETIMEOUT);
            ok = false;
            break;
          }
          if (cnt < 32) ulen = base + cnt;  // the last chunk
        }
        const bool cand = lane < cnt && lt <= limit;
        const int w = lji + lt + 1;
        int pos = 0;
        bool found = false;
        if (cand) {
          pos = lower_bound_i(cols, p + 1, m, (int32_t)t);
          found = pos < m && cols[pos] == t;
          if (found && w < (int)lev[pos]) lev[pos] = (uint8_t)w;
        }
        const bool ins = cand && !found;
        const unsigned insmask = __ballot_sync(FULL_MASK, ins);
        __syncwarp();
        if (insmask) {
          const int c = __popc(insmask);
          if (m + c > cap) {
            if (lane == 0) {
              set_err(err, row, ILUK_ENOMEM);
              atomicMax(&err->need, (unsigned long long)(m + c));
            }
            ok = false;
            break;
          }
          const int lb = ins ? pos : INT_MAX;
          const int lbmin = __reduce_min_sync(FULL_MASK, lb);
          // Shift the tail [lbmin, m) up, top chunk first, so that every
          // element moves past the insertions that precede it.
          for (int top = m - 1; top >= lbmin; top -= 32) {
            const int q2 = top - lane;
            const bool act = q2 >= lbmin;
            int32_t cv = 0;
            uint8_t lv = 0;
            if (act) {
              cv = cols[q2];
              lv = lev[q2];
            }
            int sh = 0;
#pragma unroll
            for (int r = 0; r < 32; ++r) sh += (__shfl_sync(FULL_MASK, lb, r) <= q2) ? 1 : 0;
            __syncwarp();
            if (act) {
              cols[q2 + sh] = cv;
              lev[q2 + sh] = lv;
            }
            __syncwarp();
          }
          if (ins) {
            const int rank = __popc(insmask & ((1u << lane) - 1u));
            cols[pos + rank] = t;
            lev[pos + rank] = (uint8_t)w;
          }
          m += c;
          __syncwarp();
        }
      }
      if (!ok) break;
    }
    if (!ok) return;

    // Row final.  Upper part starts at the first column > row.
    const int dpos = lower_bound_i(cols, 0, m, (int32_t)row);
    const bool has_diag = dpos < m && cols[dpos] == row;
    const int ust = has_diag ? dpos + 1 : dpos;
    if (!has_diag && lane == 0) set_err(err, row, ILUK_ENODIAG);

    // The slot: upper part, end marker, then lower part and diagonal (m + 1
    // entries).  k <= 1 rows allocate theirs now.
    const int mu = m - ust;
    if (INDEP || chunk == 0) {
      unsigned long long c0 = 0;
      if (lane == 0) c0 = atomicAdd(arena_top, (unsigned long long)(m + 1));
      slot = __shfl_sync(FULL_MASK, c0, 0);
    } else {
      ch_off = slot + (unsigned long long)(m + 1);
    }
    if ((int64_t)(slot + m + 1) > arena_cap) {
      if (lane == 0) set_err(err, row, ILUK_ENOMEM);
      return;
    }
    for (int q = lane; q <= m; q += 32) {
      const int src = q < mu ? ust + q : q - mu - 1;  // q == mu: the end marker
      arena_col[slot + q] = q == mu ? kEndCol : cols[src];
      arena_lev[slot + q] = q == mu ? (uint8_t)0 : lev[src];
    }
    if (lane == 0) {
      row_off[row] = (int64_t)slot;
      row_len[row] = m;
      row_ust[row] = ust;
    }
    // the next chunk, now that the row is written, if this one cannot take
    // the longest row
    if (!INDEP && chunk > 0 && ch_end - ch_off < (unsigned long long)cap + 1) {
      unsigned long long c0 = 0;
      if (lane == 0) c0 = atomicAdd(arena_top, (unsigned long long)chunk);
      ch_off = __shfl_sync(FULL_MASK, c0, 0);
      ch_end = ch_off + (unsigned long long)chunk;
    }
    __syncwarp();
  }
}

// Chunk size: room for four of the longest rows (with their end markers); a
// warp renews its chunk after a row whenever the longest row would no longer
// fit, so every claimed row has its slot at once.  Rows that never wait on
// other rows (k <= 1) allocate per row.
int64_t symbolic_chunk(int k, int cap) { return k <= 1 ? 0 : 4 * ((int64_t)cap + 1); }

// Warps per CTA and CTAs of the symbolic launch for this row capacity and map.
static cudaError_t symbolic_shape(int k, int cap, int mapw, int *warps_out, size_t *smem_out,
                                  int *blocks_per_sm_out) {
  if (k < 2) mapw = 0;
  const size_t per_warp = symbolic_smem_per_warp(cap) + symbolic_map_per_warp(mapw);
  int warps = kSymThreads / 32;
  while (warps > 1 && per_warp * warps > (size_t)max_smem_optin()) warps >>= 1;
  const size_t smem = per_warp * warps;
  int bps = 0;
  cudaError_t e;
  if (k <= 1) {
    e = cudaFuncSetAttribute(k_symbolic_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e == cudaSuccess)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_symbolic_rows<true>, warps * 32, smem);
  } else {
    e = cudaFuncSetAttribute(k_symbolic_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e == cudaSuccess)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_symbolic_rows<false>, warps * 32,
                                                    smem);
  }
  *warps_out = warps;
  *smem_out = smem;
  *blocks_per_sm_out = bps < 1 ? 1 : bps;
  return e;
}

// Arena entries the chunked allocation may leave unused, beyond the rows
// themselves: every warp's open chunk, plus what chunk changes leave behind
// (at most cap entries of each chunk of 4 (cap + 1): a third of what the
// chunk held), given an estimate `rows_est` of the rows' entries.  The end
// markers (one per row) come on top.
int64_t symbolic_arena_slack(int64_t n, int k, int cap, int mapw, int64_t rows_est) {
  if (k <= 1) return n;  // per-row allocation: only the end markers
  int warps, bps;
  size_t smem;
  if (symbolic_shape(k, cap, mapw, &warps, &smem, &bps) != cudaSuccess) return 0;
  int64_t grid = (int64_t)bps * num_sms();
  const int64_t want = (n + warps - 1) / warps;
  if (grid > want) grid = want;
  return grid * warps * symbolic_chunk(k, cap) + rows_est / 3 + n;
}

cudaError_t launch_symbolic_rows(int64_t n, const int64_t *arp, const int32_t *aci, int k,
                                 const SymArena &ar, DevErr *err, int cap, int mapw,
                                 cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_SYMBOLIC, s);
  if (k < 2) mapw = 0;
  int warps, blocks_per_sm;
  size_t smem;
  cudaError_t e = symbolic_shape(k, cap, mapw, &warps, &smem, &blocks_per_sm);
  if (e != cudaSuccess) return e;
  const int threads = warps * 32;
  const bool indep = k <= 1;
  const int64_t chunk = symbolic_chunk(k, cap);
  int64_t want = (n + warps - 1) / warps;
  int64_t grid = (int64_t)blocks_per_sm * num_sms();
  if (grid > want) grid = want;
  if (grid < 1) grid = 1;
  if (indep)
    k_symbolic_rows<true><<<(unsigned)grid, threads, smem, s>>>(
        n, arp, aci, k, ar.col, ar.lev, ar.cap, ar.top, ar.row_off, ar.row_len, ar.row_ust,
        ar.meta, ar.ticket, err, cap, mapw, chunk, wait_limit());
  else
    k_symbolic_rows<false><<<(unsigned)grid, threads, smem, s>>>(
        n, arp, aci, k, ar.col, ar.lev, ar.cap, ar.top, ar.row_off, ar.row_len, ar.row_ust,
        ar.meta, ar.ticket, err, cap, mapw, chunk, wait_limit());
  note_launch();
  return cudaGetLastError();
}

// Copy every row from the arena into CSR order; record the diagonal position
// and the longest row.
__global__ void k_symbolic_compact(int64_t n, const int32_t *__restrict__ acol,
                                   const uint8_t *__restrict__ alev,
                                   const int64_t *__restrict__ row_off,
                                   const int32_t *__restrict__ row_len,
                                   const int32_t *__restrict__ row_ust,
                                   const int64_t *__restrict__ frp, int32_t *fci, uint8_t *flev,
                                   int64_t *fdiag, int32_t *maxrow) {
  const int lane = threadIdx.x & 31;
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < n; row += nw) {
    // the slot holds the upper part, an end marker, then the lower part and
    // the diagonal; CSR wants lower, diagonal, upper
    const int64_t off = row_off[row], dst = frp[row];
    const int len = row_len[row], ust = row_ust[row], mu = len - ust;
    for (int q = lane; q < len; q += 32) {
      const int64_t src = q < ust ? off + mu + 1 + q : off + (q - ust);
      fci[dst + q] = acol[src];
      flev[dst + q] = alev[src];
    }
    if (lane == 0) {
      fdiag[row] = dst + ust - 1;
      atomicMax(maxrow, len);
    }
  }
}

cudaError_t launch_symbolic_compact(int64_t n, const SymArena &ar, const int64_t *frp,
                                    int32_t *fci, uint8_t *flev, int64_t *fdiag, int32_t *maxrow,
                                    cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_COMPACT, s);
  int64_t blocks = (n * 32 + 255) / 256;
  int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_symbolic_compact<<<(unsigned)blocks, 256, 0, s>>>(n, ar.col, ar.lev, ar.row_off, ar.row_len,
                                                       ar.row_ust, frp, fci, flev, fdiag, maxrow);
  note_launch();
  return cudaGetLastError();
}

// a2f[p] = offset of A's entry p inside its F row (A's pattern is a subset).
__global__ void k_a2f(int64_t n, const int64_t *__restrict__ arp, const int32_t *__restrict__ aci,
                      const int64_t *__restrict__ frp, const int32_t *__restrict__ fci,
                      int32_t *a2f) {
  const int lane = threadIdx.x & 31;
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < n; row += nw) {
    const int64_t f0 = frp[row], f1 = frp[row + 1];
    for (int64_t p = arp[row] + lane; p < arp[row + 1]; p += 32) {
      const int64_t pos = lower_bound_l(fci, f0, f1, aci[p]);
      a2f[p] = (int32_t)(pos - f0);
    }
  }
}

cudaError_t launch_a2f(int64_t n, const int64_t *arp, const int32_t *aci, const int64_t *frp,
                       const int32_t *fci, int32_t *a2f, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_COMPACT, s);
  int64_t blocks = (n * 32 + 255) / 256;
  int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_a2f<<<(unsigned)blocks, 256, 0, s>>>(n, arp, aci, frp, fci, a2f);
  note_launch();
  return cudaGetLastError();
}

}  // namespace iluk
