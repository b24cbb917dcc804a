// symbolic_body.cuh -- the row walk of the symbolic ILU(k) phase (Algorithm 1,
// Sec. 2.2, with the level of Def. 2.3), shared by the symbolic kernel and the
// factorization kernel that runs the numeric phase beside it.  See
// symbolic.cu for the design.
#pragma once
#include <climits>

#include "internal.h"

namespace iluk {

constexpr int kSymThreads = 256;

// Hand-off between rows without fences.  The arena is filled with pending
// markers (column -1, level 255: levels never exceed k <= 250) before the
// launch, and each entry is written once, so a reader simply retries while it
// sees a marker.  A claimed row announces its arena slot in one 64-bit word
// (kMetaPending until then).  The slot holds the diagonal, the strictly upper
// part in ascending order, an entry with column kEndCol, then the strictly
// lower part: the diagonal is followed by the upper part, as in CSR.
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
// `slot` (the upper part begins one entry later) into (t, lt) and waits until every entry of this chunk up to the end
// marker is visible (entries past the marker are not waited for).  Returns how
// many entries of the chunk belong to the upper part (32 when the marker lies
// beyond the chunk), or -1 on time-out or an earlier row's failure.
__device__ __forceinline__ int load_upper_chunk(const int32_t *acol, const uint8_t *alev,
                                                int64_t arena_cap, int64_t slot, int b0,
                                                int lane, int &t, int &lt, const DevErr *err,
                                                int64_t row, int64_t limit_ns) {
  const int64_t a = slot + 1 + b0 + lane;
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

// PUBLISH: also announce each finished row's (length << 32 | upper start) in
// rinfo, for a numeric phase running beside this one.
template <bool INDEP, bool PUBLISH>
__device__ __forceinline__ void symbolic_rows_body(int64_t n, const int64_t *__restrict__ arp, const int32_t *__restrict__ aci,
                int k, int32_t *arena_col, uint8_t *arena_lev, int64_t arena_cap,
                unsigned long long *arena_top, int64_t *row_off, int32_t *row_len,
                int32_t *row_ust, unsigned long long *meta, unsigned long long *ticket, DevErr *err,
                int cap, int mapw, int64_t chunk, int64_t limit_ns,
                unsigned long long *rinfo, unsigned char *smem, bool rev = false) {
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
    const int64_t tkt = (int64_t)__shfl_sync(FULL_MASK, tk, 0);
    if (tkt >= n) return;
    // independent rows may go last row first (rev); waiting rows never do
    const int64_t row = (INDEP && rev) ? n - 1 - tkt : tkt;
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
    if (!has_diag) {  // no slot layout without a diagonal: the factorization fails here
      if (lane == 0) set_err(err, row, ILUK_ENODIAG);
      return;
    }
    const int ust = dpos + 1;

    // The slot: diagonal, upper part, end marker, then the strictly lower
    // part (m + 1 entries).  k <= 1 rows allocate theirs now.
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
      // q <= mu: the diagonal (q = 0) and the upper part, from position ust - 1
      // on; q = mu + 1: the end marker; then the lower part from position 0
      const int src = q <= mu ? ust - 1 + q : q - mu - 2;
      arena_col[slot + q] = q == mu + 1 ? kEndCol : cols[src];
      arena_lev[slot + q] = q == mu + 1 ? (uint8_t)0 : lev[src];
    }
    if (PUBLISH) {  // every lane's slot entries before the announcement below
      __threadfence();
      __syncwarp();
    }
    if (lane == 0) {
      row_off[row] = (int64_t)slot;
      row_len[row] = m;
      row_ust[row] = ust;
      if (PUBLISH) {
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(&rinfo[row]),
                     "l"(((unsigned long long)(unsigned)m << 32) | (unsigned)ust)
                     : "memory");
      }
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

}  // namespace iluk
