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
// row) and announces the slot; the finished row is written diagonal and upper
// part first, closed by an end marker, so a row that needs it polls those
// entries directly, one round trip after they land.  Rows are compacted into CSR
// afterwards (Sec. 3.4).
//
// With k <= 1 rows are independent (Sec. 3.3: only level-0 entries can cause
// fill), so the warp reads the pivot rows straight from A and never waits;
// rows are claimed in ascending order, or last row first (the order Sec. 3.3
// found fastest on a CPU), or they take the general walk with waits
// (iluk_set_symbolic_variant, a study of the three: the results are the
// same).
#include "symbolic_body.cuh"

namespace iluk {

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
                int cap, int mapw, int64_t chunk, int64_t limit_ns, int rev) {
  extern __shared__ __align__(16) unsigned char smem[];
  symbolic_rows_body<INDEP, false>(n, arp, aci, k, arena_col, arena_lev, arena_cap, arena_top, row_off,
                            row_len, row_ust, meta, ticket, err, cap, mapw, chunk, limit_ns,
                            nullptr, smem, rev != 0);
}

// Chunk size: room for four of the longest rows (with their end markers); a
// warp renews its chunk after a row whenever the longest row would no longer
// fit, so every claimed row has its slot at once.  Rows that never wait on
// other rows (k <= 1) allocate per row.
int64_t symbolic_chunk(int k, int cap) { return symbolic_indep(k) ? 0 : 4 * ((int64_t)cap + 1); }

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
  if (symbolic_indep(k)) {
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
  if (symbolic_indep(k)) return n;  // per-row allocation: only the end markers
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
  const bool indep = symbolic_indep(k);
  const int rev = indep && symbolic_variant() == 1;  // independent rows, last row first
  const int64_t chunk = symbolic_chunk(k, cap);
  int64_t want = (n + warps - 1) / warps;
  int64_t grid = (int64_t)blocks_per_sm * num_sms();
  if (grid > want) grid = want;
  if (grid < 1) grid = 1;
  if (indep)
    k_symbolic_rows<true><<<(unsigned)grid, threads, smem, s>>>(
        n, arp, aci, k, ar.col, ar.lev, ar.cap, ar.top, ar.row_off, ar.row_len, ar.row_ust,
        ar.meta, ar.ticket, err, cap, mapw, chunk, wait_limit(), rev);
  else
    k_symbolic_rows<false><<<(unsigned)grid, threads, smem, s>>>(
        n, arp, aci, k, ar.col, ar.lev, ar.cap, ar.top, ar.row_off, ar.row_len, ar.row_ust,
        ar.meta, ar.ticket, err, cap, mapw, chunk, wait_limit(), 0);
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
    // the slot holds the diagonal, the upper part, an end marker, then the
    // lower part; CSR wants lower, diagonal, upper
    const int64_t off = row_off[row], dst = frp[row];
    const int len = row_len[row], ust = row_ust[row], mu = len - ust;
    for (int q = lane; q < len; q += 32) {
      const int64_t src = q < ust - 1 ? off + mu + 2 + q : off + (q - (ust - 1));
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

// The values of a factorization kept in a value arena laid out like the
// column arena (diagonal, upper part, end marker, lower part per slot), in CSR
// order.
__global__ void k_compact_values(int64_t n, const double *__restrict__ aval,
                                 const int64_t *__restrict__ row_off,
                                 const int32_t *__restrict__ row_len,
                                 const int32_t *__restrict__ row_ust,
                                 const int64_t *__restrict__ frp, double *fval) {
  const int lane = threadIdx.x & 31;
  int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < n; row += nw) {
    const int64_t off = row_off[row], dst = frp[row];
    const int len = row_len[row], ust = row_ust[row], mu = len - ust;
    for (int q = lane; q < len; q += 32) {
      const int64_t src = q < ust - 1 ? off + mu + 2 + q : off + (q - (ust - 1));
      fval[dst + q] = aval[src];
    }
  }
}

cudaError_t launch_compact_values(int64_t n, const SymArena &ar, const double *aval,
                                  const int64_t *frp, double *fval, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_COMPACT, s);
  int64_t blocks = (n * 32 + 255) / 256;
  int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_compact_values<<<(unsigned)blocks, 256, 0, s>>>(n, aval, ar.row_off, ar.row_len, ar.row_ust,
                                                     frp, fval);
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
