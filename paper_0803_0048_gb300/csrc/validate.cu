// validate.cu -- a1 pattern check (CSR storage of Sec. 2.1) and the
// row-length scan used to turn per-row lengths into CSR row pointers.
#include "internal.h"

namespace iluk {

// One thread per row: rowptr monotone, columns in range and strictly
// ascending.  The smallest failing row wins (atomicMin on the error key).
__global__ void k_validate(int64_t n, int64_t nnz, const int64_t *__restrict__ rp,
                           const int32_t *__restrict__ ci, DevErr *err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && (rp[0] != 0 || rp[n] != nnz)) set_err(err, 0, ILUK_EPATTERN);
  if (i >= n) return;
  int64_t b = rp[i], e = rp[i + 1];
  if (e < b || b < 0 || e > nnz) { set_err(err, i, ILUK_EPATTERN); return; }
  int32_t prev = -1;
  for (int64_t p = b; p < e; ++p) {
    int32_t c = ci[p];
    if (c <= prev || c >= n) { set_err(err, i, ILUK_EPATTERN); return; }
    prev = c;
  }
}

cudaError_t launch_validate(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *ci,
                            DevErr *err, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_VALIDATE, s);
  int64_t blocks = (n + 255) / 256;
  if (blocks == 0) blocks = 1;
  k_validate<<<(unsigned)blocks, 256, 0, s>>>(n, nnz, rp, ci, err);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_fill_err(DevErr *err) {
  err->key = kNoErr;
  err->need = 0;
}

cudaError_t launch_fill_err(DevErr *err, cudaStream_t s) {
  k_fill_err<<<1, 1, 0, s>>>(err);
  note_launch();
  return cudaGetLastError();
}

// Exclusive scan of int32 lengths into int64 offsets, three passes:
// per-block sums, a scan of the block sums by one block, then per-block
// scans plus the block offset.
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t *sh) {
  // Hillis-Steele over the block in shared memory.
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int off = 1; off < blockDim.x; off <<= 1) {
    int64_t add = (t >= off) ? sh[t - off] : 0;
    __syncthreads();
    sh[t] += add;
    __syncthreads();
  }
  int64_t r = sh[t];
  __syncthreads();
  return r;
}

__global__ void k_scan_block_sums(int64_t n, const int32_t *__restrict__ len, int64_t *bsum) {
  __shared__ int64_t sh[kScanThreads];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v = 0;
  for (int q = 0; q < kScanItems; ++q)
    if (base + q < n) v += len[base + q];
  int64_t incl = block_incl_scan(v, sh);
  if (threadIdx.x == blockDim.x - 1) bsum[blockIdx.x] = incl;
}

__global__ void k_scan_top(int64_t nb, int64_t *bsum) {
  __shared__ int64_t sh[kScanThreads];
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int64_t v = (i < nb) ? bsum[i] : 0;
    int64_t incl = block_incl_scan(v, sh);
    if (i < nb) bsum[i] = carry + incl - v;  // exclusive
    int64_t tot = sh[blockDim.x - 1];  // inclusive total of this chunk
    __syncthreads();                   // before the next chunk rewrites sh
    carry += tot;
  }
}

__global__ void k_scan_apply(int64_t n, const int32_t *__restrict__ len,
                             const int64_t *__restrict__ bsum, int64_t *out) {
  __shared__ int64_t sh[kScanThreads];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t tot = 0;
  for (int q = 0; q < kScanItems; ++q) {
    v[q] = (base + q < n) ? len[base + q] : 0;
    tot += v[q];
  }
  int64_t incl = block_incl_scan(tot, sh);
  int64_t run = bsum[blockIdx.x] + incl - tot;
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
  for (int q = 0; q < kScanItems; ++q) {
    run += v[q];
    if (base + q < n) out[base + q + 1] = run;
  }
}

int64_t scan_tmp_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t launch_scan_lengths(int64_t n, const int32_t *len, int64_t *out, int64_t *tmp,
                                cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_COMPACT, s);
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 0) {
    return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
  }
  k_scan_block_sums<<<(unsigned)nb, kScanThreads, 0, s>>>(n, len, tmp);
  note_launch();
  k_scan_top<<<1, kScanThreads, 0, s>>>(nb, tmp);
  note_launch();
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(n, len, tmp, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace iluk
