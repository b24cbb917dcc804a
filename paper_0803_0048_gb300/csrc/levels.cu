// levels.cu -- level sets of the two sweep DAGs (the level/backward
// scheduling of the paper's related work: Anderson 1988, Heroux 1991).
//
// depth(i) = 1 + max depth(h) over the rows h that row i reads (h < i in the
// forward sweep, h > i in the backward sweep); rows of equal depth are
// independent.  The sweeps walk rows in level order, with every level
// starting on a warp boundary (short levels are padded with -1), so the 32
// rows of a warp never depend on one another: a warp's lanes only ever wait
// for rows held by other warps.
#include "internal.h"

namespace iluk {

constexpr int kDepthThreads = 512;

// One warp per row, rows claimed in sweep order through a global ticket per
// direction; depth[] doubles as the ready flag (0 until the row is final),
// handed over through L2.  A warp claims a row only while it runs, and every
// row it reads holds an earlier ticket, so the waits end whether or not all
// CTAs are resident: the launch can share the GPU with the numeric phase, and
// wide DAGs (thousands of rows per level) get thousands of warps.
template <bool FORWARD>
__device__ void depth_rows(int64_t n, const int64_t *__restrict__ rp,
                           const int32_t *__restrict__ ci, const int64_t *__restrict__ dg,
                           int32_t *depth, int32_t *maxdepth, DevErr *err, int64_t limit_ns,
                           unsigned long long *ticket, int *fail) {
  const int lane = threadIdx.x & 31;
  int dmax_local = 0;
  for (;;) {
    unsigned long long tk = 0;
    if (lane == 0) tk = atomicAdd(ticket, 1ull);
    const int64_t t = (int64_t)__shfl_sync(FULL_MASK, tk, 0);
    if (t >= n) break;
    const int64_t row = FORWARD ? t : n - 1 - t;
    const int64_t d = dg[row];
    const int64_t b0 = FORWARD ? rp[row] : d + 1;
    const int64_t b1 = FORWARD ? d : rp[row + 1];
    int dm = 0;
    bool ok = true;
    for (int64_t base = b0; base < b1; base += 32) {
      const int64_t q = base + lane;
      int v = 1;
      const int32_t *src = nullptr;
      if (q < b1) {
        src = &depth[ci[q]];
        asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(src));
      }
      if (__any_sync(FULL_MASK, v == 0)) {
        const uint64_t t0 = globaltimer_ns();
        unsigned backoff = 16;
        for (unsigned it = 0; __any_sync(FULL_MASK, v == 0); ++it) {
          if (v == 0) asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(src));
          const bool stop = (it & 15u) == 15u &&
                            (*((volatile int *)fail) || (int64_t)(globaltimer_ns() - t0) > limit_ns);
          if (__any_sync(FULL_MASK, stop)) {  // the whole warp gives up together
            ok = false;
            break;
          }
          if (it >= 4) {
            __nanosleep(backoff);
            if (backoff < 64u) backoff <<= 1;
          }
        }
      }
      if (!__all_sync(FULL_MASK, ok)) break;
      if (q < b1 && v > dm) dm = v;
    }
    if (!__all_sync(FULL_MASK, ok)) {
      if (lane == 0) {
        atomicExch(fail, 1);
        set_err(err, t, ILUK_ETIMEOUT);
      }
      return;
    }
    dm = __reduce_max_sync(FULL_MASK, dm) + 1;
    if (lane == 0) {
      asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(&depth[row]), "r"(dm) : "memory");
      if (dm > dmax_local) dmax_local = dm;
    }
  }
  if (lane == 0 && dmax_local) atomicMax(maxdepth, dmax_local);
}

// Even CTAs compute the forward depths, odd CTAs the backward depths (the two
// DAGs are independent).  ctl: two tickets, then two failure flags.
__global__ void __launch_bounds__(kDepthThreads)
k_depth_pair(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
             const int64_t *__restrict__ dg, int32_t *depth_f, int32_t *depth_b, int32_t *mx,
             DevErr *err, unsigned long long *ctl, int64_t limit_ns) {
  int *fail = reinterpret_cast<int *>(ctl + 2);
  if ((blockIdx.x & 1) == 0)
    depth_rows<true>(n, rp, ci, dg, depth_f, mx, err, limit_ns, ctl, fail);
  else
    depth_rows<false>(n, rp, ci, dg, depth_b, mx + 1, err + 1, limit_ns, ctl + 1, fail + 1);
}

__global__ void k_level_count(int64_t n, const int32_t *__restrict__ depth, int32_t *cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[depth[i] - 1], 1);
}

__global__ void k_level_pad(int64_t nlev, int32_t *cnt) {
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nlev;
       l += (int64_t)gridDim.x * blockDim.x)
    cnt[l] = (cnt[l] + 31) & ~31;
}

__global__ void k_level_scatter(int64_t n, const int32_t *__restrict__ depth,
                                const int64_t *__restrict__ lstart, int32_t *cursor,
                                int32_t *order) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int l = depth[i] - 1;
    order[lstart[l] + atomicAdd(&cursor[l], 1)] = (int32_t)i;
  }
}

static unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

// Padded level order from depths, and the same order without padding
// (synchronous).
static int order_from_depth(int64_t n, const int32_t *depth, int32_t nlev, LevelOrder *lo,
                            cudaStream_t s) {
  int32_t *cnt = nullptr, *cursor = nullptr;
  int64_t *lstart = nullptr, *scan_tmp = nullptr, *cstart = nullptr;
  auto cleanup = [&]() {
    if (cnt) cudaFreeAsync(cnt, s);
    if (cursor) cudaFreeAsync(cursor, s);
    if (cstart) cudaFreeAsync(cstart, s);
    if (scan_tmp) cudaFreeAsync(scan_tmp, s);
  };
#define CKL(call)                              \
  do {                                         \
    if ((call) != cudaSuccess) {               \
      cleanup();                               \
      if (lstart) cudaFreeAsync(lstart, s);    \
      if (lo->order) cudaFreeAsync(lo->order, s); \
      if (lo->corder) cudaFreeAsync(lo->corder, s); \
      lo->order = lo->corder = nullptr;        \
      return ILUK_ECUDA;                       \
    }                                          \
  } while (0)
  CKL(cudaMallocAsync((void **)&cnt, (size_t)nlev * sizeof(int32_t), s));
  CKL(cudaMallocAsync((void **)&cursor, (size_t)nlev * sizeof(int32_t), s));
  CKL(cudaMallocAsync((void **)&lstart, ((size_t)nlev + 1) * sizeof(int64_t), s));
  CKL(cudaMallocAsync((void **)&scan_tmp, (size_t)scan_tmp_elems(nlev) * sizeof(int64_t), s));
  CKL(cudaMemsetAsync(cnt, 0, (size_t)nlev * sizeof(int32_t), s));
  CKL(cudaMemsetAsync(cursor, 0, (size_t)nlev * sizeof(int32_t), s));
  CKL(cudaMallocAsync((void **)&cstart, ((size_t)nlev + 1) * sizeof(int64_t), s));
  k_level_count<<<grid_for(n), 256, 0, s>>>(n, depth, cnt);
  note_launch();
  CKL(launch_scan_lengths(nlev, cnt, cstart, scan_tmp, s));  // unpadded level starts
  k_level_pad<<<grid_for(nlev), 256, 0, s>>>(nlev, cnt);
  note_launch();
  CKL(launch_scan_lengths(nlev, cnt, lstart, scan_tmp, s));
  int64_t len = 0;
  CKL(cudaMemcpyAsync(&len, lstart + nlev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CKL(cudaStreamSynchronize(s));
  CKL(cudaMallocAsync((void **)&lo->order, (size_t)len * sizeof(int32_t), s));
  CKL(cudaMemsetAsync(lo->order, 0xff, (size_t)len * sizeof(int32_t), s));
  k_level_scatter<<<grid_for(n), 256, 0, s>>>(n, depth, lstart, cursor, lo->order);
  note_launch();
  CKL(cudaMallocAsync((void **)&lo->corder, (size_t)n * sizeof(int32_t), s));
  CKL(cudaMemsetAsync(cursor, 0, (size_t)nlev * sizeof(int32_t), s));
  k_level_scatter<<<grid_for(n), 256, 0, s>>>(n, depth, cstart, cursor, lo->corder);
  note_launch();
  CKL(cudaGetLastError());
#undef CKL
  cleanup();
  lo->lstart = lstart;
  lo->len = len;
  lo->nlev = nlev;
  lo->clen = n;
  return ILUK_OK;
}

// Synchronous: the depths of both sweep DAGs (one launch, one block each),
// then the two padded level orders.  On success fwd->order / bwd->order (and
// their level starts) are new device allocations.
int build_levels_pair(int64_t n, const int64_t *rp, const int32_t *ci, const int64_t *dg,
                      LevelOrder *fwd, LevelOrder *bwd, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_DEPTH, s);
  *fwd = LevelOrder();
  *bwd = LevelOrder();
  if (n == 0) return ILUK_OK;
  int32_t *depth = nullptr, *mx = nullptr;
  DevErr *err = nullptr;
  unsigned long long *ctl = nullptr;  // two tickets, two failure flags
  auto cleanup = [&]() {
    if (depth) cudaFreeAsync(depth, s);
    if (mx) cudaFreeAsync(mx, s);
    if (err) cudaFreeAsync(err, s);
    if (ctl) cudaFreeAsync(ctl, s);
  };
  if (cudaMallocAsync((void **)&depth, 2 * n * sizeof(int32_t), s) != cudaSuccess ||
      cudaMallocAsync((void **)&mx, 2 * sizeof(int32_t), s) != cudaSuccess ||
      cudaMallocAsync((void **)&err, 2 * sizeof(DevErr), s) != cudaSuccess ||
      cudaMallocAsync((void **)&ctl, 3 * sizeof(unsigned long long), s) != cudaSuccess ||
      cudaMemsetAsync(depth, 0, 2 * n * sizeof(int32_t), s) != cudaSuccess ||
      cudaMemsetAsync(mx, 0, 2 * sizeof(int32_t), s) != cudaSuccess ||
      cudaMemsetAsync(ctl, 0, 3 * sizeof(unsigned long long), s) != cudaSuccess ||
      launch_fill_err(err, s) != cudaSuccess || launch_fill_err(err + 1, s) != cudaSuccess) {
    cleanup();
    return ILUK_ECUDA;
  }
  // one forward and one backward CTA per SM: 1024 threads, which leaves room
  // beside the numeric phase's 256-thread CTA when both run at once
  int64_t grid = 2 * (int64_t)num_sms();
  const int64_t want = 2 * ((n * 32 + kDepthThreads - 1) / kDepthThreads);
  if (grid > want) grid = want;
  if (grid < 2) grid = 2;
  k_depth_pair<<<(unsigned)grid, kDepthThreads, 0, s>>>(n, rp, ci, dg, depth, depth + n, mx, err,
                                                        ctl, wait_limit());
  note_launch();
  DevErr herr[2];
  int32_t nlev[2] = {0, 0};
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(nlev, mx, sizeof(nlev), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cleanup();
    return ILUK_ECUDA;
  }
  for (int d = 0; d < 2; ++d)
    if (herr[d].key != kNoErr) {
      cleanup();
      return (int)(herr[d].key & 0xff);
    }
  int st = order_from_depth(n, depth, nlev[0], fwd, s);
  if (st == ILUK_OK) st = order_from_depth(n, depth + n, nlev[1], bwd, s);
  cleanup();
  return st;
}

// Index orders for the warp-per-row sweeps of a factorization whose level
// orders are not built: rows ascending (forward) and descending (backward),
// valid since every dependency lies at a smaller (forward) or larger
// (backward) index.  Only corder/clen are set.
__global__ void k_index_orders(int64_t n, int32_t *fwd, int32_t *bwd) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    fwd[i] = (int32_t)i;
    bwd[i] = (int32_t)(n - 1 - i);
  }
}

cudaError_t build_index_orders(int64_t n, LevelOrder *fwd, LevelOrder *bwd, cudaStream_t s) {
  *fwd = LevelOrder();
  *bwd = LevelOrder();
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMallocAsync((void **)&fwd->corder, (size_t)n * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&bwd->corder, (size_t)n * sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  k_index_orders<<<grid_for(n), 256, 0, s>>>(n, fwd->corder, bwd->corder);
  note_launch();
  fwd->clen = bwd->clen = n;
  return cudaGetLastError();
}

}  // namespace iluk

// LevelOrder is declared at global scope (internal.h), and so is this.
void level_order_free(LevelOrder &lo, cudaStream_t s) {
  if (lo.order) cudaFreeAsync(lo.order, s);
  if (lo.corder) cudaFreeAsync(lo.corder, s);
  if (lo.lstart) cudaFreeAsync(lo.lstart, s);
  for (OwnerCode &oc : lo.owner)
    if (oc.code) cudaFreeAsync(oc.code, s);
  lo = LevelOrder();
}
