// krylov.cu -- a6: building blocks of right-preconditioned GMRES(m).
//
// Inner products use one fixed reduction shape, independent of the GPU:
// 4096 partial sums, partial p summing indices p, p+4096, ... left to right
// from +0.0 (products rounded, then sums rounded), then the pairwise tree
// s[p] = s[p] + s[p+w] for w = 2048, 1024, ..., 1.  The result therefore does
// not depend on launch configuration, and a sequential program that follows
// the same shape reproduces it bit for bit (Sec. 3.5 keeps inner products in a
// fixed order for the same reason).
//
// The modified Gram-Schmidt step w <- w - h_ij v_i is fused with the next
// inner product: the thread that updates w_q also forms w_q * vnext_q, so no
// other thread needs the updated value.
#include "internal.h"

namespace iluk {

// A CTA owns 32 consecutive partials (128 CTAs).  The element operations
// (products, and the Gram-Schmidt update) are independent; only the additions
// into a partial form a chain.  FP64 issue is what limits these kernels on
// this part: one warp instruction occupies an SM sub-partition's FP64 pipe
// for ~75 clocks, and a dependent addition waits ~64.  So warp 0 runs the
// CTA's 32 chains (one per lane) from products staged in shared memory, alone
// on its sub-partition, while the warps of the other three sub-partitions
// (warp % 4 != 0) evaluate the products.
constexpr int kRedWarps = 8;
constexpr int kRedThreads = kRedWarps * 32;
constexpr int kRedBlocks = kDotP / 32;
constexpr int kRowsPerWarp = 8;                          // rows m per compute warp per chunk
constexpr int kComputeWarps = kRedWarps * 3 / 4;
constexpr int kChunk = kComputeWarps * kRowsPerWarp;     // rows m per chunk
static_assert(2 * kChunk * 32 <= kDotP, "chunk buffers reuse the reduction array");
static_assert(kDotP % kRedThreads == 0, "the finishing CTA holds kDotP / kRedThreads partials");

// Index of a compute warp, or -1 for the warps of sub-partition 0.
__device__ __forceinline__ int compute_index(int warp) {
  return (warp & 3) ? warp - (warp >> 2) - 1 : -1;
}

// y = A x (b_minus == nullptr) or y = b - A x; each row summed left to right
// from +0.0.  One thread per row: a row's sum is a chain of dependent FP64
// additions, so a warp advances 32 rows' chains with each instruction.
__global__ void __launch_bounds__(256)
k_spmv(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ ci,
       const double *__restrict__ v, const double *__restrict__ x, double *y,
       const double *b_minus) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b0 = rp[row], b1 = rp[row + 1];
    double s = 0.0;
#pragma unroll 4
    for (int64_t q = b0; q < b1; ++q) s = __dadd_rn(s, __dmul_rn(v[q], x[ci[q]]));
    y[row] = b_minus ? __dsub_rn(b_minus[row], s) : s;
  }
}

cudaError_t launch_spmv(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                        const double *x, double *y, const double *b_minus, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_SPMV, s);
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  k_spmv<<<(unsigned)blocks, 256, 0, s>>>(n, rp, ci, v, x, y, b_minus);
  note_launch();
  return cudaGetLastError();
}

// Last-CTA tree reduction of the 4096 partials (sh: at least kRedThreads
// doubles).  Thread t holds s[t + 256 k], k < 16, so the levels w = 2048..256
// pair two values of one thread and run in registers; w = 128..32 go through
// shared memory and w = 16..1 are shuffles of warp 0.
__device__ void dot_finish(double *partial, unsigned *counter, double *out, int take_sqrt,
                           double *sh) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned)(gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  constexpr int K = kDotP / kRedThreads;
  const int t = threadIdx.x;
  double v[K];
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = __ldcg(&partial[t + kRedThreads * k]);
#pragma unroll
  for (int h = K / 2; h >= 1; h >>= 1)
#pragma unroll
    for (int k = 0; k < h; ++k) v[k] = __dadd_rn(v[k], v[k + h]);
  sh[t] = v[0];
  __syncthreads();
  for (int w = kRedThreads / 2; w >= 32; w >>= 1) {
    if (t < w) sh[t] = __dadd_rn(sh[t], sh[t + w]);
    __syncthreads();
  }
  if (t < 32) {
    double x = sh[t];
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
      const double o = __shfl_down_sync(0xffffffffu, x, w);
      if (t < w) x = __dadd_rn(x, o);
    }
    if (t == 0) {
      out[0] = take_sqrt ? __dsqrt_rn(x) : x;
      *counter = 0u;
    }
  }
}

// The CTA's 32 partials: partial p = 32 blockIdx.x + lane sums prod(i) for
// i = p, p + 4096, ... (row m of the partial is i = p + 4096 m) left to right
// from +0.0.  Rows are taken kChunk at a time: warps 1..7 evaluate chunk c
// into one half of sh, with the operands of chunk c+1 already loading, while
// warp 0 adds chunk c-1 from the other half.  Returns the partial in warp 0's
// lanes.  Op::load fetches the operands of kRowsPerWarp rows i0, i0 + 4096,
// ... (those < n) and Op::eval turns them into the rows' products.
template <class Op>
__device__ double chained_partials(int64_t n, const Op &op, double *sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t p = (int64_t)blockIdx.x * 32 + lane;
  const int64_t rows = (n + kDotP - 1) / kDotP;
  const int64_t lane_rows = p < n ? (n - p + kDotP - 1) / kDotP : 0;  // i = p + 4096 m < n
  const int64_t nchunks = (rows + kChunk - 1) / kChunk;
  const int cw = compute_index(warp);
  const int r0 = cw * kRowsPerWarp;
  auto first = [&](int64_t c) { return p + (c * kChunk + r0) * (int64_t)kDotP; };
  typename Op::Regs cur, nxt;
  if (cw >= 0 && nchunks > 0) op.load(first(0), n, cur);
  double s = 0.0;
  for (int64_t c = 0; c <= nchunks; ++c) {
    if (cw >= 0) {
      if (c < nchunks) {
        if (c + 1 < nchunks) op.load(first(c + 1), n, nxt);
        double *buf = sh + (c & 1) * (kChunk * 32);
        double pr[kRowsPerWarp];
        op.eval(first(c), n, cur, pr);
#pragma unroll
        for (int u = 0; u < kRowsPerWarp; ++u) buf[(r0 + u) * 32 + lane] = pr[u];
        if (c + 1 < nchunks) cur = nxt;
      }
    } else if (warp == 0 && c > 0) {
      const double *buf = sh + ((c - 1) & 1) * (kChunk * 32) + lane;
      const int64_t left = lane_rows - (c - 1) * kChunk;  // this lane's rows from the chunk on
      if (left >= kChunk) {
#pragma unroll 16
        for (int r = 0; r < kChunk; ++r) s = __dadd_rn(s, buf[r * 32]);
      } else {
        for (int r = 0; r < (int)left; ++r) s = __dadd_rn(s, buf[r * 32]);
      }
    }
    __syncthreads();
  }
  return s;
}

struct DotOp {
  const double *x, *y;
  struct Regs { double x[kRowsPerWarp], y[kRowsPerWarp]; };
  __device__ void load(int64_t i0, int64_t n, Regs &r) const {
#pragma unroll
    for (int u = 0; u < kRowsPerWarp; ++u) {
      const int64_t i = i0 + (int64_t)u * kDotP;
      r.x[u] = i < n ? x[i] : 0.0;
      r.y[u] = i < n ? y[i] : 0.0;
    }
  }
  __device__ void eval(int64_t, int64_t, const Regs &r, double *pr) const {
#pragma unroll
    for (int u = 0; u < kRowsPerWarp; ++u) pr[u] = __dmul_rn(r.x[u], r.y[u]);
  }
};

// w_i <- w_i - h v_i, product w_i * vnext_i (vnext == w: w_i * w_i of the
// updated w).  Each w_i is read and written by the one thread that owns it.
struct MgsOp {
  double *w;
  const double *vi, *vnext;
  double h;
  bool self;
  struct Regs { double w[kRowsPerWarp], v[kRowsPerWarp], nx[kRowsPerWarp]; };
  __device__ void load(int64_t i0, int64_t n, Regs &r) const {
#pragma unroll
    for (int u = 0; u < kRowsPerWarp; ++u) {
      const int64_t i = i0 + (int64_t)u * kDotP;
      r.w[u] = i < n ? w[i] : 0.0;
      r.v[u] = i < n ? vi[i] : 0.0;
      r.nx[u] = (i < n && !self) ? vnext[i] : 0.0;
    }
  }
  __device__ void eval(int64_t i0, int64_t n, const Regs &r, double *pr) const {
#pragma unroll
    for (int u = 0; u < kRowsPerWarp; ++u) {
      const int64_t i = i0 + (int64_t)u * kDotP;
      const double wi = __dsub_rn(r.w[u], __dmul_rn(h, r.v[u]));
      if (i < n) w[i] = wi;
      pr[u] = __dmul_rn(wi, self ? wi : r.nx[u]);
    }
  }
};

__global__ void __launch_bounds__(kRedThreads)
k_dot(int64_t n, const double *x, const double *y, double *partial, unsigned *counter,
      double *out, int take_sqrt) {
  __shared__ double sh[kDotP];
  const double s = chained_partials(n, DotOp{x, y}, sh);
  if (threadIdx.x < 32) partial[blockIdx.x * 32 + threadIdx.x] = s;
  dot_finish(partial, counter, out, take_sqrt, sh);
}

// w <- w - h * v_i (h read from device memory), then the fixed-shape inner
// product of the new w with vnext (vnext == w gives ||w||^2).
__global__ void __launch_bounds__(kRedThreads)
k_mgs_step(int64_t n, double *w, const double *vi, const double *hij, const double *vnext,
           double *partial, unsigned *counter, double *out, int take_sqrt) {
  __shared__ double sh[kDotP];
  const double s =
      chained_partials(n, MgsOp{w, vi, vnext, *hij, vnext == w}, sh);
  if (threadIdx.x < 32) partial[blockIdx.x * 32 + threadIdx.x] = s;
  dot_finish(partial, counter, out, take_sqrt, sh);
}

cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *out, int take_sqrt,
                       const DotScratch &ds, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_DOT, s);
  k_dot<<<kRedBlocks, kRedThreads, 0, s>>>(n, x, y, ds.partial, ds.counter, out, take_sqrt);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_mgs_step(int64_t n, double *w, const double *vi, const double *hij,
                            const double *vnext, double *out, int take_sqrt,
                            const DotScratch &ds, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_DOT, s);
  k_mgs_step<<<kRedBlocks, kRedThreads, 0, s>>>(n, w, vi, hij, vnext, ds.partial, ds.counter,
                                                out, take_sqrt);
  note_launch();
  return cudaGetLastError();
}

// y = x / den[0], skipped when den[0] == 0 (GMRES breakdown).
__global__ void k_scale_div(int64_t n, const double *__restrict__ x, const double *den, double *y) {
  const double d = *den;
  if (d == 0.0) return;
  const DivPrep pd = div_prep(d);  // one reciprocal, n quotients
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = div_fin(x[i], pd);
}

static unsigned vec_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_scale_div(int64_t n, const double *x, const double *den, double *y,
                             cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_VECTOR, s);
  if (n == 0) return cudaSuccess;
  k_scale_div<<<vec_blocks(n), 256, 0, s>>>(n, x, den, y);
  note_launch();
  return cudaGetLastError();
}

// u_q = sum_j y_j V[j][q], j ascending from +0.0.
__global__ void k_combine(int64_t n, const double *__restrict__ V, int64_t ldv,
                          const double *__restrict__ y, int cnt, double *__restrict__ u) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < cnt; ++j) s = __dadd_rn(s, __dmul_rn(y[j], V[(int64_t)j * ldv + q]));
    u[q] = s;
  }
}

cudaError_t launch_combine(int64_t n, const double *V, int64_t ldv, const double *y, int cnt,
                           double *u, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_VECTOR, s);
  if (n == 0) return cudaSuccess;
  k_combine<<<vec_blocks(n), 256, 0, s>>>(n, V, ldv, y, cnt, u);
  note_launch();
  return cudaGetLastError();
}

// u_i = u_i + y * z_i (y read on the device), one rounding each: one term
// of k_combine's sum at a time, in the same order.
__global__ void k_acc_scaled(int64_t n, double *u, const double *__restrict__ y,
                             const double *__restrict__ z) {
  const double yj = *y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    u[i] = __dadd_rn(u[i], __dmul_rn(yj, z[i]));
}

cudaError_t launch_acc_scaled(int64_t n, double *u, const double *y, const double *z,
                              cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_VECTOR, s);
  if (n == 0) return cudaSuccess;
  k_acc_scaled<<<vec_blocks(n), 256, 0, s>>>(n, u, y, z);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_add(int64_t n, double *x, const double *__restrict__ z) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = __dadd_rn(x[i], z[i]);
}

cudaError_t launch_add(int64_t n, double *x, const double *z, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_VECTOR, s);
  if (n == 0) return cudaSuccess;
  k_add<<<vec_blocks(n), 256, 0, s>>>(n, x, z);
  note_launch();
  return cudaGetLastError();
}

// BiCGSTAB vector updates, each operation rounded once in the oracle's order.
// p = r + beta * (p - omega * v)
__global__ void k_bicg_dir(int64_t n, double *p, const double *__restrict__ r,
                           const double *__restrict__ v, double beta, double omega) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = __dadd_rn(r[i], __dmul_rn(beta, __dsub_rn(p[i], __dmul_rn(omega, v[i]))));
}

// out = a - alpha * b
__global__ void k_axmy(int64_t n, double *out, const double *__restrict__ a, double alpha,
                       const double *__restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __dsub_rn(a[i], __dmul_rn(alpha, b[i]));
}

// x = (x + alpha * ph) + omega * sh, or x = x + alpha * ph when sh is null
__global__ void k_bicg_x(int64_t n, double *x, double alpha, const double *__restrict__ ph,
                         double omega, const double *__restrict__ sh) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double xa = __dadd_rn(x[i], __dmul_rn(alpha, ph[i]));
    x[i] = sh ? __dadd_rn(xa, __dmul_rn(omega, sh[i])) : xa;
  }
}

cudaError_t launch_bicg_dir(int64_t n, double *p, const double *r, const double *v, double beta,
                            double omega, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_VECTOR, s);
  if (n == 0) return cudaSuccess;
  k_bicg_dir<<<vec_blocks(n), 256, 0, s>>>(n, p, r, v, beta, omega);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_axmy(int64_t n, double *out, const double *a, double alpha, const double *b,
                        cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_VECTOR, s);
  if (n == 0) return cudaSuccess;
  k_axmy<<<vec_blocks(n), 256, 0, s>>>(n, out, a, alpha, b);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bicg_x(int64_t n, double *x, double alpha, const double *ph, double omega,
                          const double *sh, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_VECTOR, s);
  if (n == 0) return cudaSuccess;
  k_bicg_x<<<vec_blocks(n), 256, 0, s>>>(n, x, alpha, ph, omega, sh);
  note_launch();
  return cudaGetLastError();
}

// gA[p] = -(lambda_i * x_j) for entry p = (i, j).
__global__ void k_adjoint_scatter(int64_t n, const int64_t *__restrict__ rp,
                                  const int32_t *__restrict__ ci, const double *__restrict__ lam,
                                  const double *__restrict__ x, double *__restrict__ gA) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += nw) {
    const double li = lam[row];
    for (int64_t p = rp[row] + lane; p < rp[row + 1]; p += 32) gA[p] = -__dmul_rn(li, x[ci[p]]);
  }
}

cudaError_t launch_adjoint_scatter(int64_t n, const int64_t *rp, const int32_t *ci,
                                   const double *lam, const double *x, double *gA,
                                   cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_VECTOR, s);
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n * 32 + 255) / 256;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  k_adjoint_scatter<<<(unsigned)blocks, 256, 0, s>>>(n, rp, ci, lam, x, gA);
  note_launch();
  return cudaGetLastError();
}

}  // namespace iluk
