// krylov.cu -- a6 building blocks of right-preconditioned GMRES(m).
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
// inner product: the thread that updates w_q is the one that owns index q in
// the reduction, so no other thread needs the updated value first.
#include "internal.h"

namespace iluk {

constexpr int kDotThreads = 256;
constexpr int kDotBlocks = kDotP / kDotThreads;

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

// Last-block tree reduction of the 4096 partials.
__device__ void dot_finish(double *partial, unsigned *counter, double *out, int take_sqrt) {
  __shared__ double sh[kDotP];
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned)(gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  for (int p = threadIdx.x; p < kDotP; p += blockDim.x) sh[p] = __ldcg(&partial[p]);
  __syncthreads();
  for (int w = kDotP / 2; w >= 1; w >>= 1) {
    for (int p = threadIdx.x; p < w; p += blockDim.x) sh[p] = __dadd_rn(sh[p], sh[p + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = take_sqrt ? __dsqrt_rn(sh[0]) : sh[0];
    *counter = 0u;
  }
}

__global__ void __launch_bounds__(kDotThreads)
k_dot(int64_t n, const double *__restrict__ x, const double *__restrict__ y, double *partial,
      unsigned *counter, double *out, int take_sqrt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  for (int64_t i = p; i < n; i += kDotP) s = __dadd_rn(s, __dmul_rn(x[i], y[i]));
  partial[p] = s;
  dot_finish(partial, counter, out, take_sqrt);
}

cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *out, int take_sqrt,
                       const DotScratch &ds, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_DOT, s);
  k_dot<<<kDotBlocks, kDotThreads, 0, s>>>(n, x, y, ds.partial, ds.counter, out, take_sqrt);
  note_launch();
  return cudaGetLastError();
}

// w <- w - h * v_i (h read from device memory), then the fixed-shape inner
// product of the new w with vnext (vnext == w gives ||w||^2).
__global__ void __launch_bounds__(kDotThreads)
k_mgs_step(int64_t n, double *w, const double *__restrict__ vi, const double *hij,
           const double *vnext, double *partial, unsigned *counter, double *out, int take_sqrt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const double h = *hij;
  double s = 0.0;
  for (int64_t i = p; i < n; i += kDotP) {
    const double wi = __dsub_rn(w[i], __dmul_rn(h, vi[i]));
    w[i] = wi;
    s = __dadd_rn(s, __dmul_rn(wi, vnext[i]));
  }
  partial[p] = s;
  dot_finish(partial, counter, out, take_sqrt);
}

cudaError_t launch_mgs_step(int64_t n, double *w, const double *vi, const double *hij,
                            const double *vnext, double *out, int take_sqrt,
                            const DotScratch &ds, cudaStream_t s) {
  ProfScope prof_scope(ILUK_PROF_DOT, s);
  k_mgs_step<<<kDotBlocks, kDotThreads, 0, s>>>(n, w, vi, hij, vnext, ds.partial, ds.counter, out,
                                                take_sqrt);
  note_launch();
  return cudaGetLastError();
}

// y = x / den[0], skipped when den[0] == 0 (GMRES breakdown).
__global__ void k_scale_div(int64_t n, const double *__restrict__ x, const double *den, double *y) {
  const double d = *den;
  if (d == 0.0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __ddiv_rn(x[i], d);
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
