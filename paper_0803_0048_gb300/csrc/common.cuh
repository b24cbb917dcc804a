// common.cuh -- device helpers shared by the libiluk kernels.
//
// Row-to-row synchronisation: every output a later row may read starts out
// as a pending marker (a signalling-NaN bit pattern for values, an
// impossible column or level for patterns) and is written exactly once, so a
// dependent row polls the data itself with relaxed loads: no flags, no
// fences.  Every wait is bounded by a time limit read from %globaltimer; on
// running out, or when an earlier row has failed, the wait returns false and
// the kernel records a status and returns (no trap, no endless loop).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/iluk.h"

#define FULL_MASK 0xffffffffu

namespace iluk {

// Error word: (row << 8) | code, combined with atomicMin so that the smallest
// failing row wins, whatever order the rows fail in.  ~0ull means "no error".
struct DevErr {
  unsigned long long key;
  unsigned long long need;
};

static constexpr unsigned long long kNoErr = ~0ull;

__device__ __forceinline__ unsigned long long err_key(int64_t row, int code) {
  return ((unsigned long long)row << 8) | (unsigned long long)code;
}

__device__ __forceinline__ void set_err(DevErr *e, int64_t row, int code) {
  atomicMin(&e->key, err_key(row, code));
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
  return *((volatile const unsigned long long *)p);
}

// True if a row smaller than `row` has failed (its dependants must stop).
__device__ __forceinline__ bool earlier_failed(const DevErr *e, int64_t row) {
  unsigned long long k = ld_volatile_u64(&e->key);
  return k != kNoErr && (int64_t)(k >> 8) < row;
}

__device__ __forceinline__ bool any_failed(const DevErr *e) {
  return ld_volatile_u64(&e->key) != kNoErr;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Lower bound of `key` in the sorted array a[lo, hi).
template <typename T>
__device__ __forceinline__ int lower_bound_i(const T *a, int lo, int hi, T key) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <typename T>
__device__ __forceinline__ int64_t lower_bound_l(const T *a, int64_t lo, int64_t hi, T key) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// One IEEE multiply then one IEEE subtract, each rounded to nearest.
__device__ __forceinline__ double sub_prod(double acc, double a, double b) {
  return __dsub_rn(acc, __dmul_rn(a, b));
}

__device__ __forceinline__ double add_prod(double acc, double a, double b) {
  return __dadd_rn(acc, __dmul_rn(a, b));
}

// Correctly rounded division from a precomputed reciprocal.
//
// recip_dd(b) = (y, t): y = RN(1/b), and t = RN(e*y) with e = 1 - b*y (exact:
// the residual of a correctly rounded reciprocal is representable), so that
// y + t = 1/b within a relative 2^-104.  Then for a dividend a
//   q0 = RN(a*y + RN(a*t))      is within 1/2 ulp + 2^-104 of a/b: faithful,
//   r  = a - b*q0               is exact (fma) because q0 is faithful,
//   q  = RN(q0 + r*y)           is RN(a/b) by Markstein's theorem (P. Markstein,
//                               IBM J. Res. Dev. 34(1), 1990; J.-M. Muller et
//                               al., Handbook of Floating-Point Arithmetic,
//                               ch. 4), y being within 1/2 ulp of 1/b.
// Four dependent FP64 operations instead of a full IEEE division on the
// critical path.  The argument assumes no intermediate underflows or
// overflows: both operands must have magnitudes in [2^-400, 2^401), else
// (zero, subnormal, huge, infinite, NaN) the quotient comes from __ddiv_rn.
// recip_dd marks such a divisor with y = 0, and any y outside that range
// (0, NaN) also selects __ddiv_rn.
__device__ __forceinline__ bool dd_in_range(double x) {
  const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
  return ex - 623u <= 800u;  // biased exponent in [1023-400, 1023+400]
}

__device__ __forceinline__ double2 recip_dd(double b) {
  if (!dd_in_range(b)) return make_double2(0.0, 0.0);
  const double y = __drcp_rn(b);
  const double e = __fma_rn(-b, y, 1.0);
  return make_double2(y, __dmul_rn(e, y));
}

__device__ __forceinline__ double div_rn_recip(double a, double b, double2 rb) {
  if (!dd_in_range(rb.x) || !dd_in_range(a)) return __ddiv_rn(a, b);
  const double q0 = __fma_rn(a, rb.x, __dmul_rn(a, rb.y));
  const double r = __fma_rn(-b, q0, a);
  return __fma_rn(r, rb.x, q0);
}

}  // namespace iluk
