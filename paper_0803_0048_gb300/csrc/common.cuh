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

// Correctly rounded double division on the integer pipes.
//
// On this GPU a double-precision instruction holds its sub-partition's FP64
// pipe for tens of cycles and an IEEE division (__ddiv_rn) is a chain of
// about ten of them (~1,000 cycles of latency when timed in a dependent
// chain).  The multipliers of the numeric phase (f_ih / f_hh, Eq. lufactor2)
// and the backward sweep's division by u_ii (Eq. triangleSolve) lie on the
// critical path, so they are computed with integer arithmetic instead, in
// two parts:
//
// div_prep(b), once per divisor: D = b's 53-bit significand in [2^52, 2^53)
//   and X ~ 2^115 / D, a 64-bit fixed-point reciprocal.  Seed: the fp32
//   number 1.f with f = D's top 23 fraction bits (built from bits, no
//   conversion instruction), its rcp.approx (relative error below 2^-22),
//   read back from its bits as Y ~ 2^84 / D.  One Newton-Raphson step
//   y <- y + y (1 - d y) on the top 32 bits of D brings Y to ~31 bits, one
//   more at 64-bit precision, X = Y 2^31 + X (1 - d X), to ~61 bits
//   (|X - 2^115/D| below a few units).
// div_fin(a, prep), per quotient: with A = a's significand and s = (A < D),
//   the exact integer quotient Q = floor(A 2^(52+s) / D) lies in [2^52, 2^53);
//   Q0 = floor(A 2^(1+s) X / 2^64) is within one of it (the error term is
//   below A 2^(1+s) 2^3 / 2^64 < 2^-6), and with the remainder
//   R = A 2^(52+s) - Q0 D (exact in the low 64 bits, |R| < 2D) the correctly
//   rounded significand is Q0 - 1 + [2R > -D] + [2R > D] + [2R > 3D]: the
//   three comparisons fold the correction of Q0 and the round-to-nearest
//   decision into one step (2R never equals -D, D or 3D: the quotient of two
//   binary floating-point numbers is never a rounding midpoint).  It is
//   packed with exponent ea - eb + 1023 - s; a carry of the rounding into bit
//   53 lands in the exponent field, and into infinity at the top of the
//   range, as IEEE rounding does.
// This is the textbook scheme of a reciprocal approximation followed by an
// exact remainder correction (S. F. Oberman and M. J. Flynn, "Division
// algorithms and implementations", IEEE Trans. Computers 46(8), 1997;
// J.-M. Muller et al., Handbook of Floating-Point Arithmetic, ch. 4).  Only
// normal operands with a normal quotient (and a zero dividend) take it; any
// other case (zero, subnormal, infinite or NaN divisor, subnormal, infinite
// or NaN dividend, quotient that underflows or overflows the exponent range)
// returns __ddiv_rn(a, b).  The results equal IEEE division bit for bit
// (pinned against it by the library's tests through iluk_div_rn).
struct __align__(16) DivPrep {
  unsigned long long x;  // ~2^115 / D, or 0 when b is not a normal number
  double b;
};

// floor(a * x / 2^64) for a < 2^55, x < 2^63, from four independent 32x32
// products (the sums stay below 2^64).
__device__ __forceinline__ unsigned long long mulhi_55x63(unsigned long long a,
                                                          unsigned long long x) {
  const unsigned al = (unsigned)a, ah = (unsigned)(a >> 32);
  const unsigned xl = (unsigned)x, xh = (unsigned)(x >> 32);
  const unsigned long long ll = (unsigned long long)al * xl;
  const unsigned long long mid =
      (unsigned long long)ah * xl + (unsigned long long)al * xh + (ll >> 32);
  return (unsigned long long)ah * xh + (mid >> 32);
}

__device__ __forceinline__ DivPrep div_prep(double b) {
  DivPrep p;
  p.b = b;
  p.x = 0;
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
  const unsigned eb = (unsigned)(ub >> 52) & 0x7ffu;
  if (eb - 1u >= 2046u) return p;  // zero, subnormal, infinite or NaN
  const unsigned long long D = (ub & 0xfffffffffffffull) | (1ull << 52);
  const float f = __int_as_float(0x3f800000 | (int)((D >> 29) & 0x7fffffu));  // D/2^52, truncated
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(f));  // in (1/2, 1]
  const unsigned rb = (unsigned)__float_as_int(r);
  // Y = r 2^32: r's significand shifted by its exponent (126, or 127 for r = 1)
  unsigned long long Y = (unsigned long long)((rb & 0x7fffffu) | 0x800000u) << ((rb >> 23) - 118u);
  const unsigned d32 = (unsigned)(D >> 21);  // top 32 bits of D, d = d32 / 2^32
  const long long e1 = (long long)((1ull << 63) - (unsigned long long)d32 * Y);  // (1 - d y) 2^63
  Y += (unsigned long long)(((long long)Y * (e1 >> 31)) >> 32);
  if (Y > 0xffffffffull) Y = 0xffffffffull;
  const unsigned y = (unsigned)Y;
  const unsigned long long Dn = D << 11;  // d = Dn / 2^64
  // t = floor(Dn X / 2^64) with X = y 2^31: floor(Dn y / 2^33), ~2^62
  const unsigned long long t =
      (((Dn >> 32) * (unsigned long long)y + (((unsigned long long)(unsigned)Dn * y) >> 32)) >> 1);
  const long long e = (long long)((1ull << 62) - t);  // (1 - d X) 2^62, |e| < 2^33
  const long long corr = ((long long)y * (e >> 1)) >> 30;  // X e / 2^62 = y e / 2^31
  unsigned long long x = ((unsigned long long)y << 31) + (unsigned long long)corr;
  if (x > 0x7fffffffffffffffull) x = 0x7fffffffffffffffull;
  p.x = x;
  return p;
}

__device__ __forceinline__ double div_fin(double a, const DivPrep &p) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ub = (unsigned long long)__double_as_longlong(p.b);
  const unsigned long long sign = (ua ^ ub) & (1ull << 63);
  const unsigned ea = (unsigned)(ua >> 52) & 0x7ffu;
  const int eb = (int)((ub >> 52) & 0x7ffu);
  const unsigned long long A = (ua & 0xfffffffffffffull) | (1ull << 52);
  const unsigned long long D = (ub & 0xfffffffffffffull) | (1ull << 52);
  const bool s = A < D;
  const int E = (int)ea - eb + 1023 - (int)s;  // biased exponent of the quotient
  const unsigned long long A2 = s ? A << 2 : A << 1;
  const unsigned long long N = s ? A << 53 : A << 52;  // low 64 bits of A 2^(52+s)
  const unsigned long long q0 = mulhi_55x63(A2, p.x);
  const long long T = (long long)(N - q0 * D) * 2;  // 2R, |2R| < 2^56
  const long long Dl = (long long)D;
  const unsigned long long q =
      q0 + (unsigned long long)((T > -Dl) + (T > Dl) + (T > 3 * Dl)) - 1ull;
  if (p.x != 0 && ea - 1u < 2046u && E >= 1 && E <= 2046)
    return __longlong_as_double((long long)(sign | (((unsigned long long)(E - 1) << 52) + q)));
  if (p.x != 0 && (ua << 1) == 0) return __longlong_as_double((long long)sign);  // 0 / b
  return __ddiv_rn(a, p.b);
}

__device__ __forceinline__ double div_int(double a, double b) { return div_fin(a, div_prep(b)); }

}  // namespace iluk
