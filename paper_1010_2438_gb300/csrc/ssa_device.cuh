// Device primitives of the direct-method step (Sec. 2.2): counter-based
// random words, the exact 52-bit uniform, the fixed FP64 logarithm for
// tau = -ln(u)/a0, and the FNV-1a event hash.
//
// On GB300 the FP64 pipe retires about 1.6 lane-operations per clock per SM
// (~1/70 of FP32), so everything here that can be done exactly with integer
// instructions is: the uniform is assembled bit by bit, comparisons of
// non-negative doubles are integer comparisons of their bit patterns, and
// halving / doubling a double is an exponent-field add.  Every remaining FP64
// operation is an explicit round-to-nearest intrinsic (__dadd_rn, __dmul_rn,
// __ddiv_rn), which the compiler never fuses into an FMA.
#pragma once

#include <cstdint>

namespace cwcgpu {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): per round two
// 32x32->64-bit products of counter words 0 and 2 with the round multipliers;
// the key is bumped by the two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// u = (k + 1/2) 2^-52 = (2k + 1) 2^-53 with k = (wa >> 6) : (wb >> 6), 52 bits.
// v = 2k + 1 < 2^53 is exactly representable, so the double is assembled from
// v's bits: exponent from the position of its leading one, mantissa from the
// bits below it.  Identical to converting v and scaling by 2^-53.
__device__ __forceinline__ double uniform52(uint32_t wa, uint32_t wb) {
  const unsigned long long k = ((unsigned long long)(wa >> 6) << 26) | (unsigned long long)(wb >> 6);
  const unsigned long long v = 2ull * k + 1ull;
  const int lead = 63 - __clzll((long long)v);                     // 0..52
  const unsigned long long mant = (v << (52 - lead)) & 0x000FFFFFFFFFFFFFull;
  const unsigned long long expo = (unsigned long long)(lead - 53 + 1023);
  return __longlong_as_double((long long)((expo << 52) | mant));
}

// Bit pattern of a double as a signed 64-bit integer.  For doubles >= +0 the
// integer order equals the numeric order.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// Coefficients of the logarithm: c[k] = 1/k for odd k = 3..21 (IEEE-divided
// on the host), and e*ln2 rounded to nearest for e = -53..0.
struct LogConstants {
  double c[22];
  double e_ln2[54];   // index e + 53
};

// ln(u) for u in (0,1):  u = f 2^E with f in [1,2); if f >= sqrt2 (the double
// nearest) then m = f/2, e = E + 1, else m = f, e = E; s = (m-1)/(m+1),
// z = s^2, p = c21 z + c19 ... + c3 by Horner, r = 2 (s + s (z p)),
// ln(u) = e ln2 + r.  ln m = 2 atanh(s) (Abramowitz & Stegun 4.1.27); the
// truncation after s^21/21 is below 1e-18 relative for |s| <= 0.1716.
// c: the coefficients (uniform index); eln2: the e*ln2 table (per-lane index,
// kept in shared memory).
__device__ __forceinline__ double log_fixed(double u, const double* c, const double* eln2) {
  const long long SQRT2_BITS = 0x3FF6A09E667F3BCDll;                 // 1.4142135623730951
  const long long ub = dbits(u);
  int e = (int)((ub >> 52) & 0x7ff) - 1023;
  long long fb = (ub & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll;  // f in [1,2)
  if (fb >= SQRT2_BITS) {
    fb -= (1ll << 52);                                               // f * 0.5, exact
    e += 1;
  }
  const double m = __longlong_as_double(fb);
  const double s = __ddiv_rn(__dadd_rn(m, -1.0), __dadd_rn(m, 1.0));
  const double z = __dmul_rn(s, s);
  double p = c[21];
#pragma unroll
  for (int k = 19; k >= 3; k -= 2) p = __dadd_rn(__dmul_rn(p, z), c[k]);
  const double inner = __dadd_rn(s, __dmul_rn(s, __dmul_rn(z, p)));
  // 2 * inner, exact: inner is 0 or a normal number far from the top of the range
  const long long ib = dbits(inner);
  const double r = (ib & 0x7FFFFFFFFFFFFFFFll) == 0 ? inner : __longlong_as_double(ib + (1ll << 52));
  return __dadd_rn(eln2[e + 53], r);
}

// FNV-1a 64-bit over the little-endian bytes of (uint32 rule, uint32 slot).
__device__ __forceinline__ unsigned long long fnv1a_event(unsigned long long h, uint32_t rule, uint32_t slot) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h ^= (rule >> (8 * i)) & 0xffu;
    h *= 0x100000001b3ull;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h ^= (slot >> (8 * i)) & 0xffu;
    h *= 0x100000001b3ull;
  }
  return h;
}

constexpr unsigned long long FNV_OFFSET = 0xcbf29ce484222325ull;

// (double)x for 0 <= x < 2^63, rounded to nearest-even, with integer
// instructions only.  Same value as the conversion instruction, which on
// GB300 issues to the FP64 pipe.  Below 2^53 the value is exact: the double
// is assembled from x's leading-one position and the bits under it; above,
// the dropped low bits decide the rounding (ties to even), and a carry out of
// the 53-bit significand bumps the exponent.
__device__ __forceinline__ double u63_to_double_rn(unsigned long long x) {
  if ((x >> 53) == 0ull) {
    // exact: shift the leading one to bit 52 and add the exponent (x = 0 -> +0)
    const int lead = 63 - __clzll((long long)x);
    const unsigned long long bits = ((unsigned long long)(1023 + lead) << 52) + ((x << (52 - lead)) - (1ull << 52));
    return x == 0ull ? 0.0 : __longlong_as_double((long long)bits);
  }
  int lead = 63 - __clzll((long long)x);
  unsigned long long m;
  if (lead <= 52) {
    m = x << (52 - lead);
  } else {
    const int sh = lead - 52;
    m = x >> sh;
    const unsigned long long rem = x & ((1ull << sh) - 1ull);
    const unsigned long long half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) m += 1ull;
    if (m == (1ull << 53)) {
      m >>= 1;
      lead += 1;
    }
  }
  const unsigned long long bits = ((unsigned long long)(1023 + lead) << 52) | (m & 0x000FFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

// Combinatorial count C(n, nu) for nu in {1, 2}, n >= 0 (Match_Populations).
__device__ __forceinline__ unsigned long long binom12(int n, int nu) {
  const unsigned long long un = (unsigned long long)n;
  return nu == 1 ? un : (un * (un - (un > 0 ? 1ull : 0ull))) >> 1;
}

// a * b for a, b <= 2^63-1; sets *ovf if the product exceeds 2^63-1.
__device__ __forceinline__ unsigned long long mul_checked(unsigned long long a, unsigned long long b, bool* ovf) {
  const unsigned long long hi = __umul64hi(a, b);
  const unsigned long long lo = a * b;
  if (hi != 0ull || (lo >> 63) != 0ull) *ovf = true;
  return lo;
}

// Exact 128-bit accumulation of x^2 (x < 2^31) into (low, high): the thread
// whose add wraps the low word, seen from the value it replaced, carries one
// into the high word, so the sum is exact whatever the order of the adds.
__device__ __forceinline__ void add_square_u128(unsigned long long* lohi, int x) {
  const unsigned long long v = (unsigned long long)(unsigned)x * (unsigned)x;
  const unsigned long long old = atomicAdd(lohi, v);
  if (old + v < old) atomicAdd(lohi + 1, 1ull);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace cwcgpu
