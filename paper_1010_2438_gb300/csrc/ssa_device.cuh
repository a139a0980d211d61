// Device primitives of the direct-method step (Sec. 2.2): counter-based
// random words, the exact 52-bit uniform, the fixed logarithm for
// tau = -ln(u)/a0 (integer arithmetic), and the FNV-1a event hash.
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

// Constants of the logarithm, filled on the host: cq[n] = floor(2^63 / n);
// ln 2 in Q120 as the truncated series sum_{k=1..120} floor(2^(120-k) / k)
// (ln 2 = sum 1/(k 2^k)), in two words; per 6-bit significand prefix j,
// rj[j] = ceil(2^69 / (64 + j)) (1/c_j in Q63, c_j = 1 + j/64) and tj[j] =
// ln c_j in Q64 (atanh series).  Kernels keep rj / tj in shared memory (they
// are indexed per lane).
struct LogConstants {
  unsigned long long cq[40];
  unsigned long long ln2_lo, ln2_hi;
  unsigned long long rj[64];
  unsigned long long tj[64];
};

// (x * 2^scale) rounded to the nearest double, ties to even, assembled from
// the integer's bits; x > 0 and the result normal.
__device__ __forceinline__ double round_q128(unsigned __int128 x, int scale) {
  const unsigned long long hi = (unsigned long long)(x >> 64), lo = (unsigned long long)x;
  const int lead = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
  unsigned long long mant;
  int e = lead;
  if (lead <= 52) {
    mant = lo << (52 - lead);
  } else {
    const int sh = lead - 52;
    mant = (unsigned long long)(x >> sh);
    const unsigned __int128 rem = x & ((((unsigned __int128)1) << sh) - 1);
    const unsigned __int128 half = ((unsigned __int128)1) << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) mant += 1ull;
    if (mant == (1ull << 53)) {
      mant >>= 1;
      e += 1;
    }
  }
  const unsigned long long bexp = (unsigned long long)(e + scale + 1023);
  return __longlong_as_double((long long)((bexp << 52) | (mant & 0x000FFFFFFFFFFFFFull)));
}

// ln(u) for u in [2^-53, 1), in exact integer arithmetic with one rounding
// at the end.  u = F 2^(E-52), F the 53-bit significand, f = F 2^-52.
//  * Near one (E = -1, D = 2^53 - F < 2^46, d = 1 - u < 2^-7): -ln u =
//    d (1 + d/2 + ... + d^8/9) (Mercator series, Abramowitz & Stegun
//    4.1.24), Horner with q in Q63 and d in Q64; -ln u = D q 2^-116.
//  * Otherwise, j = the top 6 fraction bits of f: -ln u = -E ln2 - ln c_j -
//    ln(1 + y), y = f rj[j] - 1 in [0, 2^-6) in Q64, ln(1 + y) = y (1 - y/2
//    + ... + y^10/11) by Horner in Q63, the sum in Q120.
// Every product is floored to the stated width.  No division, no FP64
// instruction.  Error < 0.55 ulp.
__device__ __forceinline__ double log_spec_q(double u, const LogConstants& lc, const unsigned long long* s_rj,
                                             const unsigned long long* s_tj) {
  typedef unsigned __int128 u128;
  const unsigned long long b = (unsigned long long)__double_as_longlong(u);
  const int E = (int)((b >> 52) & 0x7ff) - 1023;
  const unsigned long long F = (b & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long D = (1ull << 53) - F;
  double y;
  if (E == -1 && D < (1ull << 46)) {
    const unsigned long long dq = D << 11;
    unsigned long long q = lc.cq[9];
#pragma unroll
    for (int n = 8; n >= 1; --n) q = lc.cq[n] + __umul64hi(q, dq);
    y = round_q128((u128)D * q, -116);
  } else {
    const int j = (int)((F >> 46) & 63);
    const u128 fr = (u128)(F << 11) * s_rj[j];                       // f rj in Q126
    const unsigned long long yq = (unsigned long long)(fr >> 62);    // f rj - 1 in Q64 (the 2^64 drops)
    unsigned long long p = lc.cq[11];
#pragma unroll
    for (int k = 10; k >= 2; --k) p = lc.cq[k] - __umul64hi(p, yq);
    p = (1ull << 63) - __umul64hi(p, yq);
    const u128 l1 = ((u128)yq * p) >> 7;
    const u128 ln2 = (((u128)lc.ln2_hi) << 64) | lc.ln2_lo;
    y = round_q128((u128)(unsigned long long)(-E) * ln2 - (((u128)s_tj[j]) << 56) - l1, -120);
  }
  return __longlong_as_double(__double_as_longlong(y) | (long long)0x8000000000000000ull);
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

// A double / 64-bit word stored as two int32 words (low word first, the
// bytes of the little-endian 64-bit value) at any 4-byte-aligned address:
// checkpoint records are int32 arrays whose length can be odd, so their
// 64-bit fields are not always 8-byte aligned.
__device__ __forceinline__ void put_f64(int32_t* p, double v) {
  p[0] = __double2loint(v);
  p[1] = __double2hiint(v);
}
__device__ __forceinline__ double get_f64(const int32_t* p) { return __hiloint2double(p[1], p[0]); }
__device__ __forceinline__ void put_u64(int32_t* p, unsigned long long v) {
  p[0] = (int32_t)(uint32_t)v;
  p[1] = (int32_t)(uint32_t)(v >> 32);
}
__device__ __forceinline__ unsigned long long get_u64(const int32_t* p) {
  return (unsigned long long)(uint32_t)p[0] | ((unsigned long long)(uint32_t)p[1] << 32);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

}  // namespace cwcgpu
