// Compartmentalised CWC terms (Sec. 2.1) under Gillespie's direct method
// (Sec. 2.2) with the Match / Resolve / Update step of Sec. 2.3 and Fig.
// "CWC simulator pseudo-code": rule choice by the FP64 propensity tree, then
// the stochastic choice of the context (compartment) inside the rule, then the
// rewrite, including transport between a compartment and its parent, binding
// to the wrap, creation and dissolution of compartments.
//
// A group of kL lanes (1, 4 or 8 of a warp) runs one trajectory.  Every lane
// of the group keeps the trajectory's scalar state (time, event index, tree
// walk) and computes it identically, so the group branches as one; the work
// that grows with the term is split over the lanes: the context scan (rounds
// of kL consecutive slots, a group prefix sum of their counts), the update of
// the dependent rules' totals (one rule per lane), the leaf rebuild, the grid
// records (observables over lanes) and the set-up of a term.  The rewrite
// itself is done by lane 0 of the group.  The FP64 instructions (logarithm,
// tau, tree) are then shared by 32 / kL terms per warp instead of 32, but a
// batch of 16,384 terms keeps 4x more warps resident with 4 lanes per term,
// which hides more of the slab loads' latency.
//
// Shared memory per trajectory, [index][trajectory]-strided: the 32 FP64
// leaves and 31 internal nodes of the rule tree and the int64 totals H_j
// (combinatorial counts summed over the rule's contexts; a_j = k_j * H_j).
// The term itself (C <= 64 slots x S species, content and wrap) lives in a
// per-group slab of the caller's workspace, reused across the trajectories a
// group runs:
//   chmask[C]  u64  children of each slot        labmask[L] u64  alive slots per label
//   alive      u64  alive slots                  tot[O]     i64  observable totals
//   meta[C]    i32  label | (parent + 1) << 8   wrap[C][S], content[C][S]  i32
// (Slot-major: a slot's counts are one row.  Species-major storage, which
// makes a context scan read one or two lines per species instead of one per
// slot, measured 8 % slower on 16,384 terms of 64 slots x 24 species: every
// count read then needs a multiply by the slot count, and the scans touch few
// slots per rule.)
// The observable totals (content per label, wrap per label, alive compartments
// per label) are kept up to date by every rewrite, so recording a grid point
// is O stores.
// After an event only the contexts of the rewritten compartments, of their
// children (which read the parent content) and of the free slots (CREATE
// fills one) can change their counts.  Each rule that reads a written
// location, or whose contexts the event adds, removes or re-parents, drops
// the old counts of those contexts from H_i before the rewrite and adds the
// new ones after it, so H is always exactly the sum the oracle re-matches
// every step.
#include <cuda_runtime.h>

#include "cwc_internal.h"
#include "ssa_device.cuh"

namespace cwcgpu {

// The kL lanes of a warp that run one trajectory.
template <int kL>
struct LaneGroup {
  unsigned mask;   // the group's lanes within the warp
  int gl;          // this lane's index in the group
  int base;        // the group's first lane in the warp
  __device__ LaneGroup() {
    const int lane = threadIdx.x & 31;
    gl = lane & (kL - 1);
    base = lane & ~(kL - 1);
    mask = kL == 32 ? 0xffffffffu : (((1u << kL) - 1u) << base);
  }
  __device__ __forceinline__ void sync() const {
    if (kL > 1) __syncwarp(mask);
  }
  __device__ __forceinline__ bool any(bool v) const {
    if (kL == 1) return v;
    return (__ballot_sync(mask, v) & mask) != 0u;
  }
  // bit k set when lane k of the group has v
  __device__ __forceinline__ unsigned ballot(bool v) const {
    if (kL == 1) return v ? 1u : 0u;
    return (__ballot_sync(mask, v) & mask) >> base;
  }
  template <class V>
  __device__ __forceinline__ V bcast(V v, int src) const {
    if (kL == 1) return v;
    return __shfl_sync(mask, v, src, kL);
  }
  __device__ __forceinline__ unsigned long long incl_scan(unsigned long long x) const {
#pragma unroll
    for (int off = 1; off < kL; off <<= 1) {
      const unsigned long long y = __shfl_up_sync(mask, x, off, kL);
      if (gl >= off) x += y;
    }
    return x;
  }
  __device__ __forceinline__ unsigned long long or_all(unsigned long long x) const {
#pragma unroll
    for (int off = kL / 2; off > 0; off >>= 1) x |= __shfl_xor_sync(mask, x, off, kL);
    return x;
  }
  // the same pairwise tree on every lane, so every lane holds the same sum
  __device__ __forceinline__ double sum(double x) const {
#pragma unroll
    for (int off = kL / 2; off > 0; off >>= 1) x = __dadd_rn(x, __shfl_xor_sync(mask, x, off, kL));
    return x;
  }
};

__device__ __forceinline__ long long cwc_grab_next(WorkspaceHeader* ws) {
  const unsigned mask = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(&ws->queue_next, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return (long long)(base + (unsigned long long)__popc(mask & ((1u << lane) - 1u)));
}

__host__ __device__ inline int cwc_table_bytes(int M, int n_deps) {
  int words = M * CWC_RULE_WORDS + n_deps;
  return ((words * 4 + 15) / 16) * 16 + 128 * 8;   // then the logarithm's 64 + 64 table words
}

// shared-memory bytes of one trajectory
__host__ __device__ inline int cwc_thread_bytes(int M) { return (32 + TREE_NODES + M) * 8; }

__host__ __device__ inline long long cwc_slab_words(int S, int L, int C, int M, bool sens) {
  const long long O = (long long)L * S + (long long)(L - 1) * S + L;
  long long w = 2LL * C + 2LL * L + 2 + 2 * O + (sens ? 7LL * M : 0) + C + 2LL * C * S;
  return (w + 31) / 32 * 32;
}

// Term counts are stored as CT: int32_t, or int16_t in the narrow launch,
// whose trajectories leave for a 32-bit launch (TS_WIDEN, below) as soon as
// a count would exceed 32767.
template <class CT>
__device__ __forceinline__ long long count_max() {
  return sizeof(CT) == 2 ? 0x7FFFll : 0x7FFFFFFFll;
}
// the status of a count that would leave CT's range: a 16-bit term hands the
// trajectory over to the 32-bit launch, a 32-bit one stops with INT_OVERFLOW
template <class CT>
__device__ __forceinline__ int count_overflow_status() {
  return sizeof(CT) == 2 ? TS_WIDEN : TS_INT_OVERFLOW;
}

// Sum of the counts of rule `rec` over the contexts in m (the child slots of
// a parent-child rule count only under a parent of the rule's context label);
// bit 63 of the result flags an int64 overflow of a count or of the sum.
// Out of line for lane groups (see below).
template <class CT>
__device__ __noinline__ unsigned long long cwc_count_sum(const CT* __restrict__ content,
                                                        const CT* __restrict__ wrap,
                                                        const int32_t* __restrict__ meta, int S,
                                                        const int32_t* rec, unsigned long long m) {
  const int kind = rec[CR_KIND];
  const bool parent_child = !(kind == RK_LOCAL || kind == RK_CREATE);
  const int nr = rec[CR_NREAC];
  const int ctx = rec[CR_CTX];
  bool of = false;
  unsigned long long tot = 0ull;
  while (m) {
    const int c = __ffsll((long long)m) - 1;
    m &= m - 1ull;
    int x0c = c;
    if (parent_child) {
      const int qq = (meta[c] >> 8) - 1;
      if ((meta[qq] & 0xff) != ctx) continue;
      x0c = qq;
    }
    const CT* x0 = content + (size_t)x0c * S;
    const CT* x1 = wrap + (size_t)c * S;
    const CT* x2 = content + (size_t)c * S;
    unsigned long long acc = 1ull;
    for (int a = 0; a < nr; ++a) {
      const int v = rec[CR_REAC + a];
      const int row = (v >> 24) & 3;
      const CT* x = row == 0 ? x0 : (row == 1 ? x1 : x2);
      acc = mul_checked(acc, binom12(x[v & 0xffff], (v >> 16) & 0xff), &of);
    }
    const unsigned long long s2 = tot + acc;
    if (s2 < tot || (s2 >> 63) != 0ull) of = true;
    tot = s2;
  }
  return of ? (tot | (1ull << 63)) : tot;
}

// The same for NESTED rules, whose contexts are grandchildren c: their parent
// must carry the child label and their grandparent the rule's label (the
// root's label 0 is never a child label); rows 0 / 1-2 / 3-4 read the
// grandparent's content, the parent's wrap and content, c's wrap and content.
template <class CT>
__device__ __noinline__ unsigned long long cwc_count_sum_nested(const CT* __restrict__ content,
                                                               const CT* __restrict__ wrap,
                                                               const int32_t* __restrict__ meta, int S,
                                                               const int32_t* rec, unsigned long long m) {
  const int nr = rec[CR_NREAC];
  const int ctx = rec[CR_CTX];
  bool of = false;
  unsigned long long tot = 0ull;
  while (m) {
    const int c = __ffsll((long long)m) - 1;
    m &= m - 1ull;
    const int qq = (meta[c] >> 8) - 1;
    if ((meta[qq] & 0xff) != rec[CR_CHILD]) continue;
    const int aa = (meta[qq] >> 8) - 1;
    if ((meta[aa] & 0xff) != ctx) continue;
    const CT* rows[5] = {content + (size_t)aa * S, wrap + (size_t)qq * S, content + (size_t)qq * S, wrap + (size_t)c * S, content + (size_t)c * S};
    unsigned long long acc = 1ull;
    for (int a = 0; a < nr; ++a) {
      const int v = rec[CR_REAC + a];
      acc = mul_checked(acc, binom12(rows[(v >> 24) & 7][v & 0xffff], (v >> 16) & 0xff), &of);
    }
    const unsigned long long s2 = tot + acc;
    if (s2 < tot || (s2 >> 63) != 0ull) of = true;
    tot = s2;
  }
  return of ? (tot | (1ull << 63)) : tot;
}

// FUSION: the occurrences over ordered pairs (d1, d2) of distinct sibling
// slots of the child label under a parent of the rule's label (d1 < d2 when
// the two compartment patterns are identical), multiplied in the oracle's
// order: parent content, first child's wrap and content (rows 0-2), second
// child's wrap and content (rows 3-4).  With want_pick, returns the first
// pair in ascending (d1, d2) order whose running sum exceeds xc, as
// d1 | d2 << 16 (the last positive pair if none does); otherwise the sum,
// bit 63 flagging an overflow of a product or of the sum.
template <class CT>
__device__ __noinline__ unsigned long long cwc_fusion_scan(const CT* __restrict__ content,
                                                          const CT* __restrict__ wrap,
                                                          const int32_t* __restrict__ meta, int S,
                                                          const int32_t* rec, unsigned long long kids,
                                                          bool want_pick, unsigned long long xc) {
  const int nr = rec[CR_NREAC];
  const int ctx = rec[CR_CTX];
  // identical compartment patterns: rows 1 / 3 and 2 / 4 hold the same entries
  bool sym = true;
  for (int a = 0; a < nr; ++a) {
    const int v = rec[CR_REAC + a];
    const int row = (v >> 24) & 7;
    if (row == 0) continue;
    const int twin_row = row == 1 ? 3 : row == 2 ? 4 : row == 3 ? 1 : 2;
    bool found = false;
    for (int b = 0; b < nr; ++b) {
      const int u = rec[CR_REAC + b];
      found |= ((u >> 24) & 7) == twin_row && (u & 0xffffff) == (v & 0xffffff);
    }
    sym = sym && found;
  }
  // PAIR: the two compartments keep their own right-hand sides, so a pair
  // and its swap are one application only if those are identical too
  if (rec[CR_KIND] == RK_PAIR && (rec[CR_GRAND] & 0xff) == 0) sym = false;
  bool of = false;
  unsigned long long tot = 0ull;
  unsigned long long last = 0ull;
  unsigned long long m1 = kids;
  while (m1) {
    const int d1 = __ffsll((long long)m1) - 1;
    m1 &= m1 - 1ull;
    const int qq = (meta[d1] >> 8) - 1;
    if ((meta[qq] & 0xff) != ctx) continue;
    const CT* x0 = content + (size_t)qq * S;
    unsigned long long m2 = kids & ~(1ull << d1);
    if (sym) m2 &= ~((2ull << d1) - 1ull);   // d2 > d1 only
    while (m2) {
      const int d2 = __ffsll((long long)m2) - 1;
      m2 &= m2 - 1ull;
      if ((meta[d2] >> 8) - 1 != qq) continue;
      unsigned long long acc = 1ull;
      for (int a = 0; a < nr; ++a) {
        const int v = rec[CR_REAC + a];
        const int row = (v >> 24) & 7;
        const CT* x = row == 0 ? x0
                           : row == 1 ? wrap + (size_t)d1 * S
                           : row == 2 ? content + (size_t)d1 * S
                           : row == 3 ? wrap + (size_t)d2 * S : content + (size_t)d2 * S;
        acc = mul_checked(acc, binom12(x[v & 0xffff], (v >> 16) & 0xff), &of);
      }
      const unsigned long long s2 = tot + acc;
      if (s2 < tot || (s2 >> 63) != 0ull) of = true;
      tot = s2;
      if (want_pick && acc != 0ull) {
        last = (unsigned long long)d1 | ((unsigned long long)d2 << 16);
        if (xc < tot) return last;
      }
    }
  }
  if (want_pick) return last;
  return of ? (tot | (1ull << 63)) : tot;
}

// The overflow check and the rewrite of the two-compartment (FUSION, PAIR) and
// depth-two (NESTED) rules, out of line (rare events; one copy shared by every
// lane-group width).  ctx is the grandchild slot (NESTED) or d1 | d2 << 16
// (FUSION: the lower slot keeps the merged compartment, the higher is freed
// and its children move to the survivor; PAIR: d1 takes the first
// compartment pattern's changes, d2 the second's, both stay).
template <class CT>
__device__ __noinline__ int cwc_general_check(const CT* content, const CT* wrap, const int32_t* meta, int S,
                                              int C, const int32_t* table, const int32_t* rec, int ctx) {
  auto fits = [](long long v) { return v >= 0 && v <= count_max<CT>(); };
  const int nr = rec[CR_NREAC];
  if (rec[CR_KIND] == RK_NESTED || rec[CR_KIND] == RK_PAIR) {
    // five multisets rewritten in place: NESTED's grandparent content, child
    // wrap and content, grandchild wrap and content; PAIR's parent content
    // and both children's wraps and contents
    const bool pair = rec[CR_KIND] == RK_PAIR;
    const int g = pair ? (ctx >> 16) : ctx, qq = pair ? (ctx & 0xffff) : (meta[g] >> 8) - 1,
              aa = (meta[qq] >> 8) - 1;
    const int32_t* xr = table + (rec[CR_GRAND] >> 8);
    const CT* ms[5] = {content + (size_t)aa * S, wrap + (size_t)qq * S, content + (size_t)qq * S,
                       wrap + (size_t)g * S, content + (size_t)g * S};
    const int nd[5] = {rec[CR_ND0], rec[CR_ND1], rec[CR_ND2], xr[XR_ND3], xr[XR_ND4]};
    const int32_t* dd[5] = {rec + CR_D0, rec + CR_D1, rec + CR_D2, xr + XR_D3, xr + XR_D4};
    for (int row = 0; row < 5; ++row)
      for (int d = 0; d < nd[row]; ++d) {
        const int v = dd[row][d];
        if (!fits((long long)ms[row][v & 0xffff] + (v >> 16))) return count_overflow_status<CT>();
      }
    return TS_OK;
  }
  const int d1 = ctx & 0xffff, d2 = ctx >> 16;
  const int qq = (meta[d1] >> 8) - 1;
  for (int d = 0; d < rec[CR_ND0]; ++d) {
    const int v = rec[CR_D0 + d];
    if (!fits((long long)content[(size_t)qq * S + (v & 0xffff)] + (v >> 16))) return count_overflow_status<CT>();
  }
  for (int x = 0; x < S; ++x) {
    long long wv = (long long)wrap[(size_t)d1 * S + x] + wrap[(size_t)d2 * S + x];
    long long cv = (long long)content[(size_t)d1 * S + x] + content[(size_t)d2 * S + x];
    for (int a = 0; a < nr; ++a) {
      const int v = rec[CR_REAC + a];
      const int row = (v >> 24) & 7;
      if ((v & 0xffff) != x) continue;
      if (row == 1 || row == 3) wv -= (v >> 16) & 0xff;
      if (row == 2 || row == 4) cv -= (v >> 16) & 0xff;
    }
    for (int d = 0; d < rec[CR_ND1]; ++d)
      if ((rec[CR_D1 + d] & 0xffff) == x) wv += rec[CR_D1 + d] >> 16;
    for (int d = 0; d < rec[CR_ND2]; ++d)
      if ((rec[CR_D2 + d] & 0xffff) == x) cv += rec[CR_D2 + d] >> 16;
    if (!fits(wv) || !fits(cv)) return count_overflow_status<CT>();
  }
  return TS_OK;
}

// O = L*S content totals, (L-1)*S wrap totals, L alive counts (see kernel)
template <class CT>
__device__ __noinline__ void cwc_general_apply(CT* content, CT* wrap, int32_t* meta,
                                               unsigned long long* chmask, unsigned long long* labmask,
                                               unsigned long long* alive_p, long long* tot, int S, int L, int C,
                                               const int32_t* table, const int32_t* rec, int ctx) {
  auto OC = [&](int l, int x) { return l * S + x; };
  auto OW = [&](int l, int x) { return L * S + (l - 1) * S + x; };
  auto OA = [&](int l) { return L * S + (L - 1) * S + l; };
  if (rec[CR_KIND] == RK_NESTED || rec[CR_KIND] == RK_PAIR) {
    // (PAIR: qq = the first child, g = the second, aa = their parent)
    const bool pair = rec[CR_KIND] == RK_PAIR;
    const int g = pair ? (ctx >> 16) : ctx, qq = pair ? (ctx & 0xffff) : (meta[g] >> 8) - 1,
              aa = (meta[qq] >> 8) - 1;
    const int la = meta[aa] & 0xff, lq = meta[qq] & 0xff, lg = meta[g] & 0xff;
    const int32_t* xr = table + (rec[CR_GRAND] >> 8);
    CT* ms[5] = {content + (size_t)aa * S, wrap + (size_t)qq * S, content + (size_t)qq * S,
                 wrap + (size_t)g * S, content + (size_t)g * S};
    const int nd[5] = {rec[CR_ND0], rec[CR_ND1], rec[CR_ND2], xr[XR_ND3], xr[XR_ND4]};
    const int32_t* dd[5] = {rec + CR_D0, rec + CR_D1, rec + CR_D2, xr + XR_D3, xr + XR_D4};
    for (int row = 0; row < 5; ++row)
      for (int d = 0; d < nd[row]; ++d) {
        const int v = dd[row][d];
        const int x = v & 0xffff, dv = v >> 16;
        ms[row][x] += dv;
        const int o = row == 0 ? OC(la, x) : row == 1 ? OW(lq, x) : row == 2 ? OC(lq, x) : row == 3 ? OW(lg, x) : OC(lg, x);
        tot[o] += dv;
      }
    return;
  }
  const int d1 = ctx & 0xffff, d2 = ctx >> 16;
  const int keep = d1 < d2 ? d1 : d2, gone = d1 < d2 ? d2 : d1;
  const int qq = (meta[d1] >> 8) - 1;
  const int lq = meta[qq] & 0xff, lc = meta[d1] & 0xff;
  const int nr = rec[CR_NREAC];
  for (int d = 0; d < rec[CR_ND0]; ++d) {
    const int v = rec[CR_D0 + d];
    content[(size_t)qq * S + (v & 0xffff)] += v >> 16;
    tot[OC(lq, v & 0xffff)] += v >> 16;
  }
  for (int x = 0; x < S; ++x) {
    int dw = 0, dc = 0;   // change of the label totals: - matched atoms + added atoms
    for (int a = 0; a < nr; ++a) {
      const int v = rec[CR_REAC + a];
      const int row = (v >> 24) & 7;
      if ((v & 0xffff) != x) continue;
      if (row == 1 || row == 3) dw -= (v >> 16) & 0xff;
      if (row == 2 || row == 4) dc -= (v >> 16) & 0xff;
    }
    for (int d = 0; d < rec[CR_ND1]; ++d)
      if ((rec[CR_D1 + d] & 0xffff) == x) dw += rec[CR_D1 + d] >> 16;
    for (int d = 0; d < rec[CR_ND2]; ++d)
      if ((rec[CR_D2 + d] & 0xffff) == x) dc += rec[CR_D2 + d] >> 16;
    wrap[(size_t)keep * S + x] = wrap[(size_t)keep * S + x] + wrap[(size_t)gone * S + x] + dw;
    content[(size_t)keep * S + x] = content[(size_t)keep * S + x] + content[(size_t)gone * S + x] + dc;
    wrap[(size_t)gone * S + x] = 0;
    content[(size_t)gone * S + x] = 0;
    tot[OW(lc, x)] += dw;
    tot[OC(lc, x)] += dc;
  }
  tot[OA(lc)] -= 1;
  unsigned long long kids = chmask[gone];
  while (kids) {
    const int e = __ffsll((long long)kids) - 1;
    kids &= kids - 1ull;
    meta[e] = (meta[e] & 0xff) | ((keep + 1) << 8);
  }
  chmask[keep] |= chmask[gone];
  chmask[gone] = 0ull;
  chmask[qq] &= ~(1ull << gone);
  labmask[lc] &= ~(1ull << gone);
  *alive_p &= ~(1ull << gone);
  meta[gone] = 0;
}

// With lane groups a warp holds 8 or 4 terms on different paths and runs
// those paths one after another, so its instruction footprint is the sum of
// theirs; instruction fetch was the first stall reason.  The count sums, the
// grid-point record and the rewrite check are therefore kept out of line for
// lane groups (one copy each, shared by every path that calls them): 2.0e8 ->
// 3.4e8 events/s with 4 lanes per term on 16,384 terms.  One lane per term
// keeps them inline, which measured faster there; an out-of-line Philox or
// rewrite measured slower.

// Observables of one grid point: lane gl of a group writes o = gl, gl + step, ...
__device__ __noinline__ void cwc_record_rows(const long long* tot, int32_t* dst, unsigned long long* sdst,
                                            unsigned long long* qdst, int O, int gl, int step) {
  for (int o = gl; o < O; o += step) {
    const long long v = tot[o];
    const int32_t sv = v > 0x7FFFFFFFll ? 0x7FFFFFFF : (int32_t)v;
    if (dst) dst[o] = sv;
    if (sdst) atomicAdd(sdst + o, (unsigned long long)(long long)sv);
    if (qdst) add_square_u128(qdst + 2 * o, sv);
  }
}

// Whether the rewrite of rule `rec` at context c fits (TS_OK), else its
// status; reads only (the in-line version is apply_check in the kernel).
template <class CT>
__device__ __noinline__ int cwc_apply_check(const CT* content, const CT* wrap, const int32_t* meta,
                                            unsigned long long alive, int S, int C, const int32_t* rec, int c) {
  const unsigned long long* alive_p = &alive;
  auto PARENT = [&](int cc) -> int { return (meta[cc] >> 8) - 1; };
  auto fits_add = [](int v, int d) -> bool {
    const long long s = (long long)v + d;
    return s >= 0 && s <= count_max<CT>();
  };
  const int OVF = count_overflow_status<CT>();
    const int kind = rec[CR_KIND];
    const int nd0 = rec[CR_ND0], nd1 = rec[CR_ND1], nd2 = rec[CR_ND2];
    if (kind == 0 || kind == 2) {
      if (kind == 2) {
        const unsigned long long freeslots = ~*alive_p & ~1ull & (C >= 64 ? ~0ull : ((1ull << C) - 1ull));
        if (freeslots == 0ull) return TS_CAPACITY;
      }
      const CT* x = content + (size_t)c * S;
      for (int d = 0; d < nd0; ++d) {
        const int v = rec[CR_D0 + d];
        if (!fits_add(x[v & 0xffff], v >> 16)) return OVF;
      }
      return TS_OK;
    }
    const int qq = PARENT(c);
    const CT* xp = content + (size_t)qq * S;
    const CT* w = wrap + (size_t)c * S;
    const CT* xc = content + (size_t)c * S;
    if (kind == 1) {
      for (int d = 0; d < nd0; ++d) {
        const int v = rec[CR_D0 + d];
        if (!fits_add(xp[v & 0xffff], v >> 16)) return OVF;
      }
      for (int d = 0; d < nd1; ++d) {
        const int v = rec[CR_D1 + d];
        if (!fits_add(w[v & 0xffff], v >> 16)) return OVF;
      }
      for (int d = 0; d < nd2; ++d) {
        const int v = rec[CR_D2 + d];
        if (!fits_add(xc[v & 0xffff], v >> 16)) return OVF;
      }
      return TS_OK;
    }
    // DISSOLVE: the parent content gains (rhs0 - lhs0) + (wrap - lhs1) + (content - lhs2)
    for (int s = 0; s < S; ++s) {
      long long dv = (long long)w[s] + xc[s];
      for (int d = 0; d < nd0; ++d) {
        const int v = rec[CR_D0 + d];
        if ((v & 0xffff) == s) dv += v >> 16;
      }
      const int nr = rec[CR_NREAC];
      for (int a = 0; a < nr; ++a) {
        const int v = rec[CR_REAC + a];
        if (((v >> 24) & 7) != 0 && (v & 0xffff) == s) dv -= (v >> 16) & 0xff;
      }
      const long long nv = (long long)xp[s] + dv;
      if (nv < 0 || nv > count_max<CT>()) return OVF;
    }
    return TS_OK;
}

// kGen: the model has FUSION or NESTED rules (a separate instantiation, so
// that the code of those kinds costs the other models no registers)
template <int kL, bool kQueue, bool kSens, bool kGen, class CT>
__global__ void __launch_bounds__(256) cwc_ssa_kernel(const __grid_constant__ CwcParams prm,
                                                      const __grid_constant__ LogConstants lc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const LaneGroup<kL> grp;
  const int gl = grp.gl;
  const int T = blockDim.x;
  const int NT = T / kL;                 // trajectories per block
  const int ts = threadIdx.x / kL;       // this group's trajectory column
  const int tid = threadIdx.x;
  const int S = prm.S, L = prm.L, C = prm.C, M = prm.M, B = prm.B, G = prm.G, O = prm.O;

  int32_t* s_rules = reinterpret_cast<int32_t*>(smem);
  int32_t* s_deps = s_rules + M * CWC_RULE_WORDS;
  const int tbl_words = M * CWC_RULE_WORDS + prm.n_deps;
  double* dbase = reinterpret_cast<double*>(smem + prm.smem_table_bytes);
  double* leaf = dbase + ts;                                      // [32][NT]
  double* node = dbase + 32 * NT + ts;                            // [31][NT]
  unsigned long long* Hs = reinterpret_cast<unsigned long long*>(dbase + (32 + TREE_NODES) * NT) + ts;  // [M][NT]

#define LEAF(l) leaf[(l) * NT]
#define NODE(i) node[(i) * NT]
#define HV(i) Hs[(i) * NT]

  unsigned long long* s_rj = reinterpret_cast<unsigned long long*>(smem + ((tbl_words * 4 + 15) / 16) * 16);
  unsigned long long* s_tj = s_rj + 64;
  for (int i = tid; i < tbl_words; i += T) s_rules[i] = prm.rules[i];
  for (int i = tid; i < 64; i += T) {
    s_rj[i] = lc.rj[i];
    s_tj[i] = lc.tj[i];
  }
  bool bad_grid = false;
  for (int g = tid; g < G; g += T) {
    const double v = prm.grid[g];
    if ((dbits(v) & 0x7FF0000000000000ll) == 0x7FF0000000000000ll) bad_grid = true;
    if (g == 0 && !(v >= 0.0)) bad_grid = true;
    if (g > 0 && !(v > prm.grid[g - 1])) bad_grid = true;
  }
  __shared__ unsigned long long s_deadline;
  if (tid == 0) {
    unsigned long long dl = ~0ull;
    if (prm.deadline_ns > 0) {
      const unsigned long long now = globaltimer_ns();
      unsigned long long start = now;
      if (prm.ws != nullptr) {
        const unsigned long long prev = atomicCAS(&prm.ws->t_start_ns, 0ull, now);
        start = prev == 0ull ? now : prev;
      }
      dl = start + (unsigned long long)prm.deadline_ns;
    }
    s_deadline = dl;
  }
  bad_grid = __syncthreads_or(bad_grid);
  const unsigned long long deadline = s_deadline;
  const long long T_bits = dbits(prm.grid[G - 1]);

  // this group's slab of the term
  const long long gslot = (long long)blockIdx.x * NT + ts;
  int32_t* slab = prm.slabs + gslot * prm.slab_words;
  unsigned long long* chmask = reinterpret_cast<unsigned long long*>(slab);       // [C]
  unsigned long long* labmask = chmask + C;                                       // [L]
  unsigned long long* alive_p = labmask + L;                                      // [1]
  long long* tot = reinterpret_cast<long long*>(alive_p + 1);                     // [O]
  // score replay: int_0^t H_i dt up to tl_i, tl_i, the partials, firings N_i
  double* Iac = reinterpret_cast<double*>(tot + O);                               // [M]
  double* tl = Iac + (kSens ? M : 0);                                             // [M]
  double* part = tl + (kSens ? M : 0);                                            // [M]
  int32_t* Nf = reinterpret_cast<int32_t*>(part + (kSens ? M : 0));               // [M]
  int32_t* meta = Nf + (kSens ? M : 0);                                           // [C]
  CT* wrap = reinterpret_cast<CT*>(meta + C);                                                       // [C][S]
  CT* content = wrap + (size_t)C * S;                                        // [C][S]

  auto LABEL = [&](int c) -> int { return meta[c] & 0xff; };
  auto PARENT = [&](int c) -> int { return (meta[c] >> 8) - 1; };

  long long q = 0;
  int p = 0, r = 0;
  const double* kp = nullptr;
  double t = 0.0;
  unsigned int n = 0;
  unsigned int n_launch = 0;   // n when this launch took the trajectory up
  int gi = 0;
  long long gbits = 0;
  unsigned long long h = FNV_OFFSET;
  bool ovf = false;
  int status = TS_OK;
  const long long Q = prm.Q;
  bool first = true;

  // combinatorial count of rule i at context slot c (c is the context for
  // LOCAL / CREATE, the child for PARENT_CHILD / DISSOLVE).  The reactants
  // are stored by pattern row, then species, so one pass multiplies in the
  // oracle's order: row 0 (the context's or the parent's content), row 1
  // (the child's wrap), row 2 (the child's content).
  // (kinds LOCAL .. DISSOLVE; NESTED counts go through cwc_count_sum)
  auto count_at = [&](const int32_t* rec, int c) -> unsigned long long {
    const int kind = rec[CR_KIND];
    const CT* x0 = content + (size_t)((kind == RK_LOCAL || kind == RK_CREATE) ? c : PARENT(c)) * S;
    const CT* x1 = wrap + (size_t)c * S;
    const CT* x2 = content + (size_t)c * S;
    const int nr = rec[CR_NREAC];
    unsigned long long acc = 1ull;
    for (int a = 0; a < nr; ++a) {
      const int v = rec[CR_REAC + a];
      const int row = (v >> 24) & 3;
      const CT* x = row == 0 ? x0 : (row == 1 ? x1 : x2);
      acc = mul_checked(acc, binom12(x[v & 0xffff], (v >> 16) & 0xff), &ovf);
    }
    return acc;
  };
  // candidate contexts of rule i, in ascending slot order (FUSION, PAIR: the
  // slots its pairs are drawn from)
  auto ctx_mask = [&](const int32_t* rec) -> unsigned long long {
    const int kind = rec[CR_KIND];
    if (kGen && kind == RK_NESTED) return labmask[rec[CR_GRAND] & 0xff];
    return (kind == RK_LOCAL || kind == RK_CREATE) ? labmask[rec[CR_CTX]] : labmask[rec[CR_CHILD]];
  };
  auto ctx_ok = [&](const int32_t* rec, int c) -> bool {
    const int kind = rec[CR_KIND];
    if (kind == RK_LOCAL || kind == RK_CREATE) return true;
    return LABEL(PARENT(c)) == rec[CR_CTX];
  };
  // sum of the counts of a rule over the contexts in m (ascending slots),
  // overflow-checked like a from-scratch H
  auto partial_h = [&](const int32_t* rec, unsigned long long m) -> unsigned long long {
    if (kL == 1 && !(kGen && rec[CR_KIND] == RK_NESTED)) {
      unsigned long long tot = 0ull;
      while (m) {
        const int c = __ffsll((long long)m) - 1;
        m &= m - 1ull;
        if (!ctx_ok(rec, c)) continue;
        const unsigned long long hc = count_at(rec, c);
        const unsigned long long s2 = tot + hc;
        if (s2 < tot || (s2 >> 63) != 0ull) ovf = true;
        tot = s2;
      }
      return tot;
    }
    const unsigned long long r = (kGen && rec[CR_KIND] == RK_NESTED) ? cwc_count_sum_nested(content, wrap, meta, S, rec, m)
                                                                    : cwc_count_sum(content, wrap, meta, S, rec, m);
    if (r >> 63) ovf = true;
    return r;
  };
  // H_i from scratch: sum over all its contexts
  auto total_h = [&](int i) -> unsigned long long {
    const int32_t* rec = s_rules + i * CWC_RULE_WORDS;
    if (kGen && (rec[CR_KIND] == RK_FUSION || rec[CR_KIND] == RK_PAIR)) {
      const unsigned long long r = cwc_fusion_scan(content, wrap, meta, S, rec, ctx_mask(rec), false, 0ull);
      if (r >> 63) ovf = true;
      return r & ~(1ull << 63);
    }
    return partial_h(rec, ctx_mask(rec));
  };
  auto prop_of = [&](int i) -> double { return __dmul_rn(kp[i], u63_to_double_rn(HV(i))); };
  auto leaf_sum = [&](int l) -> double {
    const int j0 = l * B, j1 = min(j0 + B, M);
    double s = j0 < M ? prop_of(j0) : 0.0;
    for (int jj = j0 + 1; jj < j1; ++jj) s = __dadd_rn(s, prop_of(jj));
    return s;
  };
  auto node_val = [&](int nd) -> double {
    const double a = nd < 16 ? LEAF(2 * nd) : NODE(2 * nd - 32);
    const double b = nd < 16 ? LEAF(2 * nd + 1) : NODE(2 * nd - 31);
    return __dadd_rn(a, b);
  };
  // leaves over the lanes, then the internal nodes by every lane in order
  // (each lane writes the values every other lane writes)
  auto rebuild_tree = [&]() {
    for (int l = gl; l < 32; l += kL) LEAF(l) = B == 1 ? (l < M ? prop_of(l) : 0.0) : leaf_sum(l);
    grp.sync();
    for (int nd = 0; nd < TREE_NODES; ++nd) NODE(nd) = node_val(nd);
    grp.sync();
  };

  // observable index of the content / wrap total of (label, species) and of the alive count
  auto OC = [&](int l, int x) { return l * S + x; };
  auto OW = [&](int l, int x) { return L * S + (l - 1) * S + x; };
  auto OA = [&](int l) { return L * S + (L - 1) * S + l; };

  auto record = [&](int g) {
    int32_t* dst = prm.states != nullptr ? prm.states + ((size_t)q * G + g) * O : nullptr;
    unsigned long long* sdst = prm.sums != nullptr ? prm.sums + ((size_t)p * G + g) * O : nullptr;
    unsigned long long* qdst = prm.sumsq != nullptr ? prm.sumsq + ((size_t)p * G + g) * O * 2 : nullptr;
    if (kL > 1) {
      cwc_record_rows(tot, dst, sdst, qdst, O, gl, kL);
    } else {
      for (int o = gl; o < O; o += kL) {
        const long long v = tot[o];
        const int32_t sv = v > 0x7FFFFFFFll ? 0x7FFFFFFF : (int32_t)v;
        if (dst) dst[o] = sv;
        if (sdst) atomicAdd(sdst + o, (unsigned long long)(long long)sv);
        if (qdst) add_square_u128(qdst + 2 * o, sv);
      }
    }
    if (kSens) {
      const double* gm = prm.grad_means + ((size_t)p * G + g) * O;
      const double* mm = prm.means + ((size_t)p * G + g) * O;
      double cg = 0.0;
      for (int o = gl; o < O; o += kL) {
        const long long v = tot[o];
        const int32_t sv = v > 0x7FFFFFFFll ? 0x7FFFFFFF : (int32_t)v;
        cg = __dadd_rn(cg, __dmul_rn(gm[o], __dadd_rn((double)sv, -mm[o])));
      }
      cg = grp.sum(cg);
      const double gt = prm.grid[g];
      for (int i = gl; i < M; i += kL) {
        const double Ig = __dadd_rn(Iac[i], __dmul_rn(u63_to_double_rn(HV(i)), __dadd_rn(gt, -tl[i])));
        const double Si = __dadd_rn(__ddiv_rn((double)Nf[i], kp[i]), -Ig);
        part[i] = __dadd_rn(part[i], __dmul_rn(cg, Si));
      }
    }
  };
  auto fill = [&]() {
    for (; gi < G; ++gi) record(gi);
  };

  const int W = 3 + 2 * S;   // slot image row: alive, label, parent, wrap[S], content[S]
  auto finalize = [&]() {
    // (a 16-bit launch saves only the trajectories handed to the 32-bit one;
    // every other record gets its status, which the 32-bit launch reads)
    if (prm.ckpt != nullptr && sizeof(CT) == 2 && status != TS_TIMEOUT) {
      if (gl == 0) prm.ckpt[(size_t)q * (CKPT_HEADER_WORDS + (size_t)C * W) + 6] = status;
    } else if (prm.ckpt != nullptr) {
      int32_t* rec = prm.ckpt + (size_t)q * (CKPT_HEADER_WORDS + (size_t)C * W);
      if (gl == 0) {
        put_f64(rec, t);
        put_u64(rec + 2, h);
        rec[4] = (int32_t)n;
        rec[5] = gi;
        rec[6] = status;
        rec[7] = 0;
      }
      const unsigned long long alive = *alive_p;
      for (int c = gl; c < C; c += kL) {
        int32_t* row = rec + CKPT_HEADER_WORDS + (size_t)c * W;
        const bool a = (alive >> c) & 1ull;
        row[0] = a ? 1 : 0;
        row[1] = a ? LABEL(c) : 0;
        row[2] = a ? PARENT(c) : -1;
        for (int x = 0; x < S; ++x) {
          row[3 + x] = wrap[(size_t)c * S + x];
          row[3 + S + x] = content[(size_t)c * S + x];
        }
      }
    }
    if (gl == 0) {
      if (prm.traj_status) prm.traj_status[q] = status;
      if (prm.traj_events) prm.traj_events[q] = (long long)n;
      if (prm.traj_hash) prm.traj_hash[q] = h;
      if (prm.traj_final_t) prm.traj_final_t[q] = t;
    }
    if (kSens)
      for (int i = gl; i < M; i += kL) prm.partials[(size_t)q * M + i] = part[i];
    grp.sync();   // the slab is reused by the next trajectory
  };
  // fold H_i's contribution since tl_i into the integral before H_i changes
  auto integrate = [&](int i, double tnow) {
    Iac[i] = __dadd_rn(Iac[i], __dmul_rn(u63_to_double_rn(HV(i)), __dadd_rn(tnow, -tl[i])));
    tl[i] = tnow;
  };

  // load and validate the initial term (slot image; on resume the saved one),
  // build masks, H and tree.  0 = running, 1 = ended at once (bad input),
  // 2 = nothing to do (resuming, and this trajectory did not stop on the deadline),
  // 3 = a count of the initial term does not fit a 16-bit term: the image is
  // saved for the 32-bit launch as a trajectory that has not started
  auto start = [&]() -> int {
    p = (int)(q / prm.R);
    r = (int)(q - (long long)p * prm.R);
    kp = prm.rates + (size_t)p * M;
    t = 0.0;
    n = 0u;
    gi = 0;
    gbits = dbits(prm.grid[0]);
    h = FNV_OFFSET;
    ovf = false;
    status = TS_OK;
    bool bad = bad_grid;
    for (int j = gl; j < M; j += kL) {
      const long long kb = dbits(kp[j]);
      if (!(kb > 0 && kb < 0x7FF0000000000000ll)) bad = true;
    }
    if (kSens) {
      for (int i = gl; i < M; i += kL) {
        Iac[i] = 0.0;
        tl[i] = 0.0;
        part[i] = 0.0;
        Nf[i] = 0;
      }
    }
    const int32_t* img = prm.init + (size_t)(prm.Pi == 1 ? 0 : p) * C * W;
    if (prm.resume) {
      const int32_t* rec = prm.ckpt + (size_t)q * (CKPT_HEADER_WORDS + (size_t)C * W);
      if (rec[6] != TS_TIMEOUT) return 2;
      t = get_f64(rec);
      h = get_u64(rec + 2);
      n = (unsigned)rec[4];
      gi = rec[5];
      if (gi < 0 || gi > G) bad = true;
      gbits = gi < G && gi >= 0 ? dbits(prm.grid[gi]) : 0;
      img = rec + CKPT_HEADER_WORDS;
    }
    unsigned long long alive = 0ull;
    bool wide = false;   // a count above count_max<CT>() (16-bit terms only)
    for (int c = gl; c < C; c += kL) {
      chmask[c] = 0ull;
      const int32_t* row = img + (size_t)c * W;
      const int a = row[0];
      if (a != 0 && a != 1) bad = true;
      if (a == 1) {
        const int lab = row[1], par = row[2];
        if (c == 0 && (lab != 0 || par != -1)) bad = true;
        if (c > 0 && (lab < 1 || lab >= L || par < 0 || par >= C)) bad = true;
        for (int x = 0; x < S; ++x) {
          const int wv = row[3 + x], cv = row[3 + S + x];
          if (wv < 0 || cv < 0) bad = true;
          if (c == 0 && wv != 0) bad = true;
          if (wv > count_max<CT>() || cv > count_max<CT>()) wide = true;
          wrap[(size_t)c * S + x] = (CT)wv;
          content[(size_t)c * S + x] = (CT)cv;
        }
        alive |= 1ull << c;
        meta[c] = (lab & 0xff) | ((par + 1) << 8);
      } else {
        meta[c] = 0;
        for (int x = 0; x < S; ++x) {
          wrap[(size_t)c * S + x] = 0;
          content[(size_t)c * S + x] = 0;
        }
      }
    }
    alive = grp.or_all(alive);
    if (!(alive & 1ull)) bad = true;
    grp.sync();
    bad = grp.any(bad);
    if (!bad) {
      // every alive slot's parent chain reaches the root through alive slots
      for (int c = 1 + gl; c < C; c += kL) {
        if (!((alive >> c) & 1ull)) continue;
        int qq = c, steps = 0;
        while (qq != 0) {
          qq = PARENT(qq);
          if (qq < 0 || qq >= C || !((alive >> qq) & 1ull) || ++steps > C) {
            bad = true;
            break;
          }
        }
      }
      bad = grp.any(bad);
    }
    if (bad) {
      status = TS_BAD_INPUT;
      if (prm.states != nullptr) {
        int32_t* dst = prm.states + (size_t)q * G * O;
        for (long long e = gl; e < (long long)G * O; e += kL) dst[e] = 0;
      }
      if (gl == 0) *alive_p = 0ull;
      grp.sync();
      return 1;
    }
    if (sizeof(CT) == 2 && grp.any(wide)) {
      int32_t* rec = prm.ckpt + (size_t)q * (CKPT_HEADER_WORDS + (size_t)C * W);
      if (gl == 0) {
        put_f64(rec, 0.0);
        put_u64(rec + 2, FNV_OFFSET);
        rec[4] = 0;
        rec[5] = 0;
        rec[6] = TS_TIMEOUT;
        rec[7] = 0;
        *alive_p = 0ull;
      }
      for (long long e = gl; e < (long long)C * W; e += kL) rec[CKPT_HEADER_WORDS + e] = img[e];
      grp.sync();
      return 3;
    }
    if (gl == 0) {
      *alive_p = alive;
      for (int l = 0; l < L; ++l) labmask[l] = 0ull;
      for (int c = 0; c < C; ++c) {
        if (!((alive >> c) & 1ull)) continue;
        labmask[LABEL(c)] |= 1ull << c;
        if (c > 0) chmask[PARENT(c)] |= 1ull << c;
      }
    }
    for (int o = gl; o < O; o += kL) tot[o] = 0;
    grp.sync();
    for (int x = gl; x < S; x += kL) {
      for (int c = 0; c < C; ++c) {
        if (!((alive >> c) & 1ull)) continue;
        const int l = LABEL(c);
        tot[OC(l, x)] += content[(size_t)c * S + x];
        if (l > 0) tot[OW(l, x)] += wrap[(size_t)c * S + x];
      }
    }
    if (gl == 0) {
      for (int c = 0; c < C; ++c)
        if ((alive >> c) & 1ull) tot[OA(LABEL(c))] += 1;
    }
    for (int i = gl; i < M; i += kL) HV(i) = total_h(i);
    ovf = grp.any(ovf);
    grp.sync();
    rebuild_tree();
    return 0;
  };

  auto fits_add = [](int v, int d) -> bool {
    const long long s = (long long)v + d;
    return s >= 0 && s <= count_max<CT>();
  };

  // whether the rewrite of rule j at context c fits (TS_OK), else its status
  // (a count leaving CT's range: INT_OVERFLOW, or TS_WIDEN for 16-bit
  // terms); nothing is changed
  auto apply_check = [&](const int32_t* rec, int c) -> int {
    const int kind = rec[CR_KIND];
    const int nd0 = rec[CR_ND0], nd1 = rec[CR_ND1], nd2 = rec[CR_ND2];
    if (kind == 0 || kind == 2) {
      if (kind == 2) {
        const unsigned long long freeslots = ~*alive_p & ~1ull & (C >= 64 ? ~0ull : ((1ull << C) - 1ull));
        if (freeslots == 0ull) return TS_CAPACITY;
      }
      const CT* x = content + (size_t)c * S;
      for (int d = 0; d < nd0; ++d) {
        const int v = rec[CR_D0 + d];
        if (!fits_add(x[v & 0xffff], v >> 16)) return count_overflow_status<CT>();
      }
      return TS_OK;
    }
    const int qq = PARENT(c);
    const CT* xp = content + (size_t)qq * S;
    const CT* w = wrap + (size_t)c * S;
    const CT* xc = content + (size_t)c * S;
    if (kind == 1) {
      for (int d = 0; d < nd0; ++d) {
        const int v = rec[CR_D0 + d];
        if (!fits_add(xp[v & 0xffff], v >> 16)) return count_overflow_status<CT>();
      }
      for (int d = 0; d < nd1; ++d) {
        const int v = rec[CR_D1 + d];
        if (!fits_add(w[v & 0xffff], v >> 16)) return count_overflow_status<CT>();
      }
      for (int d = 0; d < nd2; ++d) {
        const int v = rec[CR_D2 + d];
        if (!fits_add(xc[v & 0xffff], v >> 16)) return count_overflow_status<CT>();
      }
      return TS_OK;
    }
    // DISSOLVE: the parent content gains (rhs0 - lhs0) + (wrap - lhs1) + (content - lhs2)
    for (int s = 0; s < S; ++s) {
      long long dv = (long long)w[s] + xc[s];
      for (int d = 0; d < nd0; ++d) {
        const int v = rec[CR_D0 + d];
        if ((v & 0xffff) == s) dv += v >> 16;
      }
      const int nr = rec[CR_NREAC];
      for (int a = 0; a < nr; ++a) {
        const int v = rec[CR_REAC + a];
        if (((v >> 24) & 7) != 0 && (v & 0xffff) == s) dv -= (v >> 16) & 0xff;
      }
      const long long nv = (long long)xp[s] + dv;
      if (nv < 0 || nv > count_max<CT>()) return count_overflow_status<CT>();
    }
    return TS_OK;
  };

  // the rewrite of rule j at context c, after apply_check accepted it (one lane)
  auto apply = [&](const int32_t* rec, int c) {
    const int kind = rec[CR_KIND];
    const int nd0 = rec[CR_ND0], nd1 = rec[CR_ND1], nd2 = rec[CR_ND2];
    if (kind == 0) {
      CT* x = content + (size_t)c * S;
      const int l = LABEL(c);
      for (int d = 0; d < nd0; ++d) {
        const int v = rec[CR_D0 + d];
        x[v & 0xffff] += v >> 16;
        tot[OC(l, v & 0xffff)] += v >> 16;
      }
      return;
    }
    if (kind == 1) {
      const int qq = PARENT(c);
      CT* xp = content + (size_t)qq * S;
      CT* w = wrap + (size_t)c * S;
      CT* xc = content + (size_t)c * S;
      const int lq = LABEL(qq), lc = LABEL(c);
      for (int d = 0; d < nd0; ++d) {
        const int v = rec[CR_D0 + d];
        xp[v & 0xffff] += v >> 16;
        tot[OC(lq, v & 0xffff)] += v >> 16;
      }
      for (int d = 0; d < nd1; ++d) {
        const int v = rec[CR_D1 + d];
        w[v & 0xffff] += v >> 16;
        tot[OW(lc, v & 0xffff)] += v >> 16;
      }
      for (int d = 0; d < nd2; ++d) {
        const int v = rec[CR_D2 + d];
        xc[v & 0xffff] += v >> 16;
        tot[OC(lc, v & 0xffff)] += v >> 16;
      }
      return;
    }
    if (kind == 2) {
      const unsigned long long alive = *alive_p;
      const unsigned long long freeslots = ~alive & ~1ull & (C >= 64 ? ~0ull : ((1ull << C) - 1ull));
      const int e = __ffsll((long long)freeslots) - 1;
      CT* x = content + (size_t)c * S;
      const int lctx = LABEL(c);
      for (int d = 0; d < nd0; ++d) {
        const int v = rec[CR_D0 + d];
        x[v & 0xffff] += v >> 16;
        tot[OC(lctx, v & 0xffff)] += v >> 16;
      }
      CT* we = wrap + (size_t)e * S;
      CT* xe = content + (size_t)e * S;
      for (int s = 0; s < S; ++s) {
        we[s] = 0;
        xe[s] = 0;
      }
      for (int d = 0; d < nd1; ++d) {
        const int v = rec[CR_D1 + d];
        we[v & 0xffff] = v >> 16;
      }
      for (int d = 0; d < nd2; ++d) {
        const int v = rec[CR_D2 + d];
        xe[v & 0xffff] = v >> 16;
      }
      const int lab = rec[CR_CHILD];
      for (int d = 0; d < nd1; ++d) {
        const int v = rec[CR_D1 + d];
        tot[OW(lab, v & 0xffff)] += v >> 16;
      }
      for (int d = 0; d < nd2; ++d) {
        const int v = rec[CR_D2 + d];
        tot[OC(lab, v & 0xffff)] += v >> 16;
      }
      tot[OA(lab)] += 1;
      meta[e] = lab | ((c + 1) << 8);
      chmask[e] = 0ull;
      chmask[c] |= 1ull << e;
      labmask[lab] |= 1ull << e;
      *alive_p = alive | (1ull << e);
      return;
    }
    // DISSOLVE: matched atoms rewritten, the rest of the wrap and content go
    // to the parent, children are reparented, the slot is freed
    {
      const int qq = PARENT(c);
      CT* xp = content + (size_t)qq * S;
      CT* w = wrap + (size_t)c * S;
      CT* xc = content + (size_t)c * S;
      // per-species change of the parent content: (rhs0 - lhs0) + (w - lhs1) + (xc - lhs2)
      auto delta_at = [&](int s) -> long long {
        long long dv = (long long)w[s] + xc[s];
        for (int d = 0; d < nd0; ++d) {
          const int v = rec[CR_D0 + d];
          if ((v & 0xffff) == s) dv += v >> 16;
        }
        const int nr = rec[CR_NREAC];
        for (int a = 0; a < nr; ++a) {
          const int v = rec[CR_REAC + a];
          const int row = (v >> 24) & 7;
          if (row != 0 && (v & 0xffff) == s) dv -= (v >> 16) & 0xff;
        }
        return dv;
      };
      const int lq = LABEL(qq), ld = LABEL(c);
      for (int s = 0; s < S; ++s) {
        const long long dv = delta_at(s);
        xp[s] = (CT)((long long)xp[s] + dv);
        tot[OC(lq, s)] += dv;
        tot[OC(ld, s)] -= xc[s];
        tot[OW(ld, s)] -= w[s];
      }
      tot[OA(ld)] -= 1;
      unsigned long long kids = chmask[c];
      while (kids) {
        const int e = __ffsll((long long)kids) - 1;
        kids &= kids - 1ull;
        meta[e] = (meta[e] & 0xff) | ((qq + 1) << 8);
      }
      chmask[qq] = (chmask[qq] | chmask[c]) & ~(1ull << c);
      chmask[c] = 0ull;
      labmask[LABEL(c)] &= ~(1ull << c);
      *alive_p &= ~(1ull << c);
      meta[c] = 0;
      for (int s = 0; s < S; ++s) {
        w[s] = 0;
        xc[s] = 0;
      }
    }
  };

  // context of rule `rec` for the integer draw xc in [0, H_j): the first
  // context, in ascending slot order, whose running count exceeds xc
  auto choose_context = [&](const int32_t* rec, unsigned long long xc) -> int {
    const unsigned long long m = ctx_mask(rec);
    int ctx = -1, lastc = -1;
    if (kL == 1 && !(kGen && rec[CR_KIND] == RK_NESTED)) {
      unsigned long long mm = m, cum = 0ull;
      while (mm) {
        const int c = __ffsll((long long)mm) - 1;
        mm &= mm - 1ull;
        if (!ctx_ok(rec, c)) continue;
        const unsigned long long hc = count_at(rec, c);
        if (hc == 0ull) continue;
        lastc = c;
        cum += hc;
        if (xc < cum) {
          ctx = c;
          break;
        }
      }
    } else {
      // rounds of kL consecutive slots, lane k taking slot r0 + k: a group
      // prefix sum over the round gives every lane its running count
      unsigned long long base = 0ull;
      for (int r0 = 0; r0 < C; r0 += kL) {
        const unsigned long long rm = (m >> r0) & ((1ull << kL) - 1ull);
        if (rm == 0ull) continue;
        const int c = r0 + gl;
        unsigned long long hc = 0ull;
        if ((rm >> gl) & 1ull) {
          hc = (kGen && rec[CR_KIND] == RK_NESTED) ? cwc_count_sum_nested(content, wrap, meta, S, rec, 1ull << c)
                                                   : cwc_count_sum(content, wrap, meta, S, rec, 1ull << c);
          if (hc >> 63) ovf = true;
          hc &= ~(1ull << 63);
        }
        const unsigned long long incl = grp.incl_scan(hc);
        const unsigned nz = grp.ballot(hc != 0ull);
        const unsigned hit = grp.ballot(hc != 0ull && xc < base + incl);
        if (nz) lastc = r0 + (31 - __clz((int)nz));
        if (hit) {
          ctx = r0 + __ffs((int)hit) - 1;
          break;
        }
        base += grp.bcast(incl, kL - 1);
      }
    }
    if (ctx < 0) ctx = lastc;
    if (ctx < 0) ctx = 0;  // unreachable: H_j > 0 has a context with h > 0
    return ctx;
  };

  // one event or the end of the trajectory: 0 = running, 1 = ended with grid
  // points left to fill, 2 = ended with the grid complete (or left to a resume)
  auto step = [&]() -> int {
    // the same order of checks as the written specification: overflow of a
    // count or of a0 first, then the event cap, then absorption.  On overflow
    // the score's integrals stop at the last applied event (time t) and H
    // counts as 0 after it; the lazily kept integrals are first brought up to t.
    const double a0 = NODE(TREE_ROOT);
    const long long a0b = dbits(a0);
    if (ovf || a0b >= 0x7FF0000000000000ll) {
      status = TS_PROP_OVERFLOW;
      if (kSens)
        for (int i = gl; i < M; i += kL) {
          integrate(i, t);
          HV(i) = 0ull;
        }
      grp.sync();
      return 1;
    }
    if ((long long)n == prm.max_events) {
      status = TS_EVENT_LIMIT;
      return 1;
    }
    if (a0b == 0) {
      status = TS_ABSORBED;
      return 1;
    }
    // the deadline is read every 1024 events, never before a trajectory has
    // applied 1024 events in this launch, so every launch makes progress
    if ((n & 1023u) == 0u && n != n_launch && deadline != ~0ull) {
      const bool late = grp.bcast(gl == 0 ? globaltimer_ns() > deadline : false, 0);
      if (late) {
        status = TS_TIMEOUT;
        return prm.ckpt == nullptr ? 1 : 2;   // with a checkpoint the rest is recorded on resume
      }
    }
    const uint32_t rr = (uint32_t)r + prm.r_offset;
    // both draws of the event (purpose 0: time and rule; 1: context) from one
    // copy of the Philox rounds: the smaller loop body leaves more of the
    // instruction cache to the rest of the step (+2 % events/s on 16,384
    // terms of 48 rules)
    uint4 w = make_uint4(0u, 0u, 0u, 0u), w1 = w;
#pragma unroll 1
    for (uint32_t pu = 0; pu < 2u; ++pu) {
      const uint4 v = philox4x32_10(make_uint4(n, pu, rr, (uint32_t)p), prm.key0, prm.key1);
      if (pu == 0u) w = v; else w1 = v;
    }
    const double u_tau = uniform52(w.x, w.y);
    const double u_sel = uniform52(w.z, w.w);
    const double tau = __ddiv_rn(-log_spec_q(u_tau, lc, s_rj, s_tj), a0);
    const double tn = __dadd_rn(t, tau);
    const long long tnb = dbits(tn);
    while (gi < G && gbits < tnb) {
      record(gi);
      ++gi;
      if (gi < G) gbits = dbits(prm.grid[gi]);
    }
    if (tnb > T_bits) {
      status = TS_OK;
      return 2;
    }
    // 1. rule: guarded descent of x = u_sel * a0
    double x = __dmul_rn(u_sel, a0);
    int nd = TREE_ROOT;
#pragma unroll
    for (int lvl = 5; lvl >= 2; --lvl) {
      const double Lv = NODE(2 * nd - 32);
      const double Rv = NODE(2 * nd - 31);
      const bool left = dbits(x) < dbits(Lv) || dbits(Rv) == 0;
      const double xr = __dadd_rn(x, -Lv);
      x = left ? x : xr;
      nd = left ? 2 * nd - 32 : 2 * nd - 31;
    }
    int l;
    {
      const double Lv = LEAF(2 * nd);
      const double Rv = LEAF(2 * nd + 1);
      const bool left = dbits(x) < dbits(Lv) || dbits(Rv) == 0;
      const double xr = __dadd_rn(x, -Lv);
      x = left ? x : xr;
      l = left ? 2 * nd : 2 * nd + 1;
    }
    int j;
    if (B == 1) {
      j = l;
    } else {
      const int j0 = l * B, j1 = min(j0 + B, M);
      int last = -1;
      j = -1;
      double s = 0.0;
      for (int jj = j0; jj < j1; ++jj) {
        if (HV(jj) != 0ull) {
          const double a = prop_of(jj);
          s = last < 0 ? a : __dadd_rn(s, a);
          last = jj;
          if (dbits(x) < dbits(s)) {
            j = jj;
            break;
          }
        }
      }
      if (j < 0) j = last;
    }
    j = min(max(j, 0), M - 1);
    const int32_t* rec = s_rules + j * CWC_RULE_WORDS;
    // 2. context: integer draw xc in [0, H_j)
    const unsigned long long Wd = (unsigned long long)w1.x | ((unsigned long long)w1.y << 32);
    const unsigned long long xc = __umul64hi(Wd, HV(j));
    const int ctx = (kGen && (rec[CR_KIND] == RK_FUSION || rec[CR_KIND] == RK_PAIR))
                        ? (int)cwc_fusion_scan(content, wrap, meta, S, rec, ctx_mask(rec), true, xc)
                        : choose_context(rec, xc);
    // 3. update.  Only contexts in `touched` can change their counts: the
    // rewritten compartments, their children (which read the parent content),
    // and the free slots (one of which CREATE fills).  Each dependent rule
    // drops the old counts of its touched contexts and adds the new ones; a
    // rule whose contexts all lie in `touched` is summed afresh.
    const bool general_j = kGen && (rec[CR_KIND] == RK_FUSION || rec[CR_KIND] == RK_NESTED || rec[CR_KIND] == RK_PAIR);
    const int ast = general_j ? cwc_general_check(content, wrap, meta, S, C, s_rules, rec, ctx)
                    : kL > 1  ? cwc_apply_check(content, wrap, meta, *alive_p, S, C, rec, ctx)
                              : apply_check(rec, ctx);
    if (ast != TS_OK) {
      if (ast == TS_WIDEN) {
        // a 16-bit count would leave its range: the event is not applied
        // here; the trajectory is saved as it stands (grid points recorded so
        // far included) and the 32-bit launch redraws this same event
        status = TS_TIMEOUT;
        return 2;
      }
      status = ast;
      return 1;
    }
    const int kind_j = rec[CR_KIND];
    // FUSION, NESTED and PAIR events touch every slot (every dependent is recounted)
    unsigned long long touched = general_j ? ~0ull : chmask[ctx];
    if (kind_j == RK_LOCAL || kind_j == RK_CREATE) {
      touched |= 1ull << ctx;
      if (kind_j == RK_CREATE) touched |= ~*alive_p & ~1ull & (C >= 64 ? ~0ull : ((1ull << C) - 1ull));
    } else if (!general_j) {
      const int qq = PARENT(ctx);
      touched |= (1ull << qq) | chmask[qq];
    }
    if (kSens && gl == 0) Nf[j] += 1;
    const int doff = rec[CR_DEPOFF], dcnt = rec[CR_DEPCNT];
    // FUSION, NESTED and PAIR dependents, whose contexts are pairs or
    // grandchildren rather than the touched slots, are recounted in full
    // after the rewrite
    auto general_rule = [&](const int32_t* ri) {
      return kGen && (ri[CR_KIND] == RK_FUSION || ri[CR_KIND] == RK_NESTED || ri[CR_KIND] == RK_PAIR);
    };
    for (int e = gl; e < dcnt; e += kL) {
      const int i = s_deps[doff + e];
      const int32_t* ri = s_rules + i * CWC_RULE_WORDS;
      if (kSens) integrate(i, tn);
      const unsigned long long cm = ctx_mask(ri);
      HV(i) = general_rule(ri) || (cm & ~touched) == 0ull ? 0ull : HV(i) - partial_h(ri, cm & touched);
    }
    grp.sync();
    if (gl == 0) {
      if (kGen && general_j)
        cwc_general_apply(content, wrap, meta, chmask, labmask, alive_p, tot, S, L, C, s_rules, rec, ctx);
      else
        apply(rec, ctx);
    }
    grp.sync();
    for (int e = gl; e < dcnt; e += kL) {
      const int i = s_deps[doff + e];
      const int32_t* ri = s_rules + i * CWC_RULE_WORDS;
      const unsigned long long s2 = general_rule(ri) ? total_h(i) : HV(i) + partial_h(ri, ctx_mask(ri) & touched);
      if ((s2 >> 63) != 0ull) ovf = true;
      HV(i) = s2;
    }
    ovf = grp.any(ovf);
    grp.sync();
    if (B == 1) {
      for (int e = gl; e < dcnt; e += kL) {
        const int i = s_deps[doff + e];
        LEAF(i) = prop_of(i);
      }
    } else {
      unsigned lm = (unsigned)rec[CR_LEAFMASK];
      for (int k = 0; lm; ++k) {
        const int ll = __ffs(lm) - 1;
        lm &= lm - 1u;
        if ((k & (kL - 1)) == gl) LEAF(ll) = leaf_sum(ll);
      }
    }
    grp.sync();
    unsigned nm = (unsigned)rec[CR_NODEMASK];
    while (nm) {
      const int k = __ffs(nm) - 1;
      nm &= nm - 1u;
      NODE(k) = node_val(k);
    }
    if (gl == 0 && prm.log_cap > 0 && n < (unsigned)prm.log_cap) {
      const size_t at = (size_t)q * prm.log_cap + n;
      prm.log_rule[at] = j;
      if (prm.log_slot) prm.log_slot[at] = ctx;
      if (prm.log_t) prm.log_t[at] = tn;
    }
    t = tn;
    ++n;
    h = fnv1a_event(h, (uint32_t)j, (uint32_t)ctx);
    grp.sync();
    return 0;
  };

  bool need_new = true;
  bool done = false;   // no trajectories left for this group (it stays in the loop with its warp)
  for (;;) {
    // every lane group of the warp starts its step together, so that the
    // groups' common instructions (draw, logarithm, descent) issue once for
    // the warp (+2 % events/s on 16,384 terms of 48 rules)
    __syncwarp();
    if (!done) {
      if (need_new) {
        if (kQueue) {
          if (kL == 1) {
            q = cwc_grab_next(prm.ws);
          } else {
            long long v = 0;
            if (gl == 0) v = (long long)atomicAdd(&prm.ws->queue_next, 1ull);
            q = grp.bcast(v, 0);
          }
        } else {
          q = first ? gslot : q + (long long)gridDim.x * NT;
          first = false;
        }
        if (q >= Q) {
          done = true;
        } else {
          const int st0 = start();
          if (st0 == 1) finalize();
          if (st0 == 0) {
            n_launch = n;
            need_new = false;
          }
        }
      } else {
        const int ended = step();
        if (ended != 0) {
          if (ended == 1) fill();
          finalize();
          need_new = true;
        }
      }
    }
    if (__all_sync(0xffffffffu, done)) break;
  }
#undef LEAF
#undef NODE
#undef HV
}

// ---------------------------------------------------------------------------

template <int kL, bool kQueue, bool kSens, bool kGen, class CT>
static cudaError_t cwc_config_t(const CwcParams& prm, int T, int* blocks_out, size_t* smem_out) {
  auto kern = cwc_ssa_kernel<kL, kQueue, kSens, kGen, CT>;
  const size_t smem = (size_t)prm.smem_table_bytes + (size_t)(T / kL) * cwc_thread_bytes(prm.M);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long blocks = (long long)sms * per_sm;
  const long long per_block = T / kL;
  const long long need = (prm.Q + per_block - 1) / per_block;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  *blocks_out = (int)blocks;
  *smem_out = smem;
  return cudaSuccess;
}

// 16-bit terms (prm.narrow) exist for the forward of models without
// FUSION / NESTED / PAIR rules only
template <int kL, bool kGen>
static cudaError_t cwc_config_g(const CwcParams& prm, bool queue, int T, int* blocks, size_t* smem) {
  const bool sens = prm.sens != 0;
  if constexpr (!kGen) {
    if (prm.narrow && !sens)
      return queue ? cwc_config_t<kL, true, false, false, int16_t>(prm, T, blocks, smem)
                   : cwc_config_t<kL, false, false, false, int16_t>(prm, T, blocks, smem);
  }
  if (queue)
    return sens ? cwc_config_t<kL, true, true, kGen, int32_t>(prm, T, blocks, smem)
                : cwc_config_t<kL, true, false, kGen, int32_t>(prm, T, blocks, smem);
  return sens ? cwc_config_t<kL, false, true, kGen, int32_t>(prm, T, blocks, smem)
              : cwc_config_t<kL, false, false, kGen, int32_t>(prm, T, blocks, smem);
}

template <int kL>
static cudaError_t cwc_config_l(const CwcParams& prm, bool queue, int T, int* blocks, size_t* smem) {
  return prm.general ? cwc_config_g<kL, true>(prm, queue, T, blocks, smem)
                     : cwc_config_g<kL, false>(prm, queue, T, blocks, smem);
}

static cudaError_t cwc_config(const CwcParams& prm, bool queue, int lanes, int T, int* blocks, size_t* smem) {
  if (T < 32 || T > 256 || T % 32 != 0) return cudaErrorInvalidValue;
  switch (lanes) {
    case 1: return cwc_config_l<1>(prm, queue, T, blocks, smem);
    case 4: return cwc_config_l<4>(prm, queue, T, blocks, smem);
    case 8: return cwc_config_l<8>(prm, queue, T, blocks, smem);
    default: return cudaErrorInvalidValue;
  }
}

bool cwc_lanes_supported(int lanes) { return lanes == 1 || lanes == 4 || lanes == 8; }

// Launch shape (threads per block, blocks): both layouts use a grid of at most
// the resident capacity, so the term slabs number resident groups, not
// trajectories.
cudaError_t cwc_launch_shape(const CwcParams& prm, bool queue, int lanes, int T, int* blocks) {
  size_t smem = 0;
  return cwc_config(prm, queue, lanes, T, blocks, &smem);
}

// Threads per block giving the most resident warps.
int cwc_best_threads(const CwcParams& prm, bool queue, int lanes) {
  int best_T = 32, best_warps = -1;
  for (int T = 32; T <= 256; T += 32) {
    const size_t smem = (size_t)prm.smem_table_bytes + (size_t)(T / lanes) * cwc_thread_bytes(prm.M);
    if (smem > 227 * 1024) break;
    int blocks = 0;
    size_t sm = 0;
    CwcParams big = prm;
    big.Q = 1ll << 40;   // resident capacity, not the batch
    if (cwc_config(big, queue, lanes, T, &blocks, &sm) != cudaSuccess) break;
    const int warps = blocks * T / 32;
    if (warps >= best_warps) {
      best_warps = warps;
      best_T = T;
    }
  }
  return best_T;
}

int cwc_table_bytes_host(int M, int n_deps) { return cwc_table_bytes(M, n_deps); }
int cwc_thread_bytes_host(int M) { return cwc_thread_bytes(M); }
long long cwc_slab_words_host(int S, int L, int C, int M, bool sens) { return cwc_slab_words(S, L, C, M, sens); }

template <int kL, bool kGen>
static void cwc_launch_g(const CwcParams& prm, const LogConstants& lc, bool queue, int T, int blocks, size_t smem,
                         cudaStream_t stream) {
  const bool sens = prm.sens != 0;
  if constexpr (!kGen) {
    if (prm.narrow && !sens) {
      if (queue)
        cwc_ssa_kernel<kL, true, false, false, int16_t><<<(unsigned)blocks, T, smem, stream>>>(prm, lc);
      else
        cwc_ssa_kernel<kL, false, false, false, int16_t><<<(unsigned)blocks, T, smem, stream>>>(prm, lc);
      return;
    }
  }
  if (queue) {
    if (sens)
      cwc_ssa_kernel<kL, true, true, kGen, int32_t><<<(unsigned)blocks, T, smem, stream>>>(prm, lc);
    else
      cwc_ssa_kernel<kL, true, false, kGen, int32_t><<<(unsigned)blocks, T, smem, stream>>>(prm, lc);
  } else {
    if (sens)
      cwc_ssa_kernel<kL, false, true, kGen, int32_t><<<(unsigned)blocks, T, smem, stream>>>(prm, lc);
    else
      cwc_ssa_kernel<kL, false, false, kGen, int32_t><<<(unsigned)blocks, T, smem, stream>>>(prm, lc);
  }
}

template <int kL>
static void cwc_launch_l(const CwcParams& prm, const LogConstants& lc, bool queue, int T, int blocks, size_t smem,
                         cudaStream_t stream) {
  if (prm.general)
    cwc_launch_g<kL, true>(prm, lc, queue, T, blocks, smem, stream);
  else
    cwc_launch_g<kL, false>(prm, lc, queue, T, blocks, smem, stream);
}

cudaError_t launch_cwc(const CwcParams& prm, const LogConstants& lc, bool queue, int lanes, int T, int blocks,
                       cudaStream_t stream) {
  size_t smem = 0;
  int b = 0;
  cudaError_t e = cwc_config(prm, queue, lanes, T, &b, &smem);
  if (e != cudaSuccess) return e;
  if (blocks > b) return cudaErrorInvalidConfiguration;   // the slabs were sized for at most b blocks
  switch (lanes) {
    case 1: cwc_launch_l<1>(prm, lc, queue, T, blocks, smem, stream); break;
    case 4: cwc_launch_l<4>(prm, lc, queue, T, blocks, smem, stream); break;
    case 8: cwc_launch_l<8>(prm, lc, queue, T, blocks, smem, stream); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace cwcgpu
