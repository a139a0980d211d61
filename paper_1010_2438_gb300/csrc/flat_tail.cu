// The tail of a batch of flat-network trajectories of uneven length (the
// uneven parameter sweeps of Sec. 5.2): a group of lanes per trajectory.
//
// One thread per trajectory is the efficient layout while tens of thousands
// of trajectories share the GPU, but once the work queue is empty the makespan
// is set by the longest trajectories, each a chain of up to ~1e6 sequential
// events at one lane's latency.  The thread-per-trajectory kernel therefore
// hands its last trajectories over (layout CWC_LAYOUT_TAIL): when the queue is
// exhausted and at most `handoff` trajectories are still running, each of them
// stops at its next 1024-event boundary and saves its state in the checkpoint
// record.  The kernels here then
//   1. collect the handed-over trajectories and predict each one's remaining
//      events from its own progress so far, n (T - t) / t (events per unit of
//      simulated time observed in the first part of the run, times the time
//      left to the horizon T),
//   2. order them longest-predicted-first, and
//   3. finish them with a group of kG lanes each, which cuts the per-event
//      latency:
//        - the group's lanes draw the Philox words and compute the uniforms
//          and logarithms of its next 32 events at once (32 / kG each), so
//          the integer work that dominates one lane's event is spread out;
//        - each lane owns 32 / kG leaves of the 32-lane blocked tree and the
//          nodes above them inside the lane, and recomputes the leaves the
//          fired rule dirtied;
//        - the levels above are rebuilt with xor butterflies across the group
//          (every lane of a pair adds the same two values; IEEE addition is
//          commutative, so each node equals the written tree's left + right);
//        - the guarded descent reads a node's children from the lanes that
//          hold them (shuffles); every lane walks it identically;
//        - grid records write the counts lane by lane.
// Every arithmetic step is the thread kernel's, in the same order, so the
// results are identical bit for bit whichever kernel finishes a trajectory.
#include <cuda_runtime.h>

#include "cwc_internal.h"
#include "ssa_device.cuh"

namespace cwcgpu {

// 1. handed-over trajectories (checkpoint status TIMEOUT) into list[] with
// their predicted remaining events
__global__ void tail_collect_kernel(const __grid_constant__ FlatParams prm, int32_t* __restrict__ list,
                                    double* __restrict__ est) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= prm.Q) return;
  const int32_t* rec = prm.ckpt + (size_t)q * (prm.S + CKPT_HEADER_WORDS);
  if (rec[6] != TS_TIMEOUT) return;
  const double t = get_f64(rec);
  const double n = (double)(unsigned)rec[4];
  const double T = prm.grid[prm.G - 1];
  const double e = t > 0.0 ? n * (T - t) / t : n;
  const unsigned long long i = atomicAdd(&prm.ws->tail_count, 1ull);
  list[i] = (int32_t)q;
  est[i] = e;
}

// 2. longest predicted first (ties: lower trajectory index first); a rank
// count over the collected entries (a few hundred to a few thousand)
__global__ void tail_rank_kernel(const __grid_constant__ FlatParams prm, const int32_t* __restrict__ list,
                                 const double* __restrict__ est, int32_t* __restrict__ order) {
  const unsigned long long K = prm.ws->tail_count;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < K;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const double e = est[i];
    const int32_t q = list[i];
    unsigned long long rank = 0;
    for (unsigned long long k = 0; k < K; ++k) {
      const double f = est[k];
      rank += (f > e) || (f == e && list[k] < q);
    }
    order[rank] = q;
  }
}

// 3. a group of kG lanes (8, 16 or 32) per handed-over trajectory, resumed
// from its checkpoint.  Lane gl of the group owns the LPL = 32 / kG leaves
// gl*LPL .. gl*LPL + LPL - 1 and the tree nodes above them inside the lane;
// the upper log2(kG) levels are built by xor butterflies across the group.
template <int kG>
__global__ void __launch_bounds__(128) flat_group_kernel(const __grid_constant__ FlatParams prm,
                                                         const __grid_constant__ LogConstants lc,
                                                         const int32_t* __restrict__ order) {
  constexpr int LPL = 32 / kG;                              // leaves per lane
  constexpr int LG = LPL == 4 ? 2 : (LPL == 2 ? 1 : 0);     // tree levels inside a lane
  constexpr int KG = 5 - LG;                                // tree levels across the group
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int gl = lane & (kG - 1);
  const unsigned gmask = kG == 32 ? 0xffffffffu : (((1u << kG) - 1u) << (lane & ~(kG - 1)));
  const int S = prm.S, M = prm.M, B = prm.B, G = prm.G;
  int32_t* cnt = reinterpret_cast<int32_t*>(smem) + (size_t)(threadIdx.x / kG) * S;   // this group's counts
  const int32_t* __restrict__ g_rules = prm.rules;
  const int32_t* __restrict__ g_deps = g_rules + M * RULE_WORDS;
  const uint32_t* __restrict__ g_desc = reinterpret_cast<const uint32_t*>(g_deps + prm.n_deps);
  const int tbl_words = M * RULE_WORDS + prm.n_deps + M;
  const unsigned long long* __restrict__ g_rj =
      reinterpret_cast<const unsigned long long*>(g_rules + ((tbl_words + 3) & ~3));
  const unsigned long long* __restrict__ g_tj = g_rj + 64;
  const bool checked = prm.checked_counts != 0;
  const long long T_bits = dbits(prm.grid[G - 1]);
  const unsigned long long K = prm.ws->tail_count;
  auto any = [&](bool v) { return (__ballot_sync(gmask, v) & gmask) != 0u; };

  bool ovf = false;
  // H_i at the current counts (the thread kernel's count_h)
  auto count_h = [&](int i) -> unsigned long long {
    if (!checked) {
      const uint32_t d = g_desc[i];
      const uint32_t kind = d & 3u;
      const unsigned n0 = (unsigned)cnt[(d >> 2) & 0x3fffu];
      const unsigned n1 = (unsigned)cnt[(d >> 16) & 0x3fffu];
      const unsigned m = kind == 3u ? n1 : (kind == 2u ? n0 - 1u : 1u);
      const unsigned long long prod = (unsigned long long)(kind == 0u ? 1u : n0) * m;
      return kind == 2u ? prod >> 1 : prod;
    }
    const int32_t* rec = g_rules + i * RULE_WORDS;
    const int nr = rec[R_NREAC];
    unsigned long long hh = 1ull;
    for (int a = 0; a < nr; ++a) {
      const int v = rec[R_REAC + a];
      hh = mul_checked(hh, binom12(cnt[v & 0xffff], v >> 16), &ovf);
    }
    return hh;
  };

  for (;;) {
    unsigned long long it = 0;
    if (gl == 0) it = atomicAdd(&prm.ws->tail_next, 1ull);
    it = __shfl_sync(gmask, it, 0, kG);
    if (it >= K) break;
    const long long q = order[it];
    const int p = (int)(q / prm.R);
    const int r = (int)(q - (long long)p * prm.R);
    const double* kp = prm.rates + (size_t)p * M;
    int32_t* ck = prm.ckpt + (size_t)q * (S + CKPT_HEADER_WORDS);
    double t = get_f64(ck);
    unsigned long long h = get_u64(ck + 2);
    unsigned n = (unsigned)ck[4];
    int gi = ck[5];
    for (int s = gl; s < S; s += kG) cnt[s] = ck[CKPT_HEADER_WORDS + s];
    __syncwarp(gmask);
    ovf = false;
    auto prop_of = [&](int i) -> double { return __dmul_rn(kp[i], u63_to_double_rn(count_h(i))); };
    auto leaf_sum = [&](int l) -> double {
      const int j0 = l * B, j1 = min(j0 + B, M);
      double s = j0 < M ? prop_of(j0) : 0.0;
      for (int jj = j0 + 1; jj < j1; ++jj) s = __dadd_rn(s, prop_of(jj));
      return s;
    };
    // lf: this lane's leaves; a1 / a2: its level-1 / level-2 nodes (LPL = 4, 2);
    // up[k]: its ancestor at level LG + 1 + k (up[KG - 1] = a0 on every lane)
    double lf[LPL], a1[2], a2 = 0.0, up[KG];
#pragma unroll
    for (int k = 0; k < LPL; ++k) lf[k] = leaf_sum(gl * LPL + k);
    a1[0] = a1[1] = 0.0;
    auto local_top = [&]() -> double { return LPL == 4 ? a2 : (LPL == 2 ? a1[0] : lf[0]); };
    auto rebuild = [&]() {
      if (LPL == 4) {
        a1[0] = __dadd_rn(lf[0], lf[1]);
        a1[1] = __dadd_rn(lf[2 % LPL], lf[3 % LPL]);
        a2 = __dadd_rn(a1[0], a1[1]);
      } else if (LPL == 2) {
        a1[0] = __dadd_rn(lf[0], lf[1 % LPL]);
      }
      double v = local_top();
#pragma unroll
      for (int k = 0; k < KG; ++k) {
        v = __dadd_rn(v, __shfl_xor_sync(gmask, v, 1 << k, kG));
        up[k] = v;
      }
    };
    rebuild();
    ovf = any(ovf);
    long long gbits = gi < G ? dbits(prm.grid[gi]) : 0;
    int status = TS_OK;

    // observables of grid point g, spread over the group's lanes
    auto record = [&](int g) {
      if (prm.states != nullptr) {
        int32_t* dst = prm.states + ((size_t)q * G + g) * S;
        for (int s = gl; s < S; s += kG) dst[s] = cnt[s];
      }
      if (prm.sums != nullptr) {
        unsigned long long* dst = prm.sums + ((size_t)p * G + g) * S;
        for (int s = gl; s < S; s += kG) atomicAdd(dst + s, (unsigned long long)(long long)cnt[s]);
      }
      if (prm.sumsq != nullptr) {
        unsigned long long* dst = prm.sumsq + ((size_t)p * G + g) * S * 2;
        for (int s = gl; s < S; s += kG) add_square_u128(dst + 2 * s, cnt[s]);
      }
    };

    // the next 32 events' random numbers: lane gl holds events n0 + gl + kG*s
    unsigned n0 = n;
    double myL[LPL], myU[LPL];
    auto draw = [&]() {
      n0 = n;
#pragma unroll
      for (int s2 = 0; s2 < LPL; ++s2) {
        const uint4 w = philox4x32_10(make_uint4(n0 + (unsigned)(gl + kG * s2), 0u, (uint32_t)r + prm.r_offset,
                                                 (uint32_t)p), prm.key0, prm.key1);
        myU[s2] = uniform52(w.z, w.w);
        myL[s2] = -log_spec_q(uniform52(w.x, w.y), lc, g_rj, g_tj);
      }
    };
    draw();

    bool fill_rest = true;
    for (;;) {
      const double a0 = up[KG - 1];
      const long long a0b = dbits(a0);
      if (ovf || a0b >= 0x7FF0000000000000ll) {
        status = TS_PROP_OVERFLOW;
        break;
      }
      if ((long long)n == prm.max_events) {
        status = TS_EVENT_LIMIT;
        break;
      }
      if (a0b == 0) {
        status = TS_ABSORBED;
        break;
      }
      if (n - n0 >= 32u) draw();
      const int ev = (int)(n - n0);
      const int slot = ev / kG;
      double Lsel = myL[0], Usel = myU[0];
#pragma unroll
      for (int s2 = 1; s2 < LPL; ++s2)
        if (slot == s2) {
          Lsel = myL[s2];
          Usel = myU[s2];
        }
      const double Lk = __shfl_sync(gmask, Lsel, ev & (kG - 1), kG);
      const double u_sel = __shfl_sync(gmask, Usel, ev & (kG - 1), kG);
      const double tau = __ddiv_rn(Lk, a0);
      const double tn = __dadd_rn(t, tau);
      const long long tnb = dbits(tn);
      while (gi < G && gbits < tnb) {
        record(gi);
        ++gi;
        if (gi < G) gbits = dbits(prm.grid[gi]);
      }
      if (tnb > T_bits) {
        status = TS_OK;
        fill_rest = false;
        break;
      }
      // guarded descent of x = u_sel * a0 (the same on every lane of the group)
      double x = __dmul_rn(u_sel, a0);
      int i = 0;
      auto descend = [&](double Lv, double Rv) {
        const bool left = dbits(x) < dbits(Lv) || dbits(Rv) == 0;
        const double xr = __dadd_rn(x, -Lv);
        x = left ? x : xr;
        i = 2 * i + (left ? 0 : 1);
      };
      // across lanes: node i at level L has its children at level L-1 on lanes
      // (2i) << (L-1-LG) and (2i+1) << (L-1-LG)
#pragma unroll
      for (int L = 5; L > LG; --L) {
        const int sh = L - 1 - LG;
        const double reg = (L - 1 == LG) ? local_top() : up[(L - 2 - LG) < 0 ? 0 : (L - 2 - LG)];
        descend(__shfl_sync(gmask, reg, (2 * i) << sh, kG), __shfl_sync(gmask, reg, (2 * i + 1) << sh, kG));
      }
      // inside the owning lane
      if (LPL == 4) {
        const int owner = i;
        descend(__shfl_sync(gmask, a1[0], owner, kG), __shfl_sync(gmask, a1[1], owner, kG));
        const bool hi = (i & 1) != 0;
        descend(__shfl_sync(gmask, hi ? lf[2 % LPL] : lf[0], owner, kG),
                __shfl_sync(gmask, hi ? lf[3 % LPL] : lf[1 % LPL], owner, kG));
      } else if (LPL == 2) {
        const int owner = i;
        descend(__shfl_sync(gmask, lf[0], owner, kG), __shfl_sync(gmask, lf[1 % LPL], owner, kG));
      }
      const int l = i;
      int j;
      if (B == 1) {
        j = l;
      } else {
        const int j0 = l * B, j1 = min(j0 + B, M);
        int last = -1;
        j = -1;
        double s = 0.0;
        for (int jj = j0; jj < j1; ++jj) {
          const unsigned long long hh = count_h(jj);
          if (hh != 0ull) {
            const double a = __dmul_rn(kp[jj], u63_to_double_rn(hh));
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
      // the stoichiometry change, checked first (nothing changes on overflow);
      // lane d handles change d (distinct species, at most 8 <= kG)
      const int32_t* rec = g_rules + j * RULE_WORDS;
      const int nd_ = rec[R_NDELTA];
      int sp = 0, dv = 0;
      if (gl < nd_) {
        const int v = rec[R_DELTA + gl];
        sp = v & 0xffff;
        dv = v >> 16;
      }
      if (any(gl < nd_ && dv > 0 && cnt[sp] > 0x7FFFFFFF - dv)) {
        status = TS_INT_OVERFLOW;
        break;
      }
      if (gl < nd_) cnt[sp] += dv;
      __syncwarp(gmask);
      // dirty leaves (the leaves of the fired rule's dependents), then the tree
      const unsigned lm = (unsigned)rec[R_LEAFMASK] >> (gl * LPL);
#pragma unroll
      for (int k = 0; k < LPL; ++k)
        if ((lm >> k) & 1u) lf[k] = leaf_sum(gl * LPL + k);
      ovf = any(ovf);
      rebuild();
      if (gl == 0 && prm.log_cap > 0 && n < (unsigned)prm.log_cap) {
        const size_t at = (size_t)q * prm.log_cap + n;
        prm.log_rule[at] = j;
        if (prm.log_slot) prm.log_slot[at] = 0;
        if (prm.log_t) prm.log_t[at] = tn;
      }
      t = tn;
      ++n;
      h = fnv1a_event(h, (uint32_t)j, 0u);
    }
    if (fill_rest)
      for (; gi < G; ++gi) record(gi);
    if (gl == 0) {
      put_f64(ck, t);
      put_u64(ck + 2, h);
      ck[4] = (int32_t)n;
      ck[5] = gi;
      ck[6] = status;
      if (prm.traj_status) prm.traj_status[q] = status;
      if (prm.traj_events) prm.traj_events[q] = (long long)n;
      if (prm.traj_hash) prm.traj_hash[q] = h;
      if (prm.traj_final_t) prm.traj_final_t[q] = t;
    }
    for (int s = gl; s < S; s += kG) ck[CKPT_HEADER_WORDS + s] = cnt[s];
    __syncwarp(gmask);   // the counts are reused by this group's next trajectory
  }
}

// lanes per handed-over trajectory
constexpr int kTailLanes = 16;

// Steps 1-3 on `stream` after the thread kernel's launch: list, est and order
// hold Q entries each (workspace).
cudaError_t launch_flat_tail(const FlatParams& prm, const LogConstants& lc, int32_t* list, double* est,
                             int32_t* order, cudaStream_t stream) {
  const long long Q = prm.Q;
  tail_collect_kernel<<<(unsigned)((Q + 255) / 256), 256, 0, stream>>>(prm, list, est);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  tail_rank_kernel<<<(unsigned)sms, 256, 0, stream>>>(prm, list, est, order);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  auto kern = flat_group_kernel<kTailLanes>;
  const size_t smem = (size_t)(128 / kTailLanes) * prm.S * sizeof(int32_t);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  // a resident grid; groups without a trajectory return at once
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  kern<<<(unsigned)(per_sm * sms), 128, smem, stream>>>(prm, lc, order);
  return cudaGetLastError();
}

}  // namespace cwcgpu
