// Flat mass-action networks (one compartment): Gillespie's direct method
// (Sec. 2.2) run by one thread per trajectory over replicas x sweep points
// (Sec. 5.2).
//
// Layout.  The compiled rule tables stay in global memory, read through L1
// (a few KB shared by every block, always resident there).  Shared memory
// holds only per-thread arrays stored [index][thread] with rows of T + 1
// elements, so that a warp's lanes reading their own elements, or several
// lanes reading rows of one column (the pooled leaf rounds), spread over banks.
//   leaf[32][Ts] double  leaves of the 32-lane blocked tree.  With B = 1 leaf
//                        l is a_l itself (l >= M: +0); with B > 1 it is the
//                        block sum and the a_j are recomputed from the counts
//                        when needed instead of being stored
//   node[16][Ts] double  level-1 tree nodes (children: leaves 2n, 2n+1); not
//                        kept by the Michaelis-Menten kernel, which sums them
//                        from the leaves where they are read
//   cnt[S][Ts]   int32   species counts
// and, in registers, the 15 upper nodes (levels 2-5, root = a0), which the
// descent selects among without a shared-memory round trip.  For the score
// replay H_i as doubles [M][Ts] joins shared memory.  The replay's integrals,
// their times, the firing counts and the partials, touched a few at a time
// per event, live in global memory per trajectory, so that the replay keeps
// almost the forward pass's residency.
// Keeping only the leaves, the level-1 nodes and the counts (384 + 4S bytes
// per trajectory) in shared memory, and no tables, is what lets 14 warps
// share an SM at S = 32: GB300's FP64 pipe (~1.6 lane-ops per clock per SM)
// has long latency, and hiding it needs resident warps.
//
// Per event the thread: draws Philox(n, 0, r, p); computes tau with the
// fixed integer logarithm and one IEEE division; records grid points passed;
// descends the tree (integer compares of non-negative doubles, one FP64
// subtraction per level); applies the stoichiometry change.  Then only the
// leaves holding a rule whose propensity reads a changed species (Gibson-
// Bruck dependency graph) are rebuilt — with B > 1 by the whole warp at once,
// every lane's dirty leaves dealt out over the lanes — and the level-1 nodes
// above them, then the 15 register nodes (a warp's lanes fire different
// rules, so between them they dirty every upper node anyway: all 15 in every
// warp-step of the 64-rule network's event logs).  a0 is always the tree
// root, never a running sum, so values equal a full rebuild bit for bit.
#include <cuda_runtime.h>

#include <cstdio>

#include "cwc_internal.h"
#include "ssa_device.cuh"

namespace cwcgpu {

__device__ __forceinline__ long long grab_next(WorkspaceHeader* ws) {
  const unsigned mask = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(&ws->queue_next, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return (long long)(base + (unsigned long long)__popc(mask & ((1u << lane) - 1u)));
}

// Shared memory set aside for tables: none.  The kernel reads the rules, the
// dependents, the reactant descriptors and the logarithm's 64 + 64 table
// words from the model's device table (layout in cwc_internal.h) through
// L1; in shared memory they cost the block two warps of residency at S = 32.
__host__ __device__ inline int flat_table_bytes(int M, int n_deps) {
  (void)M;
  (void)n_deps;
  return 0;
}

// (mm: the Michaelis-Menten kernel keeps no level-1 nodes, see the kernel)
__host__ __device__ inline int flat_thread_bytes(int S, int M, bool sens, bool mm) {
  int doubles = 32 + (mm ? 0 : 16) + (sens ? M : 0);
  int ints = S;
  return doubles * 8 + ints * 4;
}

// kTail: the tail layout's variant of the queue kernel, which counts finished
// trajectories and hands the last ones over (a separate instantiation: the
// bookkeeping, compiled into the plain queue kernel even behind a runtime
// flag, measured 2.25x slower on the 32-species network).
// kMM: models with Michaelis-Menten rules (a separate instantiation too, so
// that mass-action networks run the kernel without the rate-law lookups).
// kPool: B > 1 and events that dirty several leaves (chosen by the host from
// the model, prm.pool): the warp rebuilds its lanes' dirty leaves together
// (pooled_leaves); otherwise every lane rebuilds its own.
template <bool kQueue, bool kSens, bool kTail, bool kMM, bool kPool>
__global__ void __maxnreg__(168) flat_ssa_kernel(const __grid_constant__ FlatParams prm,
                                                       const __grid_constant__ LogConstants lc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int T = blockDim.x;
  const int tid = threadIdx.x;
  const int S = prm.S, M = prm.M, B = prm.B, G = prm.G;

  // model tables in global memory: rules, dependents, reactant descriptors,
  // then (16-byte aligned) the logarithm's rj and tj words
  const int32_t* __restrict__ g_rules = prm.rules;
  const int32_t* __restrict__ g_deps = g_rules + M * RULE_WORDS;
  const uint32_t* __restrict__ g_desc = reinterpret_cast<const uint32_t*>(g_deps + prm.n_deps);
  const int tbl_words = M * RULE_WORDS + prm.n_deps + M;
  // Per-thread arrays [index][T + 1]: each pointer below already points at
  // this thread's column, so element i of the array is ptr[i * Ts].  The
  // padded row (Ts = T + 1 elements; T is a multiple of 32) keeps a warp's
  // own-column accesses conflict-free and puts the rows of one column in
  // different banks, which the pooled leaf rounds need: there several lanes
  // read and write one owner's counts and leaves at once (with a row of T
  // elements they all hit the owner's bank).
  const int Ts = T + 1;
  double* dbase = reinterpret_cast<double*>(smem + prm.smem_table_bytes);
  // The Michaelis-Menten kernel stores no level-1 nodes: it sums them from
  // their two leaves where they are read (the descent, the register nodes),
  // which costs FP64 additions but 128 bytes of shared memory per
  // trajectory, so that 16 instead of 14 warps fit an SM; its leaves, with
  // their divisions, are dear enough that the residency wins (+13 % events/s
  // on the 40-rule cascade, against -7 % on the 64-rule mass-action network)
  constexpr bool kNodes = !kMM;
  constexpr int kNodeRows = kNodes ? 16 : 0;
  const int n_dbl_rows = 32 + kNodeRows + (kSens ? M : 0);
  double* leaf = dbase + tid;                                   // [32][Ts]
  double* node = dbase + 32 * Ts + tid;                         // [16][Ts] level-1 nodes (kNodes)
  double* Hd = dbase + (32 + kNodeRows) * Ts + tid;             // score replay only: [M][Ts]
  // score replay, per trajectory in global memory (set by start()):
  // V_i = N_i / k_i - I_i(t_i) + H_i t_i (t_i: the last change of rule i's
  // count or firings), so that the score at grid time t_g is S_i(g) =
  // V_i - H_i t_g: a change of H_i from h to h' at time t adds (h' - h) t, a
  // firing adds 1 / k_i.  (When 1 / k_i overflows, for subnormal k_i, the
  // firings are counted in Nf instead and S_i(g) adds N_i / k_i.)
  double* Vv = nullptr;     // [M]
  double* Nf = nullptr;     // [M] firings of rules whose 1 / k_i overflows
  double* part = nullptr;   // [M] the trajectory's partials
  const double* ik = nullptr;   // [M] 1 / k_i of this sweep point
  int32_t* ibase = reinterpret_cast<int32_t*>(dbase + (size_t)n_dbl_rows * Ts);
  int32_t* cnt = ibase + tid;                                   // [S][Ts]

#define LEAF(l) leaf[(l) * Ts]
#define NODE(i) (kNodes ? node[(i) * Ts] : __dadd_rn(LEAF(2 * (i)), LEAF(2 * (i) + 1)))
#define CNT(s) cnt[(s) * Ts]

  const unsigned long long* __restrict__ g_rj =
      reinterpret_cast<const unsigned long long*>(g_rules + ((tbl_words + 3) & ~3));
  const unsigned long long* __restrict__ g_tj = g_rj + 64;
  // grid check, once per block: finite, grid[0] >= 0, strictly increasing
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
  const bool vec_states = (S % 4 == 0) && ((reinterpret_cast<uintptr_t>(prm.states) & 15) == 0);
  const bool checked = prm.checked_counts != 0;

  // ---- trajectory state (registers) ----
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
  const long long qstride = (long long)gridDim.x * T;
  bool first = true;
  // upper tree nodes: level 2 (nodes 16..23), level 3 (24..27), level 4 (28,
  // 29) and the root (30) = a0.  Indexed with constants only, so they stay in
  // registers.
  double u2[8], u3[4], u4[2], root = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) u2[k] = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) u3[k] = 0.0;
  u4[0] = u4[1] = 0.0;

  // levels 2-5 from the level-1 nodes, each node the sum of its left and
  // right child
  auto rebuild_upper = [&]() {
#pragma unroll
    for (int k = 0; k < 8; ++k) u2[k] = __dadd_rn(NODE(2 * k), NODE(2 * k + 1));
#pragma unroll
    for (int k = 0; k < 4; ++k) u3[k] = __dadd_rn(u2[2 * k], u2[2 * k + 1]);
    u4[0] = __dadd_rn(u3[0], u3[1]);
    u4[1] = __dadd_rn(u3[2], u3[3]);
    root = __dadd_rn(u4[0], u4[1]);
  };

  // observables of the current term at grid point g
  auto record = [&](int g) {
    if (prm.states != nullptr) {
      int32_t* dst = prm.states + ((size_t)q * G + g) * S;
      if (vec_states) {
        for (int s = 0; s < S; s += 4)
          *reinterpret_cast<int4*>(dst + s) = make_int4(CNT(s), CNT(s + 1), CNT(s + 2), CNT(s + 3));
      } else {
        for (int s = 0; s < S; ++s) dst[s] = CNT(s);
      }
    }
    if (prm.sums != nullptr) {
      unsigned long long* dst = prm.sums + ((size_t)p * G + g) * S;
      for (int s = 0; s < S; ++s) atomicAdd(dst + s, (unsigned long long)(long long)CNT(s));
    }
    if (prm.sumsq != nullptr) {
      unsigned long long* dst = prm.sumsq + ((size_t)p * G + g) * S * 2;
      for (int s = 0; s < S; ++s) add_square_u128(dst + 2 * s, CNT(s));
    }
    if (kSens) {
      const double* gm = prm.grad_means + ((size_t)p * G + g) * S;
      const double* mm = prm.means + ((size_t)p * G + g) * S;
      double c = 0.0;
      for (int o = 0; o < S; ++o)
        c = __dadd_rn(c, __dmul_rn(gm[o], __dadd_rn((double)CNT(o), -mm[o])));
      const double gt = prm.grid[g];
      // S_i(g) = V_i - H_i t_g (+ N_i / k_i when 1 / k_i overflows); two rules
      // per iteration, loads first, so that their latencies overlap
      auto term = [&](double v, double hd, double ikv, int i) -> double {
        double Si = __dadd_rn(v, -__dmul_rn(hd, gt));
        if (dbits(ikv) >= 0x7FF0000000000000ll) Si = __dadd_rn(Si, __ddiv_rn(Nf[i], kp[i]));
        return __dmul_rn(c, Si);
      };
      int i = 0;
      for (; i + 1 < M; i += 2) {
        const double v0 = Vv[i], v1 = Vv[i + 1], k0 = ik[i], k1 = ik[i + 1];
        const double p0 = part[i], p1 = part[i + 1];
        const double h0 = Hd[i * Ts], h1 = Hd[(i + 1) * Ts];
        part[i] = __dadd_rn(p0, term(v0, h0, k0, i));
        part[i + 1] = __dadd_rn(p1, term(v1, h1, k1, i + 1));
      }
      if (i < M) part[i] = __dadd_rn(part[i], term(Vv[i], Hd[i * Ts], ik[i], i));
    }
  };

  auto fill = [&]() {
    for (; gi < G; ++gi) record(gi);
  };

  // H_i of rule i at the current counts (Match_Populations: product of
  // binomials).  Models whose rules all have order <= 2 cannot overflow
  // (n*m < 2^62 for counts < 2^31) and take 32x32->64-bit products only.
  // (of trajectory column cc: the counts of block thread c are ibase + c)
  auto count_h_at = [&](int i, const int32_t* cc, bool* of) -> unsigned long long {
    if (!checked) {
      // one descriptor load, both count loads in flight together, no branches
      const uint32_t d = g_desc[i];
      const uint32_t kind = d & 3u;
      const unsigned n0 = (unsigned)cc[((d >> 2) & 0x3fffu) * Ts];
      const unsigned n1 = (unsigned)cc[((d >> 16) & 0x3fffu) * Ts];
      const unsigned m = kind == 3u ? n1 : (kind == 2u ? n0 - 1u : 1u);
      const unsigned long long prod = (unsigned long long)(kind == 0u ? 1u : n0) * m;
      return kind == 2u ? prod >> 1 : prod;
    }
    const int32_t* rec = g_rules + i * RULE_WORDS;
    const int nr = rec[R_NREAC];
    unsigned long long hh = 1ull;
    for (int a = 0; a < nr; ++a) {
      const int v = rec[R_REAC + a];
      hh = mul_checked(hh, binom12(cc[(v & 0xffff) * Ts], v >> 16), of);
    }
    return hh;
  };
  auto count_h = [&](int i) -> unsigned long long { return count_h_at(i, cnt, &ovf); };
  // h_i as a double: the count H_i, or for a Michaelis-Menten rule (kMM)
  // RN(RN(n_E n_S) / RN(K_i + n_S)), RN(n_S / RN(K_i + n_S)) without an enzyme
  auto h_of_at = [&](int i, const int32_t* cc, bool* of) -> double {
    if (kMM) {
      const double Km = prm.mm_K[i];
      if (dbits(Km) != 0) {
        const uint32_t md = prm.mm_desc[i];
        const double ns = (double)cc[(md & 0xffffu) * Ts];
        const uint32_t e1 = md >> 16;
        const double num = e1 != 0u ? __dmul_rn(ns, (double)cc[(e1 - 1u) * Ts]) : ns;
        return __ddiv_rn(num, __dadd_rn(Km, ns));
      }
    }
    return u63_to_double_rn(count_h_at(i, cc, of));
  };
  auto h_of = [&](int i) -> double { return h_of_at(i, cnt, &ovf); };
  // a_i = k_i h_i; the score replay keeps h_i as doubles in shared memory
  // (updated for every rule whose value changes), so it reads them there
  auto prop_of = [&](int i) -> double {
    return __dmul_rn(kp[i], kSens ? Hd[i * Ts] : h_of(i));
  };

  // leaf l as the blocked sum of its rules (B > 1)
  auto leaf_sum = [&](int l) -> double {
    const int j0 = l * B, j1 = min(j0 + B, M);
    double s = j0 < M ? prop_of(j0) : 0.0;
    for (int jj = j0 + 1; jj < j1; ++jj) s = __dadd_rn(s, prop_of(jj));
    return s;
  };
  // the same for the trajectory of block thread c (rates kc, counts ibase + c;
  // the score replay's h in column c of Hd); +inf when a count product
  // overflows, which makes that trajectory's a0 infinite, so that its next
  // step ends it with PROP_OVERFLOW as the overflow flag would
  auto leaf_sum_at = [&](int l, int c, const double* kc) -> double {
    const int32_t* cc = ibase + c;
    const double* hc = dbase + (32 + kNodeRows) * Ts + c;
    bool of = false;
    const int j0 = l * B, j1 = min(j0 + B, M);
    double s = j0 < M ? __dmul_rn(kc[j0], kSens ? hc[j0 * Ts] : h_of_at(j0, cc, &of)) : 0.0;
    for (int jj = j0 + 1; jj < j1; ++jj) s = __dadd_rn(s, __dmul_rn(kc[jj], kSens ? hc[jj * Ts] : h_of_at(jj, cc, &of)));
    return of ? __longlong_as_double(0x7FF0000000000000ll) : s;
  };

  auto finalize = [&]() {
    if (prm.ckpt != nullptr) {
      int32_t* rec = prm.ckpt + (size_t)q * (S + CKPT_HEADER_WORDS);
      put_f64(rec, t);
      put_u64(rec + 2, h);
      rec[4] = (int32_t)n;
      rec[5] = gi;
      rec[6] = status;
      rec[7] = 0;
      for (int s = 0; s < S; ++s) rec[CKPT_HEADER_WORDS + s] = CNT(s);
    }
    if (prm.traj_status) prm.traj_status[q] = status;
    if (prm.traj_events) prm.traj_events[q] = (long long)n;
    if (prm.traj_hash) prm.traj_hash[q] = h;
    if (prm.traj_final_t) prm.traj_final_t[q] = t;
  };

  // set up trajectory q: 0 = running, 1 = ended at once (bad input),
  // 2 = nothing to do (resuming, and this trajectory did not stop on the deadline)
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
    for (int j = 0; j < M; ++j) {
      const long long kb = dbits(kp[j]);
      if (!(kb > 0 && kb < 0x7FF0000000000000ll)) bad = true;
    }
    const int32_t* x0 = prm.init + (size_t)(prm.Pi == 1 ? 0 : p) * S;
    if (prm.resume) {
      const int32_t* rec = prm.ckpt + (size_t)q * (S + CKPT_HEADER_WORDS);
      if (rec[6] != TS_TIMEOUT) return 2;
      t = get_f64(rec);
      h = get_u64(rec + 2);
      n = (unsigned)rec[4];
      gi = rec[5];
      if (gi < 0 || gi > G) bad = true;
      gbits = gi < G && gi >= 0 ? dbits(prm.grid[gi]) : 0;
      x0 = rec + CKPT_HEADER_WORDS;
    }
    for (int s = 0; s < S; ++s) {
      const int v = x0[s];
      if (v < 0) bad = true;
      CNT(s) = v;
    }
    if (kSens) {
      double* sa = prm.sens_acc + (size_t)q * 2 * M;   // per trajectory: V [M], Nf [M]
      Vv = sa;
      Nf = sa + M;
      part = prm.partials + (size_t)q * M;
      ik = prm.inv_rates + (size_t)p * M;
      for (int i = 0; i < M; ++i) part[i] = 0.0;
    }
    if (bad) {
      status = TS_BAD_INPUT;
      if (prm.states != nullptr) {
        int32_t* dst = prm.states + (size_t)q * G * S;
        for (long long e = 0; e < (long long)G * S; ++e) dst[e] = 0;
      }
      return 1;
    }
    if (kSens) {
      for (int i = 0; i < M; ++i) {
        Hd[i * Ts] = h_of(i);
        Vv[i] = 0.0;
        Nf[i] = 0.0;
      }
    }
    for (int l = 0; l < 32; ++l) LEAF(l) = B == 1 ? (l < M ? prop_of(l) : 0.0) : leaf_sum(l);
    if (kNodes)
      for (int nd = 0; nd < 16; ++nd) node[nd * Ts] = __dadd_rn(LEAF(2 * nd), LEAF(2 * nd + 1));
    rebuild_upper();
    return 0;
  };

  // propensity overflow: the current term's H is unusable, so the score's
  // integrals stop at the last applied event (time t) and H counts as 0
  // after it; the lazily kept integrals are first brought up to t
  auto freeze_h = [&]() {
    for (int i = 0; i < M; ++i) {
      Vv[i] = __dadd_rn(Vv[i], __dmul_rn(-Hd[i * Ts], t));   // H_i drops to 0 at t
      Hd[i * Ts] = 0.0;
    }
  };

  int pend_j = 0;
  double pend_t = 0.0;
  unsigned pend_lm = 0u;
  // one event or the end of the trajectory: 0 = running, 1 = ended with grid
  // points left to fill, 2 = ended with the grid complete (or left to a resume)
  auto step = [&]() -> int {
    // the same order of checks as the written specification: overflow of a
    // count product or of a0 first, then the event cap, then absorption
    const double a0 = root;
    const long long a0b = dbits(a0);
    if (ovf || a0b >= 0x7FF0000000000000ll) {
      status = TS_PROP_OVERFLOW;
      if (kSens) freeze_h();
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
    // applied 1024 events in this launch, so every launch makes progress.
    // At the same points the tail layout hands the trajectory over to the
    // warp-per-trajectory kernel once the queue is empty and few trajectories
    // are left (its checkpoint record carries the state)
    if ((n & 1023u) == 0u && n != n_launch) {
      if (deadline != ~0ull && globaltimer_ns() > deadline) {
        status = TS_TIMEOUT;
        return prm.ckpt == nullptr ? 1 : 2;   // with a checkpoint the rest is recorded on resume
      }
      // once the queue is empty every trajectory has started, so Q - finished
      // of them are still running
      if (kTail &&
          *reinterpret_cast<volatile unsigned long long*>(&prm.ws->queue_next) >= (unsigned long long)Q &&
          (unsigned long long)Q - *reinterpret_cast<volatile unsigned long long*>(&prm.ws->finished) <=
              (unsigned long long)prm.handoff) {
        status = TS_TIMEOUT;
        return 2;
      }
    }
    const uint4 w = philox4x32_10(make_uint4(n, 0u, (uint32_t)r + prm.r_offset, (uint32_t)p), prm.key0, prm.key1);
    const double u_tau = uniform52(w.x, w.y);
    const double u_sel = uniform52(w.z, w.w);
    const double tau = __ddiv_rn(-log_spec_q(u_tau, lc, g_rj, g_tj), a0);
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
    // rule selection: guarded descent of x = u_sel * a0; k is the index of
    // the chosen node within its level
    double x = __dmul_rn(u_sel, a0);
    int k;
    auto descend = [&](double L, double Rv) -> int {
      const bool left = dbits(x) < dbits(L) || dbits(Rv) == 0;
      const double xr = __dadd_rn(x, -L);
      x = left ? x : xr;
      return left ? 0 : 1;
    };
    k = descend(u4[0], u4[1]);                                       // root -> node 28 + k
    k = 2 * k + descend(k ? u3[2] : u3[0], k ? u3[3] : u3[1]);       // -> node 24 + k
    {
      const double L = (k & 2) ? ((k & 1) ? u2[6] : u2[4]) : ((k & 1) ? u2[2] : u2[0]);
      const double Rv = (k & 2) ? ((k & 1) ? u2[7] : u2[5]) : ((k & 1) ? u2[3] : u2[1]);
      k = 2 * k + descend(L, Rv);                                    // -> node 16 + k
    }
    k = 2 * k + descend(NODE(2 * k), NODE(2 * k + 1));               // -> level-1 node k
    const int l = 2 * k + descend(LEAF(2 * k), LEAF(2 * k + 1));     // -> leaf l
    int j;
    if (B == 1) {
      j = l;
    } else {
      const int j0 = l * B, j1 = min(j0 + B, M);
      int last = -1;
      j = -1;
      double s = 0.0;
      for (int jj = j0; jj < j1; ++jj) {
        // (the score replay has h as a double already).  A count H >= 1 gives
        // a_j >= k_j > 0; a Michaelis-Menten h < 1 can give k_j h = 0, so
        // kMM tests a_j itself
        const double hdd = kSens ? Hd[jj * Ts] : h_of(jj);
        if (kMM || dbits(hdd) != 0) {
          const double a = __dmul_rn(kp[jj], hdd);
          if (!kMM || dbits(a) != 0) {
            s = last < 0 ? a : __dadd_rn(s, a);
            last = jj;
            if (dbits(x) < dbits(s)) {
              j = jj;
              break;
            }
          }
        }
      }
      if (j < 0) j = last;
    }
    // The guarded descent always ends on a positive entry because every node
    // equals the sum of its children; the clamp only keeps indices in range.
    j = min(max(j, 0), M - 1);
    // apply the stoichiometry change (checked first: nothing changes on overflow)
    const int32_t* rec = g_rules + j * RULE_WORDS;
    const int nd_ = rec[R_NDELTA];
    for (int d = 0; d < nd_; ++d) {
      const int v = rec[R_DELTA + d];
      const int dv = v >> 16;
      if (dv > 0 && CNT(v & 0xffff) > 0x7FFFFFFF - dv) {
        status = TS_INT_OVERFLOW;
        return 1;
      }
    }
    for (int d = 0; d < nd_; ++d) {
      const int v = rec[R_DELTA + d];
      CNT(v & 0xffff) += v >> 16;
    }
    if (kSens) {
      if (dbits(ik[j]) < 0x7FF0000000000000ll)
        Vv[j] = __dadd_rn(Vv[j], ik[j]);
      else
        Nf[j] = __dadd_rn(Nf[j], 1.0);
      const int doff = rec[R_DEPOFF], dcnt = rec[R_DEPCNT];
      // V_i += (h' - h) t for the rules whose value changed (for counts
      // h, h' < 2^53 in practice, so h' - h is exact)
      for (int e = 0; e < dcnt; ++e) {
        const int i = g_deps[doff + e];
        const double hd = h_of(i);
        Vv[i] = __dadd_rn(Vv[i], __dmul_rn(__dadd_rn(hd, -Hd[i * Ts]), tn));
        Hd[i * Ts] = hd;
      }
    }
    // the leaves, nodes and the rest of the event follow in finish_event(),
    // after the warp has rebuilt every lane's dirty leaves together
    pend_j = j;
    pend_t = tn;
    pend_lm = (unsigned)rec[R_LEAFMASK];
    return 0;
  };

  // the rest of an applied event: the lane rebuilds its dirty leaves (with
  // B = 1 they are the dependents' propensities), unless the warp has
  // already rebuilt them together (kPool)
  // The level-1 node above a dirty leaf is written by whoever rebuilds the
  // last dirty leaf of its pair (the dirty leaves are rebuilt in ascending
  // order, so the pair's other value, when dirty too, was the one just
  // before it), in the same pass as the leaves: no second, max-over-lanes
  // loop over the dirty nodes.  Returns whether leaf l's node is written
  // here; mate_dirty says whether the node's other leaf was rebuilt too.
  auto pair_last = [](int l, unsigned lmask, bool* mate_dirty) -> bool {
    *mate_dirty = (lmask >> (l ^ 1)) & 1u;
    return (l & 1) || !*mate_dirty;
  };
  auto finish_event = [&]() {
    const int32_t* rec = g_rules + pend_j * RULE_WORDS;
    if (!kPool) {
      const unsigned lmask = (unsigned)rec[R_LEAFMASK];
      double prev = 0.0;   // the previous dirty leaf's new value
      auto leaf_done = [&](int ll, double v) {
        LEAF(ll) = v;
        if (kNodes) {
          bool md;
          if (pair_last(ll, lmask, &md)) node[(ll >> 1) * Ts] = __dadd_rn(v, md ? prev : LEAF(ll ^ 1));
          prev = v;
        }
      };
      if (B == 1) {
        // (the dependents are listed in ascending order: leaf i is rule i)
        const int doff = rec[R_DEPOFF], dcnt = rec[R_DEPCNT];
        for (int e = 0; e < dcnt; ++e) {
          const int i = g_deps[doff + e];
          leaf_done(i, prop_of(i));
        }
      } else {
        unsigned lm = lmask;
        while (lm) {
          const int ll = __ffs(lm) - 1;
          lm &= lm - 1u;
          leaf_done(ll, leaf_sum(ll));
        }
      }
    } else {
      // the warp has rebuilt the leaves; the level-1 nodes above them follow
      // per lane (writing them in the pooled rounds instead, by the pair's
      // last dirty leaf, measured 0.6 % slower on the 64-rule network)
      unsigned nm = kNodes ? (unsigned)rec[R_NODEMASK] & 0xFFFFu : 0u;
      while (nm) {
        const int kk = __ffs(nm) - 1;
        nm &= nm - 1u;
        node[kk * Ts] = __dadd_rn(LEAF(2 * kk), LEAF(2 * kk + 1));
      }
    }
    rebuild_upper();
    if (prm.log_cap > 0 && n < (unsigned)prm.log_cap) {
      const size_t at = (size_t)q * prm.log_cap + n;
      prm.log_rule[at] = pend_j;
      if (prm.log_slot) prm.log_slot[at] = 0;
      if (prm.log_t) prm.log_t[at] = pend_t;
    }
    t = pend_t;
    ++n;
    h = fnv1a_event(h, (uint32_t)pend_j, 0u);
  };

  // Every lane's dirty leaves (kPool), rebuilt by the whole warp: the
  // (lane, leaf) pairs are numbered lane by lane (a prefix sum of the leaf
  // counts) and dealt out 32 at a time, so that a warp spends ceil(sum / 32)
  // rounds instead of max-over-lanes iterations of a per-lane leaf loop.
  // Each round holds the leaf's B products and B - 1 sums, and an FP64 warp
  // instruction occupies GB300's FP64 pipe for the same 16 SM cycles however
  // few lanes execute it; on the 64-rule network (4.5 dirty leaves per event)
  // a warp-step needs 4.8 rounds against 8.9 iterations of the per-lane loop
  // (+9 % events/s).  Where an event dirties at most two leaves, or a leaf is
  // one product (B = 1), the dealing costs more than it saves (-11 % on the
  // 32-species Lotka-Volterra chain, -5 % on a 24-rule network), unless the
  // leaves hold Michaelis-Menten divisions (+12 % on the 40-rule cascade).
  // All 32 lanes of the warp take part.
  auto pooled_leaves = [&](unsigned lm) {
    const unsigned FULL = 0xffffffffu;
    const int lane = tid & 31;
    const int cnt_l = __popc(lm);
    int incl = cnt_l;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += v;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    const int excl = incl - cnt_l;
    for (int base = 0; base < total; base += 32) {
      const int idx = base + lane;
      // owner: the number of lanes whose inclusive prefix is <= idx
      int o = 0;
#pragma unroll
      for (int s = 16; s >= 1; s >>= 1) {
        const int v = __shfl_sync(FULL, incl, o + s - 1);
        if (v <= idx) o += s;
      }
      o &= 31;
      const unsigned lm_o = __shfl_sync(FULL, lm, o);
      const int ex_o = __shfl_sync(FULL, excl, o);
      const int p_o = __shfl_sync(FULL, p, o);
      if (idx < total) {
        // the (idx - ex_o)-th set bit of the owner's mask
        unsigned m = lm_o;
        int k = idx - ex_o, pos = 0, c;
        c = __popc(m & 0xFFFFu); if (k >= c) { k -= c; m >>= 16; pos += 16; }
        c = __popc(m & 0xFFu);   if (k >= c) { k -= c; m >>= 8;  pos += 8; }
        c = __popc(m & 0xFu);    if (k >= c) { k -= c; m >>= 4;  pos += 4; }
        c = __popc(m & 0x3u);    if (k >= c) { k -= c; m >>= 2;  pos += 2; }
        if (k >= (int)(m & 1u)) pos += 1;
        const int col = tid - lane + o;
        dbase[pos * Ts + col] = leaf_sum_at(pos, col, prm.rates + (size_t)p_o * M);
      }
    }
    __syncwarp();
  };

  bool need_new = true;
  bool had_one = false;   // kTail: this lane has finished a trajectory before taking the next
  // a lane that finishes a trajectory takes the next one
  auto next_trajectory = [&]() -> bool {
    if (kTail && had_one) {
      // warp-aggregated count of finished trajectories (ran, or bad input)
      const unsigned mask = __activemask();
      if ((int)(threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(&prm.ws->finished, (unsigned long long)__popc(mask));
    }
    had_one = true;
    if (kQueue) {
      q = grab_next(prm.ws);
      if (prm.order != nullptr && q < Q) {
        const long long pp = prm.order[q / prm.R];
        q = pp * prm.R + (q - (q / prm.R) * prm.R);
      }
    } else {
      q = first ? (long long)blockIdx.x * T + tid : q + qstride;
      first = false;
    }
    return q < Q;
  };
  if (!kPool) {
    // every lane runs its own trajectories through
    for (;;) {
      if (need_new) {
        if (!next_trajectory()) break;
        const int st0 = start();
        if (st0 == 1) finalize();
        if (st0 != 0) continue;
        n_launch = n;
        need_new = false;
      }
      const int ended = step();
      if (ended == 0) {
        finish_event();
      } else {
        if (ended == 1) fill();
        finalize();
        need_new = true;
      }
    }
  } else {
    // the warp rebuilds its lanes' leaves together, so every lane stays in
    // the loop until all of them are out of trajectories
    bool done = false;
    for (;;) {
      unsigned lm = 0u;     // leaves of this lane's applied event, if any
      bool applied = false;
      if (!done) {
        if (need_new) {
          if (!next_trajectory()) {
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
          } else {
            lm = pend_lm;
            applied = true;
          }
        }
      }
      pooled_leaves(lm);   // ends with __syncwarp(): the warp is reconverged for the rest of the event
      if (applied) finish_event();
      if (__all_sync(0xffffffffu, done)) break;
    }
  }
#undef LEAF
#undef NODE
#undef CNT
}

// ---------------------------------------------------------------------------
// Predictive queue order (longest expected sweep point first).  The initial
// total propensity a0(x0; k_p) is the rate of events at the start, a proxy
// for the trajectory length under the same horizon; serving the longest
// sweep points first keeps them off the tail of the run.  Only the order in
// which trajectories are taken changes, never their values.
// ---------------------------------------------------------------------------

__global__ void flat_estimate_kernel(const __grid_constant__ FlatParams prm, double* __restrict__ est) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= prm.P) return;
  const int32_t* x0 = prm.init + (size_t)(prm.Pi == 1 ? 0 : p) * prm.S;
  const double* k = prm.rates + (size_t)p * prm.M;
  double a0 = 0.0;
  for (int j = 0; j < prm.M; ++j) {
    const int32_t* rec = prm.rules + j * RULE_WORDS;
    double hh = 1.0;
    for (int a = 0; a < rec[R_NREAC]; ++a) {
      const int v = rec[R_REAC + a];
      const double n = (double)max(x0[v & 0xffff], 0);
      hh *= (v >> 16) == 1 ? n : 0.5 * n * (n - 1.0);
    }
    if (prm.mm_K != nullptr && prm.mm_K[j] != 0.0)   // Michaelis-Menten: n_E n_S / (K + n_S)
      hh /= prm.mm_K[j] + (double)max(x0[prm.mm_desc[j] & 0xffffu], 0);
    a0 += k[j] * hh;
  }
  est[p] = (a0 >= 0.0 && a0 < 1e300) ? a0 : 0.0;
}

__global__ void rank_desc_kernel(const double* __restrict__ est, int P, int32_t* __restrict__ order) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const double e = est[p];
  int rank = 0;
  for (int i = 0; i < P; ++i) {
    const double f = est[i];
    rank += (f > e) || (f == e && i < p);
  }
  order[rank] = p;
}

cudaError_t launch_flat_order(const FlatParams& prm, double* est, int32_t* order, cudaStream_t stream) {
  const int blocks = (prm.P + 127) / 128;
  flat_estimate_kernel<<<blocks, 128, 0, stream>>>(prm, est);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rank_desc_kernel<<<blocks, 128, 0, stream>>>(est, prm.P, order);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host launcher
// ---------------------------------------------------------------------------

template <bool kQueue, bool kSens, bool kTail, bool kMM, bool kPool>
static cudaError_t launch_k(const FlatParams& prm, const LogConstants& lc, int T, int blocks_per_sm_cap,
                            cudaStream_t stream, int* used_blocks) {
  auto kern = flat_ssa_kernel<kQueue, kSens, kTail, kMM, kPool>;
  const size_t smem = (size_t)prm.smem_table_bytes + (size_t)(T + 1) * flat_thread_bytes(prm.S, prm.M, kSens, kMM);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  long long blocks;
  if (kQueue) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (blocks_per_sm_cap > 0 && per_sm > blocks_per_sm_cap) per_sm = blocks_per_sm_cap;
    blocks = (long long)sms * per_sm;
    const long long need = (prm.Q + T - 1) / T;
    if (blocks > need) blocks = need;
  } else {
    blocks = (prm.Q + T - 1) / T;
    if (blocks > 0x7FFFFFFFll) blocks = 0x7FFFFFFFll;
  }
  if (blocks < 1) blocks = 1;
  if (used_blocks) *used_blocks = (int)blocks;
  kern<<<(unsigned)blocks, T, smem, stream>>>(prm, lc);
  return cudaGetLastError();
}

template <bool kQueue, bool kSens, bool kTail = false, bool kMM = false>
static cudaError_t launch_t(const FlatParams& prm, const LogConstants& lc, int T, int blocks_per_sm_cap,
                            cudaStream_t stream, int* used_blocks) {
  return prm.pool ? launch_k<kQueue, kSens, kTail, kMM, true>(prm, lc, T, blocks_per_sm_cap, stream, used_blocks)
                  : launch_k<kQueue, kSens, kTail, kMM, false>(prm, lc, T, blocks_per_sm_cap, stream, used_blocks);
}

size_t flat_smem_bytes(const FlatParams& prm, int T, bool sens) {
  return (size_t)prm.smem_table_bytes + (size_t)(T + 1) * flat_thread_bytes(prm.S, prm.M, sens, prm.mm_K != nullptr);
}

int flat_table_bytes_host(int M, int n_deps) { return flat_table_bytes(M, n_deps); }

// Automatic block size.  A batch larger than the GPU's resident capacity
// takes the block size with the most resident warps per SM (ties: the larger
// block).  A batch that fits in one resident wave at some block size takes,
// among those sizes, the one whose busiest SM holds the fewest trajectories,
// ceil(blocks / SMs) * T, since that SM sets the time of the launch (ties:
// the larger block); e.g. 32,768 trajectories at 224 per block fill 147 SMs
// with one block each instead of doubling up 19 SMs with 192-thread blocks.
template <bool kQueue, bool kSens, bool kMM>
static int auto_threads_t(const FlatParams& prm) {
  auto kern = prm.pool ? flat_ssa_kernel<kQueue, kSens, false, kMM, true> : flat_ssa_kernel<kQueue, kSens, false, kMM, false>;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1)
    sms = 1;
  int per_sm[9] = {0};                  // per_sm[T / 32], T = 32..256
  int best_T = 32, best_warps = -1;
  for (int T = 32; T <= 256; T += 32) {
    const size_t smem = (size_t)prm.smem_table_bytes + (size_t)(T + 1) * flat_thread_bytes(prm.S, prm.M, kSens, kMM);
    if (smem > 227 * 1024) break;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) break;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[T / 32], kern, T, smem) != cudaSuccess) break;
    const int warps = per_sm[T / 32] * T / 32;
    if (warps >= best_warps) {
      best_warps = warps;
      best_T = T;
    }
  }
  long long best_load = -1;
  int pick = best_T;
  for (int T = 256; T >= 32; T -= 32) {
    if (per_sm[T / 32] < 1) continue;
    const long long blocks = (prm.Q + T - 1) / T;
    if (blocks > (long long)sms * per_sm[T / 32]) continue;          // more than one resident wave
    const long long load = (blocks + sms - 1) / sms * T;             // trajectories on the busiest SM
    if (best_load < 0 || load < best_load) {
      best_load = load;
      pick = T;
    }
  }
  return pick;
}

int flat_auto_threads(const FlatParams& prm, bool queue, bool sens) {
  if (prm.mm_K != nullptr) {
    if (queue) return sens ? auto_threads_t<true, true, true>(prm) : auto_threads_t<true, false, true>(prm);
    return sens ? auto_threads_t<false, true, true>(prm) : auto_threads_t<false, false, true>(prm);
  }
  if (queue) return sens ? auto_threads_t<true, true, false>(prm) : auto_threads_t<true, false, false>(prm);
  return sens ? auto_threads_t<false, true, false>(prm) : auto_threads_t<false, false, false>(prm);
}

cudaError_t launch_flat(const FlatParams& prm, const LogConstants& lc, bool queue, bool sens, int T,
                        int blocks_per_sm_cap, cudaStream_t stream, int* used_blocks) {
  if (prm.mm_K != nullptr) {   // Michaelis-Menten rules: no tail hand-over
    if (prm.handoff > 0) return cudaErrorInvalidValue;
    if (queue)
      return sens ? launch_t<true, true, false, true>(prm, lc, T, blocks_per_sm_cap, stream, used_blocks)
                  : launch_t<true, false, false, true>(prm, lc, T, blocks_per_sm_cap, stream, used_blocks);
    return sens ? launch_t<false, true, false, true>(prm, lc, T, blocks_per_sm_cap, stream, used_blocks)
                : launch_t<false, false, false, true>(prm, lc, T, blocks_per_sm_cap, stream, used_blocks);
  }
  if (queue) {
    if (!sens && prm.handoff > 0) return launch_t<true, false, true>(prm, lc, T, blocks_per_sm_cap, stream, used_blocks);
    return sens ? launch_t<true, true>(prm, lc, T, blocks_per_sm_cap, stream, used_blocks)
                : launch_t<true, false>(prm, lc, T, blocks_per_sm_cap, stream, used_blocks);
  }
  return sens ? launch_t<false, true>(prm, lc, T, blocks_per_sm_cap, stream, used_blocks)
              : launch_t<false, false>(prm, lc, T, blocks_per_sm_cap, stream, used_blocks);
}

}  // namespace cwcgpu
