// Internal layout shared by the host-side model compiler and the kernels of
// the CUDA library.  Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>

namespace cwcgpu {

// Per-rule record of a compiled flat model, RULE_WORDS int32 words:
//   [0]      number of reactant species (<= MAX_REAC)
//   [1..4]   reactant: species (low 16 bits) | multiplicity nu (high 16 bits)
//   [5]      number of species whose count changes (<= MAX_DELTA)
//   [6..13]  change: species (low 16 bits) | signed delta (high 16 bits)
//   [14]     offset of the rule's dependents in the dependency array
//   [15]     number of dependents (rules whose propensity reads a species
//            this rule changes), ascending
//   [16]     bit mask of the 32 tree leaves the dependents live in
//   [17]     bit mask of the 31 internal tree nodes above those leaves
//   [18..19] unused
constexpr int RULE_WORDS = 20;
// After the dependents, a compiled flat model has one reactant descriptor per
// rule (order <= 2 models): kind (0: order 0, 1: n0, 2: C(n0, 2), 3: n0 * n1)
// in bits 0-1, species 0 in bits 2-15, species 1 in bits 16-29 (species 0
// again when the rule has a single reactant species).  Then, padded to a
// 16-byte boundary, the logarithm's 64 rj and 64 tj words (u64 each, low
// word first; see LogConstants), which the kernel indexes per lane.
constexpr int MAX_REAC = 4;
constexpr int MAX_DELTA = 8;
constexpr int R_NREAC = 0, R_REAC = 1, R_NDELTA = 5, R_DELTA = 6, R_DEPOFF = 14, R_DEPCNT = 15,
              R_LEAFMASK = 16, R_NODEMASK = 17;

// Internal nodes of the 32-lane tree: level 1 nodes 0..15 (children: leaves
// 2n, 2n+1), level 2 nodes 16..23, level 3 24..27, level 4 28..29, root 30.
// For n >= 16 the children are nodes 2n-32 and 2n-31.
constexpr int TREE_NODES = 31;
constexpr int TREE_ROOT = 30;

// Per-rule record of a compiled compartmentalised model, CWC_RULE_WORDS words:
//   [0] kind  [1] context label  [2] child label  [3] number of reactant entries
//   [4..7]   reactant: species | nu << 16 | row << 24 (row 0 = context / parent
//            content, 1 = child wrap, 2 = child content, 3 / 4 = the second
//            child's (FUSION) or the grandchild's (NESTED) wrap / content),
//            rows then species ascending
//   [8]  n0, [9..16]   changes of the context (parent) content: species | delta << 16
//   [17] n1, [18..25]  PARENT_CHILD / NESTED / PAIR: changes of the (first)
//                      child wrap; CREATE: the new wrap; FUSION: atoms added
//                      to the merged wrap
//   [26] n2, [27..34]  the same for the child content / new content / merged content
//   [35] offset and [36] number of dependents (rules whose counts the event
//        can change; every rule after a FUSION, NESTED or PAIR event)
//   [37] dirty-leaf mask, [38] dirty-node mask of those dependents
//   [39] NESTED: grandchild label, PAIR: 1 if the two compartments' right-
//        hand patterns are identical (else 0), | (word offset of the rule's
//        extension record in the table) << 8; the extension, after the
//        dependency list, holds n3, [8] changes of the grandchild's (second
//        child's) wrap, n4, [8] changes of its content (species | delta << 16)
// The 40-word stride keeps the records of different rules in different
// shared-memory banks when the lanes of a warp read different rules.
constexpr int CWC_RULE_WORDS = 40;
constexpr int CR_KIND = 0, CR_CTX = 1, CR_CHILD = 2, CR_NREAC = 3, CR_REAC = 4, CR_ND0 = 8, CR_D0 = 9, CR_ND1 = 17,
              CR_D1 = 18, CR_ND2 = 26, CR_D2 = 27, CR_DEPOFF = 35, CR_DEPCNT = 36, CR_LEAFMASK = 37, CR_NODEMASK = 38,
              CR_GRAND = 39;
// the NESTED / PAIR extension record: XR_ND3 / XR_D3 / XR_ND4 / XR_D4 words
constexpr int XR_ND3 = 0, XR_D3 = 1, XR_ND4 = 9, XR_D4 = 10, XR_WORDS = 18;
// rule kinds (values of the C header's CWC_RULE_*)
constexpr int RK_LOCAL = 0, RK_PARENT_CHILD = 1, RK_CREATE = 2, RK_DISSOLVE = 3, RK_FUSION = 4, RK_NESTED = 5,
              RK_PAIR = 6;
constexpr int CWC_MAX_SLOTS = 64;

// Checkpoint record of a flat trajectory (int32 words): time (double, words
// 0-1), event hash (words 2-3), event count, next grid point, status, unused,
// then the S counts.
constexpr int CKPT_HEADER_WORDS = 8;

// Trajectory status codes (same values as CWC_TRAJ_* in the C header).
enum : int32_t {
  TS_OK = 0, TS_ABSORBED = 1, TS_INT_OVERFLOW = 2, TS_PROP_OVERFLOW = 3, TS_CAPACITY = 4,
  TS_EVENT_LIMIT = 5, TS_BAD_INPUT = 6, TS_TIMEOUT = 7,
  // internal, never an output: a count of a 16-bit term would leave int16's
  // range; the trajectory is saved for the 32-bit launch that follows
  TS_WIDEN = 100
};

// Workspace header (first 256 bytes when used): work-queue ticket, the
// launch timestamp for deadlines and, for the tail layout, the number of
// trajectories the thread kernel has finished, the number handed over to the
// warp kernel and that kernel's ticket.
struct WorkspaceHeader {
  unsigned long long queue_next;
  unsigned long long t_start_ns;
  unsigned long long finished;
  unsigned long long tail_count;
  unsigned long long tail_next;
  unsigned long long pad[27];
};
static_assert(sizeof(WorkspaceHeader) == 256, "workspace header size");

// Everything one flat-model launch needs.
struct FlatParams {
  // compiled model
  int S, M, B;              // species, rules, leaf block size ceil(M/32)
  int n_deps;
  int checked_counts;       // 1 if some rule has order >= 3 (int64 products may overflow)
  const int32_t* rules;     // [M][RULE_WORDS]
  const int32_t* deps;      // [n_deps]
  const double* mm_K;       // Michaelis-Menten constants [M] (0: mass action), or null when every rule is mass action
  const uint32_t* mm_desc;  // [M] substrate | (enzyme + 1) << 16 of the Michaelis-Menten rules
  int pool;                 // 1: the warp rebuilds its lanes' dirty leaves together (B > 1, see the kernel)
  // batch
  int P, R, G, Pi;
  uint32_t r_offset;        // replica index offset of the random streams
  long long Q;              // P * R
  const double* rates;      // [P][M]
  const int32_t* init;      // [Pi][S]
  const double* grid;       // [G]
  uint32_t key0, key1;
  long long max_events;
  // outputs
  int32_t* states;                 // [Q][G][S]
  unsigned long long* sums;        // [P][G][S]
  unsigned long long* sumsq;       // [P][G][S][2] 128-bit sums of squares (low, high)
  int32_t* traj_status;
  long long* traj_events;
  unsigned long long* traj_hash;
  double* traj_final_t;
  int log_cap;
  int32_t* log_rule;
  int32_t* log_slot;
  double* log_t;
  // score replay
  const double* means;             // [P][G][S]
  const double* grad_means;        // [P][G][S]
  double* partials;                // [Q][M]
  double* sens_acc;                // score replay: per trajectory V_i [M] (see the kernel), then [M] firings N_i
  const double* inv_rates;         // score replay: [P][M] 1 / k_j
  // scheduling
  WorkspaceHeader* ws;             // queue ticket / start time (may be null in static mode)
  int32_t* ckpt;                   // [Q][S + CKPT_HEADER_WORDS] trajectory checkpoints (or null)
  int resume;                      // 1: continue the TIMEOUT trajectories of ckpt
  const int32_t* order;            // queue mode: sweep points, longest expected first (or null)
  long long handoff;               // tail layout: hand over when the queue is empty and at most
                                   // this many trajectories run (0 = never)
  long long deadline_ns;
  int smem_table_bytes;            // bytes of the shared-memory table region
};

// Everything one compartmentalised-model launch needs.
struct CwcParams {
  int S, L, C, M, B, O;
  int n_deps;
  int general;              // 1 if some rule is FUSION or NESTED
  const int32_t* rules;     // [M][CWC_RULE_WORDS] then [n_deps]
  int P, R, G, Pi;
  uint32_t r_offset;
  long long Q;
  const double* rates;      // [P][M]
  const int32_t* init;      // [Pi][C][3 + 2S]
  const double* grid;       // [G]
  uint32_t key0, key1;
  long long max_events;
  int32_t* states;                 // [Q][G][O]
  unsigned long long* sums;        // [P][G][O]
  unsigned long long* sumsq;       // [P][G][O][2]
  int32_t* traj_status;
  long long* traj_events;
  unsigned long long* traj_hash;
  double* traj_final_t;
  int log_cap;
  int32_t* log_rule;
  int32_t* log_slot;
  double* log_t;
  int sens;                        // 1: score replay variant
  const double* means;             // score replay: [P][G][O]
  const double* grad_means;        // score replay: [P][G][O]
  double* partials;                // score replay: [Q][M]
  int32_t* slabs;                  // per launched thread, slab_words each
  long long slab_words;
  int32_t* ckpt;                   // [Q][CKPT_HEADER_WORDS + C * (3 + 2S)] checkpoints (or null)
  int resume;                      // 1: continue the TIMEOUT trajectories of ckpt
  int narrow;                      // 1: 16-bit term counts; a trajectory whose count would leave
                                   // int16's range is saved in ckpt as TIMEOUT for the 32-bit
                                   // resume launch that follows (every record's status is written)
  WorkspaceHeader* ws;
  long long deadline_ns;
  int smem_table_bytes;
};

}  // namespace cwcgpu
