/*
 * cwcgpu.h -- C ABI of the GB300 library for batched Gillespie direct-method
 * simulation of Calculus of Wrapped Compartments (CWC) rewrite systems.
 *
 * The method (Aldinucci et al., "On Designing Multicore-aware Simulators for
 * Biological Systems"): CWC terms and rules, Sec. 2.1; stochastic rules whose
 * rate is the kinetic constant times the number of distinct reactant
 * combinations, and Gillespie's two-step direct method, Sec. 2.2; the
 * Match / Resolve / Update simulator step, Sec. 2.3 and Fig. "CWC simulator
 * pseudo-code" (Sec. 5.1); many independent replicas and parameter-sweep
 * instances sampled on a fixed simulation-time grid, Sec. 5.2.
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA device addresses on the current device; host
 *     pointers are read before the call returns and may be freed afterwards.
 *   - The caller owns every buffer it passes.  The library owns only what
 *     cwc_model_create allocates (the compiled rule tables), released by
 *     cwc_model_destroy.  No entry point other than cwc_model_create
 *     allocates device memory.
 *   - Work is enqueued on the given CUDA stream (cudaStream_t passed as
 *     void*; NULL = the legacy default stream) and runs asynchronously; an
 *     entry point returns after enqueueing.  Argument errors are detected on
 *     the host before anything is enqueued and return a status; per-
 *     trajectory problems found on the device (bad rates, bad grid, counts
 *     out of range) are reported in the per-trajectory status array.
 *   - No entry point throws, aborts or falls back to the CPU.  On failure a
 *     description is available from cwc_last_error() (thread-local).
 */
#ifndef CWCGPU_H_
#define CWCGPU_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes of the entry points. */
typedef enum {
  CWC_OK = 0,
  CWC_ERR_INVALID_ARG = 1,   /* a pointer, size or model field is invalid      */
  CWC_ERR_UNSUPPORTED = 2,   /* outside the rule language this library runs     */
  CWC_ERR_CUDA = 3,          /* a CUDA call failed (message in cwc_last_error) */
  CWC_ERR_WORKSPACE = 4,     /* workspace missing or smaller than required     */
  CWC_ERR_INTERNAL = 5
} cwc_status;

/* Status of one trajectory (int32 array traj_status). */
enum {
  CWC_TRAJ_OK = 0,            /* reached the last grid point                       */
  CWC_TRAJ_ABSORBED = 1,      /* total propensity 0; remaining grid = current term */
  CWC_TRAJ_INT_OVERFLOW = 2,  /* an event would push a count above INT32_MAX; not applied */
  CWC_TRAJ_PROP_OVERFLOW = 3, /* an int64 combinatorial count overflowed or a0 = +inf */
  CWC_TRAJ_CAPACITY = 4,      /* CREATE found no free compartment slot; not applied */
  CWC_TRAJ_EVENT_LIMIT = 5,   /* max_events events applied                         */
  CWC_TRAJ_BAD_INPUT = 6,     /* a rate <= 0 or not finite, a negative count, an
                                 invalid slot image, or a grid that is not strictly
                                 increasing from a value >= 0                      */
  CWC_TRAJ_TIMEOUT = 7        /* the call's deadline passed                        */
};

/* Rule kinds of the CWC language this library runs (Sec. 2.1 rule
 * application: the left-hand side, a pattern that may itself hold
 * compartments, is matched against the content, or the wrap, of a
 * compartment of the rule's label). */
enum {
  CWC_RULE_LOCAL = 0,        /* l: p X -> p' X                               */
  CWC_RULE_PARENT_CHILD = 1, /* l: p X (w x | q Y)^l' -> p' X (w' x | q' Y)^l' */
  CWC_RULE_CREATE = 2,       /* l: p X -> p' X (w' | q')^l'                  */
  CWC_RULE_DISSOLVE = 3,     /* l: p X (w x | q Y)^l' -> p' X x Y            */
  CWC_RULE_FUSION = 4,       /* two compartments in one left-hand side:
                                l: p X (w1 x1 | q1 Y1)^l' (w2 x2 | q2 Y2)^l'
                                   -> p' X (w' x1 x2 | q' Y1 Y2)^l'
                                contexts: ordered pairs of sibling l' slots
                                (unordered when the two compartment patterns
                                are identical); the lower slot keeps the merged
                                compartment, the other is freed and its
                                children move to the survivor                */
  CWC_RULE_NESTED = 5,       /* a pattern of depth two:
                                l: p X (w x | q Y (v z | u Z)^l'')^l'
                                   -> p' X (w' x | q' Y (v' z | u' Z)^l'')^l'
                                contexts: grandchild slots of label l'' under
                                a slot of label l' under one of label l     */
  CWC_RULE_PAIR = 6          /* two compartments in one left-hand side, both
                                kept, each with its own right-hand side:
                                l: p X (w1 x1 | q1 Y1)^l' (w2 x2 | q2 Y2)^l'
                                   -> p' X (w1' x1 | q1' Y1)^l' (w2' x2 | q2' Y2)^l'
                                contexts: ordered pairs of sibling l' slots,
                                unordered when both the left- and the right-
                                hand patterns of the two compartments are
                                identical (a match and its swap then give the
                                same term)                                   */
};

/*
 * Model description (host memory).
 *   n_species S >= 1, n_labels L >= 1 (label 0 = the top level, whose single
 *   compartment is slot 0, the root, without a wrap), n_rules M >= 1,
 *   max_compartments C >= 1 (slots per trajectory, including the root).
 *   kind[M], ctx_label[M] in [0, L), child_label[M] in [1, L) (ignored, and
 *   conventionally -1, for LOCAL).
 *   lhs[M][3][S]: multiplicities of the context (parent) content, child wrap
 *   and child content patterns, each in {0, 1, 2}; rhs[M][3][S] >= 0 the
 *   same for the right-hand side (<= 1000).  LOCAL uses row 0 only; CREATE
 *   uses lhs row 0 and rhs rows 0..2 (rows 1, 2 = the new compartment's wrap
 *   and content); DISSOLVE uses lhs rows 0..2 and rhs row 0.  At most four
 *   species with a nonzero left-hand multiplicity per rule.
 *   FUSION, NESTED and PAIR rules need two more pattern rows and NESTED a
 *   third label (all three pointers may be NULL when no rule is of those
 *   kinds): grand_label[M] in [1, L) for NESTED (ignored otherwise);
 *   lhs_ext[M][2][S] (in {0, 1, 2}) and rhs_ext[M][2][S] (<= 1000): rows 3
 *   and 4, the second child's wrap and content (FUSION, whose rhs rows 3, 4
 *   must be 0; its rhs rows 1, 2 are added to the merged wrap and content;
 *   PAIR, whose rhs rows 1, 2 and 3, 4 are the two compartments' new wrap
 *   and content patterns) or the grandchild's wrap and content (NESTED).
 * Flat mass-action networks are L = 1, C = 1, all rules LOCAL on label 0.
 *   Rate laws (Sec. 2.2 takes mass action as the usual rate and allows other
 *   kinetics; both pointers may be NULL, meaning mass action throughout):
 *   rate_law[M]: 0 = mass action, h_j = the number of reactant
 *   combinations; 1 + s = Michaelis-Menten kinetics of substrate species s,
 *   rate_par[M] = the Michaelis constant K_j (in molecules, > 0, finite;
 *   read only for those rules).  A Michaelis-Menten rule belongs to a flat
 *   model, is LOCAL and has one or two reactant species, each of
 *   multiplicity 1, among them s; the other one, if any, is the enzyme E:
 *       h_j = RN(RN(n_E * n_s) / RN(K_j + n_s))   or   RN(n_s / RN(K_j + n_s)),
 *   each step one IEEE double operation, a_j = RN(k_j * h_j).  Anything else
 *   is CWC_ERR_INVALID_ARG.  Such models run the flat kernel's
 *   Michaelis-Menten variant and not CWC_LAYOUT_TAIL.
 */
typedef struct {
  int32_t n_species;
  int32_t n_labels;
  int32_t n_rules;
  int32_t max_compartments;
  const int32_t* kind;
  const int32_t* ctx_label;
  const int32_t* child_label;
  const int32_t* lhs;
  const int32_t* rhs;
  const int32_t* grand_label;   /* [M] or NULL */
  const int32_t* lhs_ext;       /* [M][2][S] or NULL */
  const int32_t* rhs_ext;       /* [M][2][S] or NULL */
  const int32_t* rate_law;      /* [M] or NULL (all mass action) */
  const double* rate_par;       /* [M] or NULL */
} cwc_model_desc;

typedef struct cwc_model cwc_model;

/*
 * Validate a model, compile it (reactant lists, stoichiometry changes, the
 * rule dependency graph and the propensity-tree paths each rule touches)
 * and upload the tables to the current device.
 * Errors: CWC_ERR_INVALID_ARG (NULL pointers, sizes or fields out of
 * range), CWC_ERR_UNSUPPORTED (more than four reactant species in a rule,
 * a model too large for one trajectory's state), CWC_ERR_CUDA.
 * On success *out owns device memory until cwc_model_destroy.
 */
cwc_status cwc_model_create(const cwc_model_desc* desc, cwc_model** out);

/* Free a model (NULL is ignored).  Work using it must have completed. */
void cwc_model_destroy(cwc_model* model);

/*
 * Number of observables O per grid point: S for a flat model (the root
 * content); otherwise L*S content totals by label, (L-1)*S wrap totals for
 * labels 1..L-1, and L alive-compartment counts, each an int64 sum
 * saturated at INT32_MAX.  Returns -1 for NULL.
 */
int32_t cwc_model_num_observables(const cwc_model* model);

/* Layout choices for cwc_sim_args.layout. */
enum {
  CWC_LAYOUT_AUTO = 0,        /* the autotuner's cached choice for this shape   */
  CWC_LAYOUT_STATIC = 1,      /* one thread per trajectory; a lane that finishes
                                 takes trajectory q + (threads in the grid)     */
  CWC_LAYOUT_QUEUE = 2,       /* persistent grid; a lane that finishes takes the
                                 next trajectory from a device work queue       */
  CWC_LAYOUT_TAIL = 3         /* flat mass-action models, forward only (no
                                 deadline, no checkpoint, no sensitivities): the
                                 queue layout,
                                 then, once the queue is empty and at most
                                 tail_threshold trajectories still run, those
                                 stop at their next 1024-event boundary and are
                                 finished by a group of 16 lanes each, longest
                                 predicted remaining work first (prediction: events
                                 so far x (T - t) / t).  Shortens the makespan of
                                 batches of uneven trajectory length (parameter
                                 sweeps); results are identical to the other
                                 layouts                                        */
};

/*
 * Arguments of one simulation call: P sweep points x R replicas, trajectory
 * q = p*R + r (p < P, r < R), sampled at G grid points.  The random stream
 * of trajectory q is keyed by (replica_offset + r, p), so splitting a batch's
 * replicas into shards with matching offsets reproduces it exactly.
 *
 *   rates   device double [P][M]    stochastic constants k_j > 0 per point
 *   init    device int32 [Pi][S] (flat) or [Pi][C][3+2S] slot image per
 *           point (Pi = 1: shared by all points): row c = (alive, label,
 *           parent, wrap[S], content[S]); slot 0 must be the root
 *   grid    device double [G], 0 <= grid[0] < grid[1] < ...; T = grid[G-1]
 *   seed    Philox4x32-10 key (low word, high word)
 *   max_events  per trajectory, 0 .. 2^32-1
 *
 * Outputs (device, each may be NULL):
 *   states        int32 [P][R][G][O]   observables at each grid point; device
 *                                      memory or page-locked host memory
 *                                      (cudaHostAlloc / cudaHostRegister),
 *                                      which the kernel writes directly over
 *                                      the host link while it runs (no copy
 *                                      afterwards); pageable host memory is
 *                                      CWC_ERR_INVALID_ARG
 *   sums          int64 [P][G][O]      exact sums over replicas (zeroed by
 *                                      the call before accumulation)
 *   means         double [P][G][O]     sums / R (one IEEE division)
 *   sumsq         uint64 [P][G][O][2]  exact 128-bit sums of squares over
 *                                      replicas, (low word, high word); zeroed
 *                                      by the call
 *   variance      double [P][G][O]     sample variance over replicas:
 *                                      RN(R*sumsq - sums^2) / (R * (R - 1)),
 *                                      0 when R = 1 (the numerator is exact)
 *   ci90          double [P][G][O]     half-width of the 90 % normal-
 *                                      approximation confidence interval of
 *                                      the mean: z * sqrt(variance / R),
 *                                      z = 1.6448536269514722 (Sec. 5.2:
 *                                      on-line mean, variance, confidence)
 *   traj_status   int32 [P][R]         CWC_TRAJ_* codes
 *   traj_events   int64 [P][R]         applied events
 *   traj_hash     uint64 [P][R]        FNV-1a-64 over (rule, slot) of every
 *                                      applied event, little-endian uint32s
 *   traj_final_t  double [P][R]        time of the last applied event
 *   log_rule/log_slot int32, log_t double [P][R][log_cap]: the first log_cap
 *                                      events of each trajectory (the slot is
 *                                      the context; for FUSION the pair
 *                                      d1 | d2 << 16, also in the hash)
 *
 *   checkpoint    int32 [P][R][cwc_checkpoint_words()]  the state of each
 *                 trajectory when it stops: time, event hash, event count,
 *                 next grid point, status, then the counts (flat models) or
 *                 the term as a slot image in the layout of init
 *                 (compartmentalised models).  With a
 *                 checkpoint buffer a trajectory stopped by the deadline
 *                 leaves its remaining grid points unrecorded, and a later
 *                 call with resume = 1 (same batch, seed, grid and outputs)
 *                 continues every trajectory whose saved status is
 *                 CWC_TRAJ_TIMEOUT from where it stopped and leaves the others
 *                 untouched; the result equals an uninterrupted run bit for
 *                 bit, because the random streams are keyed by the event
 *                 index (the stop / restart of instances in Sec. 5.2).  Not
 *                 combinable with sums, means, sumsq, variance or ci90.
 *   lanes         lanes of a warp per trajectory: 0 = automatic (the
 *                 autotuner's choice for this batch shape, else 1 for flat
 *                 models and 4 for compartment models), or 1, 4, 8
 *                 (compartment models; flat models take 1).  A group of lanes
 *                 computes one trajectory's scalar work identically and
 *                 shares its context scans, totals updates and grid records;
 *                 the results do not depend on this choice.
 *   layout, block_threads (0 = automatic), deadline_ns (0 = none: a
 *   trajectory still running when this many nanoseconds of device time have
 *   passed since the launch stops with CWC_TRAJ_TIMEOUT.  The clock is read
 *   every 1024 events, and not before the trajectory has applied 1024 events
 *   in this call, so every call advances each unfinished trajectory).
 *   workspace / workspace_bytes: caller-owned device scratch of at least
 *   cwc_simulate_workspace_size() bytes, 256-byte aligned (NULL if that size
 *   is 0).
 *
 * Semantics of each trajectory (the written specification this library and
 * its test oracle both follow; Sec. 2.2 steps 1-2 with Sec. 5.1's order):
 * per event n, Philox4x32-10 with counter (n, 0, r, p) gives u_tau, u_sel
 * (52-bit uniforms (k + 1/2) 2^-52); a0 is the 32-lane blocked FP64 tree
 * sum of a_j = k_j * H_j (H_j the int64 number of reactant combinations
 * summed over the rule's contexts); tau = -log(u_tau) / a0 with a fixed
 * logarithm evaluated in integer fixed point (the Mercator series near 1,
 * else a 64-entry table of ln(1 + j/64) and the Mercator series of the
 * remainder, rounded once to nearest); grid points before t + tau record the current
 * term; an event past T is discarded; rule j is chosen by guarded tree
 * descent of u_sel * a0; its context by the integer draw
 * floor(W * H_j / 2^64), W from counter (n, 1, r, p); then the rewrite.
 */
typedef struct {
  int32_t P, R, G, Pi;
  uint32_t replica_offset;   /* replica r of this call is replica r + replica_offset of
                                the random streams (shards of one large batch) */
  const double* rates;
  const int32_t* init;
  const double* grid;
  uint64_t seed;
  int64_t max_events;
  int32_t* states;
  int64_t* sums;
  double* means;
  uint64_t* sumsq;
  double* variance;
  double* ci90;
  int32_t* traj_status;
  int64_t* traj_events;
  uint64_t* traj_hash;
  double* traj_final_t;
  int32_t log_cap;
  int32_t* log_rule;
  int32_t* log_slot;
  double* log_t;
  int32_t* checkpoint;
  int32_t resume;
  int32_t layout;
  int32_t block_threads;
  int32_t lanes;
  int64_t deadline_ns;
  void* workspace;
  size_t workspace_bytes;
  int32_t tail_threshold;    /* CWC_LAYOUT_TAIL: hand over when at most this many
                                trajectories run (0 = 108 per SM) */
  int32_t term_bits;         /* compartment models: 0 or 32 = 32-bit term counts;
                                16 = 16-bit counts (half the term slab bytes, so
                                a full GPU's terms stay in L2) for forward calls
                                without FUSION / NESTED / PAIR rules, deadline or
                                checkpoints: a trajectory whose count would leave
                                int16's range is saved and finished by a 32-bit
                                launch that redraws the same event, so results
                                are identical; the workspace then also holds
                                4 * P * R * (8 + C * (3 + 2S)) bytes of those
                                hand-over records.  Ignored for flat models;
                                other values are CWC_ERR_INVALID_ARG */
} cwc_sim_args;

/*
 * cwc_simulate_noalloc: the same simulation as cwc_simulate for callers that
 * cannot allocate device memory, so cannot size and pass a workspace (for
 * example code whose device memory is owned by another framework's pool, or
 * a service with a fixed device-memory budget reserved up front).  The paper
 * has no counterpart: this is an interface convenience of this library.
 *
 * The scratch it needs lives in one statically sized device array of
 * CWC_NOALLOC_SCRATCH_BYTES inside the library; every GPU that loads the
 * library holds that array until the process exits.  args->workspace and
 * args->workspace_bytes are ignored.  The scratch is what
 * cwc_simulate_workspace_size reports for the same arguments, less the
 * hand-over records of 16-bit terms (term_bits = 16): this entry point runs
 * 32-bit terms throughout.  A call fits when that is <=
 * CWC_NOALLOC_SCRATCH_BYTES.  Its parts, each rounded up to 256 bytes:
 *   - 256 bytes: work-queue ticket and deadline timestamp;
 *   - 8 * P * G * O: int64 replica sums, when means, variance or ci90 are
 *     requested without sums;
 *   - 16 * P * G * O: 128-bit sums of squares, when variance or ci90 are
 *     requested without sumsq;
 *   - 12 * P: the longest-first sweep order of a flat model in the queue
 *     layout with P > 1;
 *   - compartment models: one term slab per resident lane group of the
 *     launch, about 13 KB each for 64 slots x 24 species; a compartment
 *     batch therefore fits only while it occupies a few dozen lane groups
 *     (roughly 70-80 trajectories at 4 lanes each for such a model).
 * A call that needs more returns CWC_ERR_INVALID_ARG and enqueues nothing.
 * It calls no cudaMalloc or cudaFree.
 *
 * The first call on each device looks up the array's device address with
 * that device current and caches it for the life of the process; make that
 * first call before any stream capture.  The cached address does not survive
 * a reset of the device's primary context (cudaDeviceReset): do not call this
 * entry point on a device after resetting it.  All calls on a device share
 * the one array and each clears what must start at zero, so calls whose work
 * overlaps on the GPU (different streams, or different host threads) race on
 * it: serialise them.
 */
#define CWC_NOALLOC_SCRATCH_BYTES (1u << 20)
cwc_status cwc_simulate_noalloc(const cwc_model* model, const cwc_sim_args* args, void* stream);

/* int32 words of one trajectory's checkpoint record: 8 + S for flat models,
 * 8 + C * (3 + 2S) for compartmentalised ones; -1 for a NULL model. */
int32_t cwc_checkpoint_words(const cwc_model* model);

/* Workspace bytes cwc_simulate needs for these arguments (0 if none). */
cwc_status cwc_simulate_workspace_size(const cwc_model* model, const cwc_sim_args* args, size_t* bytes);

/*
 * Enqueue the simulation described by args on stream.
 * Errors: CWC_ERR_INVALID_ARG (NULL model/args/rates/init/grid, P, R, G < 1,
 * Pi not 1 or P, replica_offset + R > 2^32, max_events out of range,
 * log_cap < 0 or a log buffer missing), CWC_ERR_WORKSPACE,
 * CWC_ERR_UNSUPPORTED, CWC_ERR_CUDA.
 */
cwc_status cwc_simulate(const cwc_model* model, const cwc_sim_args* args, void* stream);

/*
 * Likelihood-ratio sensitivities of mean observables with respect to the
 * rate constants, by replaying every trajectory's Philox stream (the same
 * paths cwc_simulate produces for the same args; nothing is stored between
 * the calls).  For a CTMC path the score of rule j up to time g is
 * S_j(g) = N_j(g)/k_j - int_0^g H_j(X(s)) ds (a_j = k_j H_j); with the
 * upstream gradient G = grad_means[p][g][o] of L = sum G * E[X_o(g)],
 *   grad_rates[p][j] = (1/R) sum_r sum_g c_r(g) S_rj(g),
 *   c_r(g) = sum_o G[p][g][o] (X_ro(g) - means[p][g][o]).
 *
 *   means, grad_means  device double [P][G][O]
 *   grad_rates         device double [P][M]   (output)
 *   partials           device double [P][R][M] per-trajectory terms
 *                      (output if non-NULL, else kept in the workspace)
 * A trajectory that stops with CWC_TRAJ_PROP_OVERFLOW counts H_j as 0 after
 * its last applied event; any other stop keeps the last H_j up to the end of
 * the grid.  The sum over r is a fixed pairwise tree, so results are
 * identical from run to run.  Workspace: cwc_sensitivity_workspace_size().
 * Errors as cwc_simulate, plus CWC_ERR_INVALID_ARG for missing
 * means/grad_means/grad_rates.
 */
typedef struct {
  const double* means;
  const double* grad_means;
  double* grad_rates;
  double* partials;
} cwc_sens_args;

cwc_status cwc_sensitivity_workspace_size(const cwc_model* model, const cwc_sim_args* sim,
                                          const cwc_sens_args* sens, size_t* bytes);
cwc_status cwc_sensitivity(const cwc_model* model, const cwc_sim_args* sim, const cwc_sens_args* sens,
                           void* stream);

/*
 * Pick the launch layout (CWC_LAYOUT_STATIC or CWC_LAYOUT_QUEUE), the
 * threads per block and the lanes per trajectory (1, 4, 8 for compartment
 * models; 1 for flat ones) for these arguments by timing every candidate on
 * this batch with at most `tune_events` events per trajectory (0 = 2048) and
 * no outputs; all candidates do identical work because the random streams are
 * keyed by (event, replica, point), not by thread.  On GB300 an FP64
 * instruction costs a full warp slot whatever the number of active lanes, so
 * several lanes per trajectory pay off only where the per-trajectory work
 * beyond the FP64 step (context scans, totals over compartments) dominates
 * or the batch is too small to fill the GPU one lane per trajectory.  The
 * winner is returned (best_lanes may be NULL) and cached for this model and
 * batch shape; later calls with layout CWC_LAYOUT_AUTO, block_threads 0 and
 * lanes 0 use it.  Synchronises `stream`.  Uses args->workspace (a candidate
 * that needs more than workspace_bytes is skipped).
 * Errors: as cwc_simulate; CWC_ERR_INTERNAL if no candidate could run.
 */
cwc_status cwc_autotune(const cwc_model* model, const cwc_sim_args* args, int64_t tune_events, void* stream,
                        int32_t* best_layout, int32_t* best_block_threads, double* best_ms, int32_t* best_lanes);

/*
 * The fixed logarithm of the time step (the integer fixed-point evaluation
 * described above, one rounding to nearest at the end) evaluated on the
 * device for n values: out[i] = log_spec(u[i]).  For checking the kernels'
 * logarithm against a CPU implementation bit for bit.  u and out are device
 * arrays of n doubles (caller-owned); inputs outside [2^-53, 1), the range of
 * the 52-bit uniforms, give NaN.  Asynchronous on `stream`.
 * Errors: CWC_ERR_INVALID_ARG (n < 0, NULL arrays), CWC_ERR_CUDA.
 */
cwc_status cwc_log_spec(const double* u, double* out, int64_t n, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* cwc_last_error(void);

/* Library version string. */
const char* cwc_version(void);

/*
 * The FP64 pipe's peak rate on the current device, measured (a diagnostic;
 * the paper has no counterpart): a grid of 32 warps per SM runs eight
 * independent chains of unfused round-to-nearest double multiplies and adds
 * (the FP64 instructions the simulation kernels issue) for ~20 ms, timed with
 * CUDA events (best of three after a warm-up).  *lane_ops_per_s = thread-level
 * FP64 operations per second.  It is the denominator of the kernels' FP64
 * roofline.  Synchronises `stream`; allocates nothing.
 * Errors: CWC_ERR_INVALID_ARG (NULL output), CWC_ERR_CUDA.
 */
cwc_status cwc_fp64_peak(void* stream, double* lane_ops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* CWCGPU_H_ */
