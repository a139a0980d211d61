// C ABI of the library (declared in include/cwcgpu.h): model validation and
// compilation, argument checking, workspace layout and kernel launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "cwc_internal.h"
#include "cwcgpu.h"
#include "ssa_device.cuh"

namespace cwcgpu {
cudaError_t launch_flat(const FlatParams& prm, const LogConstants& lc, bool queue, bool sens, int T,
                        int blocks_per_sm_cap, cudaStream_t stream, int* used_blocks);
size_t flat_smem_bytes(const FlatParams& prm, int T, bool sens);
int flat_table_bytes_host(int M, int n_deps);
int flat_auto_threads(const FlatParams& prm, bool queue, bool sens);
cudaError_t launch_flat_order(const FlatParams& prm, double* est, int32_t* order, cudaStream_t stream);
cudaError_t launch_flat_tail(const FlatParams& prm, const LogConstants& lc, int32_t* list, double* est,
                             int32_t* order, cudaStream_t stream);
cudaError_t launch_means(const unsigned long long* sums, double* means, long long n, int R, cudaStream_t st);
cudaError_t launch_reciprocal(const double* k, double* inv, long long n, cudaStream_t st);
cudaError_t launch_stats(const unsigned long long* sums, const unsigned long long* sumsq, double* variance,
                         double* ci90, long long n, int R, cudaStream_t st);
cudaError_t launch_reduce_partials(const double* partials, double* grad, int P, int R, int M, cudaStream_t st);
cudaError_t launch_cwc(const CwcParams& prm, const LogConstants& lc, bool queue, int lanes, int T, int blocks,
                       cudaStream_t stream);
cudaError_t cwc_launch_shape(const CwcParams& prm, bool queue, int lanes, int T, int* blocks);
int cwc_best_threads(const CwcParams& prm, bool queue, int lanes);
cudaError_t launch_log_spec(const double* u, double* out, long long n, const LogConstants& lc, cudaStream_t st);
bool cwc_lanes_supported(int lanes);
int cwc_thread_bytes_host(int M);
int cwc_table_bytes_host(int M, int n_deps);
long long cwc_slab_words_host(int S, int L, int C, int M, bool sens);
}  // namespace cwcgpu

using namespace cwcgpu;

struct cwc_model {
  int S = 0, L = 0, C = 0, M = 0;
  bool flat = false;
  int device = 0;
  // flat compilation
  int B = 1, n_deps = 0;
  int checked_counts = 0;
  int mm_off = -1;              // Michaelis-Menten tables' word offset in d_tables (-1: none)
  int pool = 0;                 // flat kernel: leaves rebuilt by the warp together
  int32_t* d_tables = nullptr;  // [M][RULE_WORDS], [n_deps], [M] descriptors, log tables (cwc_internal.h)
  std::vector<int32_t> h_tables;
  // compartmentalised compilation
  int O = 0;
  int c_n_deps = 0;
  bool general = false;          // some rule is FUSION or NESTED
  int32_t* d_ctables = nullptr;  // [M][CWC_RULE_WORDS] followed by [c_n_deps]
  std::vector<int32_t> h_ctables;
};

namespace {

thread_local std::string g_last_error;

cwc_status fail(cwc_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

cwc_status cuda_fail(cudaError_t e, const char* what) {
  return fail(CWC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Constants of the time step's logarithm: floor(2^63 / n); ln 2 in Q120 as
// the truncated sum of floor(2^(120-k) / k), k = 1..120 (ln 2 = sum over k
// of 1 / (k 2^k)); per prefix j, ceil(2^69 / (64 + j)) and ln(1 + j/64) in
// Q64 from 2 atanh(s), s = j / (128 + j): s floored in Q64, the series
// 1 + s^2/3 + ... + s^38/39 by Horner in Q63, then 2 s P floored to Q64.
LogConstants make_log_constants() {
  typedef unsigned __int128 u128;
  LogConstants lc;
  std::memset(&lc, 0, sizeof(lc));
  const u128 one = 1;
  for (int n = 1; n < 40; ++n) lc.cq[n] = (unsigned long long)((one << 63) / (u128)n);
  u128 ln2 = 0;
  for (int k = 1; k <= 120; ++k) ln2 += (one << (120 - k)) / (u128)k;
  lc.ln2_lo = (unsigned long long)ln2;
  lc.ln2_hi = (unsigned long long)(ln2 >> 64);
  auto hi64 = [](unsigned long long a, unsigned long long b) { return (unsigned long long)(((u128)a * b) >> 64); };
  for (int j = 0; j < 64; ++j) {
    lc.rj[j] = (unsigned long long)(((one << 69) + (u128)(63 + j)) / (u128)(64 + j));
    const unsigned long long s = (unsigned long long)(((u128)j << 64) / (u128)(128 + j));
    const unsigned long long z = hi64(s, s);
    unsigned long long p = lc.cq[39];
    for (int k = 37; k >= 3; k -= 2) p = lc.cq[k] + hi64(p, z);
    p = (1ull << 63) + hi64(p, z);
    lc.tj[j] = (unsigned long long)(((u128)s * p) >> 62);
  }
  return lc;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout: [header 256 B][sums P*G*O int64 if needed][partials Q*M double if needed]
struct WsLayout {
  size_t header = 0, sums = 0, sumsq = 0, partials = 0, slabs = 0, order = 0, sens_acc = 0, inv_rates = 0, total = 0;
  size_t tail = 0;                // tail layout: checkpoints [Q][S+8] i32, list [Q] i32, est [Q] f64, order [Q] i32
  bool need_tail = false;
  bool need_sumsq = false;
  bool need_order = false;        // flat queue layout over several sweep points
  bool need_header = false, need_sums = false, need_partials = false;
  int T = 0, blocks = 0, lanes = 1;   // compartmentalised launch shape (its slabs are per lane group)
  long long slab_words = 0;
  bool narrow = false;            // compartment forward: a 16-bit launch, then a 32-bit one resuming
  size_t narrow_ckpt = 0;         // the trajectories handed over: [Q][CKPT_HEADER_WORDS + C(3 + 2S)] int32
};

CwcParams cwc_shape_params(const cwc_model* m, const cwc_sim_args* a, bool sens) {
  CwcParams prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.S = m->S;
  prm.L = m->L;
  prm.C = m->C;
  prm.M = m->M;
  prm.B = m->B;
  prm.O = m->O;
  prm.n_deps = m->c_n_deps;
  prm.general = m->general ? 1 : 0;
  prm.Q = (long long)a->P * a->R;
  prm.smem_table_bytes = cwc_table_bytes_host(m->M, m->c_n_deps);
  prm.sens = sens ? 1 : 0;
  prm.slab_words = cwc_slab_words_host(m->S, m->L, m->C, m->M, sens);
  return prm;
}

// Autotuner cache: (model, P, R, G, Pi) -> (layout, threads per block, lanes per trajectory).
std::mutex g_tune_mutex;
std::map<std::tuple<const void*, int, int, int, int>, std::tuple<int, int, int>> g_tune_cache;

bool tuned_choice(const cwc_model* m, const cwc_sim_args* a, int* layout, int* threads, int* lanes) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tune_cache.find(std::make_tuple((const void*)m, a->P, a->R, a->G, a->Pi));
  if (it == g_tune_cache.end()) return false;
  *layout = std::get<0>(it->second);
  *threads = std::get<1>(it->second);
  *lanes = std::get<2>(it->second);
  return true;
}

// Lanes per trajectory when the caller leaves it to the library (and the
// autotuner has not chosen): one for flat networks, so that every FP64
// instruction of the step serves 32 trajectories; four for compartment
// terms, whose context scans and totals updates over compartments outweigh
// their FP64 step (1.9e8 against 1.5e8 events/s with one lane on a
// 16,384-term batch with 48 rules).
int chosen_lanes(const cwc_model* m, const cwc_sim_args* a) {
  if (m->flat) return 1;
  return a->lanes > 0 ? a->lanes : 4;
}

int chosen_layout(const cwc_sim_args* a) { return a->layout == CWC_LAYOUT_AUTO ? CWC_LAYOUT_QUEUE : a->layout; }

// the queue-driven layouts: the persistent grid with a work ticket
bool queue_layout(const cwc_sim_args* a) {
  return chosen_layout(a) == CWC_LAYOUT_QUEUE || chosen_layout(a) == CWC_LAYOUT_TAIL;
}

// Resolve CWC_LAYOUT_AUTO / block_threads 0 through the autotuner cache.
cwc_sim_args resolve_auto(const cwc_model* m, const cwc_sim_args* a) {
  cwc_sim_args b = *a;
  int lay = 0, thr = 0, lanes = 0;
  if (a->layout == CWC_LAYOUT_AUTO && a->block_threads == 0 && a->lanes == 0 && tuned_choice(m, a, &lay, &thr, &lanes)) {
    b.layout = lay;
    b.block_threads = thr;
    b.lanes = lanes;
  }
  return b;
}

// Shrink an automatically chosen block size until the grid (one thread per
// trajectory at most) has at least one block per SM: a small batch would
// otherwise leave SMs idle with the largest block that fits.
int cover_sms(int T, long long Q) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return T;
  while (T > 32 && (Q + T - 1) / T < sms) T -= 32;
  return T;
}

// allow_narrow: compartment forwards may run as a 16-bit launch followed by a
// 32-bit one (which needs the hand-over records in the workspace)
WsLayout ws_layout(const cwc_model* m, const cwc_sim_args* a, bool sens, bool sens_partials_given,
                   bool allow_narrow = true) {
  WsLayout w;
  const int O = m->flat ? m->S : (m->L * m->S + (m->L - 1) * m->S + m->L);
  w.need_header = queue_layout(a) || a->deadline_ns > 0;
  const bool stats = a->variance != nullptr || a->ci90 != nullptr;
  w.need_sums = !sens && (a->means != nullptr || stats) && a->sums == nullptr;
  w.need_sumsq = !sens && stats && a->sumsq == nullptr;
  w.need_partials = sens && !sens_partials_given;
  size_t off = 0;
  if (w.need_header) {
    w.header = off;
    off += 256;
  }
  if (w.need_sums) {
    w.sums = off;
    off = align256(off + (size_t)a->P * a->G * O * sizeof(long long));
  }
  if (w.need_sumsq) {
    w.sumsq = off;
    off = align256(off + (size_t)a->P * a->G * O * 2 * sizeof(unsigned long long));
  }
  if (w.need_partials) {
    w.partials = off;
    off = align256(off + (size_t)a->P * a->R * m->M * sizeof(double));
  }
  if (m->flat && sens) {   // the flat replay's per-trajectory integrals, times and firing counts
    w.sens_acc = off;      // per trajectory: V [M], firing counts [M]
    off = align256(off + (size_t)a->P * a->R * 2 * (size_t)m->M * sizeof(double));
    w.inv_rates = off;     // 1 / k per sweep point and rule
    off = align256(off + (size_t)a->P * m->M * sizeof(double));
  }
  w.need_order = m->flat && queue_layout(a) && a->P > 1 && a->P <= 65536;
  if (w.need_order) {
    w.order = off;
    off = align256(off + (size_t)a->P * (sizeof(double) + sizeof(int32_t)));
  }
  w.need_tail = m->flat && !sens && chosen_layout(a) == CWC_LAYOUT_TAIL;
  if (w.need_tail) {
    const size_t Q = (size_t)a->P * a->R;
    w.tail = off;
    off = align256(off + Q * ((size_t)(m->S + CKPT_HEADER_WORDS) * 4 + 4 + 8 + 4) + 256);
  }
  if (!m->flat) {
    const CwcParams prm = cwc_shape_params(m, a, sens);
    const bool queue = chosen_layout(a) == CWC_LAYOUT_QUEUE;
    w.lanes = chosen_lanes(m, a);
    w.T = a->block_threads > 0 ? a->block_threads
                               : cover_sms(cwc_best_threads(prm, queue, w.lanes), prm.Q * (long long)w.lanes);
    if (cwc_launch_shape(prm, queue, w.lanes, w.T, &w.blocks) != cudaSuccess) w.blocks = 0;
    w.slab_words = prm.slab_words;
    w.slabs = off;
    off = align256(off + (size_t)w.blocks * (size_t)(w.T / w.lanes) * (size_t)prm.slab_words * sizeof(int32_t));
    // Terms with 16-bit counts (term_bits = 16) halve the slab bytes a
    // trajectory touches, so that the slabs of a full GPU's terms stay in L2
    // (DRAM 238 -> 82 B per event on 16,384 terms of 24 species), but the
    // 16-bit kernel ran 2 % slower there (more instruction-fetch stalls), so
    // 32-bit terms stay the default.  A trajectory whose count would leave
    // int16's range is handed to a 32-bit launch through a checkpoint
    // record.  Forward calls without FUSION / NESTED / PAIR rules, deadline
    // or caller checkpoints only (others run 32-bit terms).
    w.narrow = allow_narrow && a->term_bits == 16 && !sens && !m->general && a->deadline_ns == 0 &&
               a->checkpoint == nullptr && a->resume == 0;
    if (w.narrow) {
      w.narrow_ckpt = off;
      const size_t words = (size_t)CKPT_HEADER_WORDS + (size_t)m->C * (3 + 2 * (size_t)m->S);
      off = align256(off + (size_t)a->P * a->R * words * sizeof(int32_t));
    }
  }
  w.total = off;
  return w;
}

cwc_status check_sim_args(const cwc_model* m, const cwc_sim_args* a) {
  if (m == nullptr || a == nullptr) return fail(CWC_ERR_INVALID_ARG, "model and args must not be NULL");
  if (a->rates == nullptr || a->init == nullptr || a->grid == nullptr)
    return fail(CWC_ERR_INVALID_ARG, "rates, init and grid must not be NULL");
  if (a->P < 1 || a->R < 1 || a->G < 1) return fail(CWC_ERR_INVALID_ARG, "P, R and G must be >= 1");
  if (a->Pi != 1 && a->Pi != a->P) return fail(CWC_ERR_INVALID_ARG, "Pi must be 1 or P");
  if ((unsigned long long)a->replica_offset + (unsigned long long)a->R > 0x100000000ull)
    return fail(CWC_ERR_INVALID_ARG, "replica_offset + R must be <= 2^32");
  if (a->max_events < 0 || a->max_events > 0xFFFFFFFFll)
    return fail(CWC_ERR_INVALID_ARG, "max_events must be in [0, 2^32-1]");
  if (a->log_cap < 0) return fail(CWC_ERR_INVALID_ARG, "log_cap must be >= 0");
  if (a->log_cap > 0 && a->log_rule == nullptr) return fail(CWC_ERR_INVALID_ARG, "log_cap > 0 needs log_rule");
  if (a->layout < CWC_LAYOUT_AUTO || a->layout > CWC_LAYOUT_TAIL) return fail(CWC_ERR_INVALID_ARG, "bad layout");
  if (a->layout == CWC_LAYOUT_TAIL &&
      (!m->flat || m->mm_off >= 0 || a->deadline_ns != 0 || a->checkpoint != nullptr || a->resume != 0))
    return fail(CWC_ERR_INVALID_ARG,
                "CWC_LAYOUT_TAIL is for flat mass-action models without deadline or checkpoints");
  if (a->tail_threshold < 0) return fail(CWC_ERR_INVALID_ARG, "tail_threshold must be >= 0");
  if (a->term_bits != 0 && a->term_bits != 16 && a->term_bits != 32)
    return fail(CWC_ERR_INVALID_ARG, "term_bits must be 0, 16 or 32");
  if (a->block_threads != 0 && (a->block_threads < 32 || a->block_threads > 256 || a->block_threads % 32 != 0))
    return fail(CWC_ERR_INVALID_ARG, "block_threads must be 0 or a multiple of 32 in [32, 256]");
  if (a->lanes != 0 && !(m->flat ? a->lanes == 1 : cwc_lanes_supported(a->lanes)))
    return fail(CWC_ERR_INVALID_ARG, m->flat ? "lanes must be 0 or 1 for flat models"
                                             : "lanes must be 0, 1, 4 or 8 for compartment models");
  if (a->deadline_ns < 0) return fail(CWC_ERR_INVALID_ARG, "deadline_ns must be >= 0");
  if (a->resume != 0 && a->resume != 1) return fail(CWC_ERR_INVALID_ARG, "resume must be 0 or 1");
  if (a->resume && a->checkpoint == nullptr) return fail(CWC_ERR_INVALID_ARG, "resume needs the checkpoint buffer");
  if (a->checkpoint != nullptr &&
      (a->sums != nullptr || a->means != nullptr || a->sumsq != nullptr || a->variance != nullptr || a->ci90 != nullptr))
    return fail(CWC_ERR_INVALID_ARG, "checkpoints cannot be combined with reductions over replicas");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != m->device) return fail(CWC_ERR_INVALID_ARG, "model was created on another device");
  return CWC_OK;
}

// The grid states may be device memory or page-locked host memory
// (cudaHostAlloc, cudaHostRegister): the latter through its device mapping,
// so that the kernels store the states across the host link (NVLink-C2C on
// Grace systems) while they run and no copy follows.  Pageable host memory
// is refused.  While the stream is being captured into a graph the pointer
// is taken as it is (no queries during capture; page-locked memory has the
// same address on the device under unified addressing).
cwc_status states_ptr(int32_t* p, cudaStream_t st, int32_t** out) {
  *out = p;
  if (p == nullptr) return CWC_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return CWC_OK;
  }
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return fail(CWC_ERR_INVALID_ARG, "states: not a device or page-locked host pointer");
  }
  if (at.type == cudaMemoryTypeUnregistered)
    return fail(CWC_ERR_INVALID_ARG, "states: pageable host memory (pass device or page-locked host memory)");
  if (at.type == cudaMemoryTypeHost) {
    if (at.devicePointer == nullptr) return fail(CWC_ERR_INVALID_ARG, "states: host memory not mapped on the device");
    *out = static_cast<int32_t*>(at.devicePointer);
  }
  return CWC_OK;
}

FlatParams make_flat_params(const cwc_model* m, const cwc_sim_args* a) {
  FlatParams prm;
  std::memset(&prm, 0, sizeof(prm));
  prm.S = m->S;
  prm.M = m->M;
  prm.B = m->B;
  prm.n_deps = m->n_deps;
  prm.checked_counts = m->checked_counts;
  prm.rules = m->d_tables;
  prm.deps = m->d_tables + (size_t)m->M * RULE_WORDS;
  prm.pool = m->pool;
  if (m->mm_off >= 0) {
    prm.mm_K = reinterpret_cast<const double*>(m->d_tables + m->mm_off);
    prm.mm_desc = reinterpret_cast<const uint32_t*>(m->d_tables + m->mm_off + 2 * m->M);
  }
  prm.P = a->P;
  prm.R = a->R;
  prm.G = a->G;
  prm.Pi = a->Pi;
  prm.r_offset = a->replica_offset;
  prm.Q = (long long)a->P * a->R;
  prm.rates = a->rates;
  prm.init = a->init;
  prm.grid = a->grid;
  prm.key0 = (uint32_t)a->seed;
  prm.key1 = (uint32_t)(a->seed >> 32);
  prm.max_events = a->max_events;
  prm.deadline_ns = a->deadline_ns;
  prm.ckpt = a->checkpoint;
  prm.resume = a->resume;
  prm.smem_table_bytes = flat_table_bytes_host(m->M, m->n_deps);
  return prm;
}

int pick_threads(const cwc_model* m, const cwc_sim_args* a, const FlatParams& prm, bool queue, bool sens) {
  if (a->block_threads > 0) return a->block_threads;
  return flat_auto_threads(prm, queue, sens);
}

}  // namespace

extern "C" {

const char* cwc_last_error(void) { return g_last_error.c_str(); }

cwc_status cwc_log_spec(const double* u, double* out, int64_t n, void* stream) {
  g_last_error.clear();
  if (n < 0) return fail(CWC_ERR_INVALID_ARG, "n must be >= 0");
  if (n > 0 && (u == nullptr || out == nullptr)) return fail(CWC_ERR_INVALID_ARG, "u and out must not be NULL");
  const LogConstants lc = make_log_constants();
  cudaError_t e = launch_log_spec(u, out, (long long)n, lc, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "log kernel launch");
  return CWC_OK;
}

const char* cwc_version(void) { return "cwcgpu 0.1 (sm_103a)"; }

cwc_status cwc_model_create(const cwc_model_desc* d, cwc_model** out) {
  g_last_error.clear();
  if (d == nullptr || out == nullptr) return fail(CWC_ERR_INVALID_ARG, "desc and out must not be NULL");
  *out = nullptr;
  const int S = d->n_species, L = d->n_labels, M = d->n_rules, C = d->max_compartments;
  if (S < 1 || S > 4096 || L < 1 || L > 64 || M < 1 || M > 65535 || C < 1 || C > 1024)
    return fail(CWC_ERR_INVALID_ARG, "sizes out of range (1<=S<=4096, 1<=L<=64, 1<=M<=65535, 1<=C<=1024)");
  if (!d->kind || !d->ctx_label || !d->child_label || !d->lhs || !d->rhs)
    return fail(CWC_ERR_INVALID_ARG, "rule arrays must not be NULL");
  // pattern row r (0..4) of rule j: rows 0-2 from lhs / rhs, rows 3-4 from
  // the extension arrays (all zero when those are NULL)
  auto lrow = [&](int j, int r) -> const int32_t* {
    if (r < 3) return d->lhs + ((size_t)j * 3 + r) * S;
    return d->lhs_ext ? d->lhs_ext + ((size_t)j * 2 + (r - 3)) * S : nullptr;
  };
  auto rrow = [&](int j, int r) -> const int32_t* {
    if (r < 3) return d->rhs + ((size_t)j * 3 + r) * S;
    return d->rhs_ext ? d->rhs_ext + ((size_t)j * 2 + (r - 3)) * S : nullptr;
  };
  auto row_nonzero = [&](const int32_t* row) {
    if (row == nullptr) return false;
    for (int x = 0; x < S; ++x)
      if (row[x] != 0) return true;
    return false;
  };
  for (int j = 0; j < M; ++j) {
    const int k = d->kind[j];
    const std::string rj = "rule " + std::to_string(j);
    if (k < CWC_RULE_LOCAL || k > CWC_RULE_PAIR) return fail(CWC_ERR_INVALID_ARG, rj + ": bad kind");
    if (d->ctx_label[j] < 0 || d->ctx_label[j] >= L) return fail(CWC_ERR_INVALID_ARG, rj + ": ctx_label out of range");
    if (k != CWC_RULE_LOCAL && (d->child_label[j] < 1 || d->child_label[j] >= L))
      return fail(CWC_ERR_INVALID_ARG, rj + ": child_label out of [1, L)");
    if ((k == CWC_RULE_FUSION || k == CWC_RULE_NESTED || k == CWC_RULE_PAIR) &&
        (d->lhs_ext == nullptr || d->rhs_ext == nullptr))
      return fail(CWC_ERR_INVALID_ARG, rj + ": FUSION, NESTED and PAIR rules need lhs_ext and rhs_ext");
    if (k == CWC_RULE_NESTED && (d->grand_label == nullptr || d->grand_label[j] < 1 || d->grand_label[j] >= L))
      return fail(CWC_ERR_INVALID_ARG, rj + ": NESTED needs grand_label in [1, L)");
    int factors = 0;
    for (int r = 0; r < 5; ++r) {
      const int32_t* lo = lrow(j, r);
      const int32_t* hi = rrow(j, r);
      for (int x = 0; x < S; ++x) {
        const int lv = lo ? lo[x] : 0, hv = hi ? hi[x] : 0;
        if (lv < 0 || lv > 2) return fail(CWC_ERR_INVALID_ARG, rj + ": lhs entries must be 0, 1 or 2");
        if (hv < 0 || hv > 1000) return fail(CWC_ERR_INVALID_ARG, rj + ": rhs entries must be in [0, 1000]");
        factors += lv != 0;
      }
    }
    if (factors > MAX_REAC) return fail(CWC_ERR_UNSUPPORTED, rj + ": more than 4 reactant species");
    const bool lhs_child = row_nonzero(lrow(j, 1)) || row_nonzero(lrow(j, 2));
    const bool rhs_child = row_nonzero(rrow(j, 1)) || row_nonzero(rrow(j, 2));
    const bool lhs_more = row_nonzero(lrow(j, 3)) || row_nonzero(lrow(j, 4));
    const bool rhs_more = row_nonzero(rrow(j, 3)) || row_nonzero(rrow(j, 4));
    if (k == CWC_RULE_LOCAL && (lhs_child || rhs_child))
      return fail(CWC_ERR_INVALID_ARG, rj + ": LOCAL rules use row 0 only");
    if (k == CWC_RULE_CREATE && lhs_child)
      return fail(CWC_ERR_INVALID_ARG, rj + ": CREATE matches the context content only");
    if (k == CWC_RULE_DISSOLVE && rhs_child)
      return fail(CWC_ERR_INVALID_ARG, rj + ": DISSOLVE writes the parent content only");
    if (k <= CWC_RULE_DISSOLVE && (lhs_more || rhs_more))
      return fail(CWC_ERR_INVALID_ARG, rj + ": pattern rows 3-4 belong to FUSION, NESTED and PAIR rules");
    if (k == CWC_RULE_FUSION && rhs_more)
      return fail(CWC_ERR_INVALID_ARG, rj + ": FUSION writes the merged wrap and content through rhs rows 1-2");
    const int law = d->rate_law ? d->rate_law[j] : 0;
    if (law < 0 || law > S) return fail(CWC_ERR_INVALID_ARG, rj + ": rate_law must be 0 or 1 + a species index");
    if (law != 0) {
      // Michaelis-Menten: flat model, LOCAL, one or two reactant species of
      // multiplicity 1 among which the substrate, K > 0 finite
      const int32_t* l0 = lrow(j, 0);
      bool ok = L == 1 && C == 1 && k == CWC_RULE_LOCAL && l0[law - 1] == 1 && factors >= 1 && factors <= 2;
      for (int x = 0; x < S; ++x) ok = ok && l0[x] <= 1;
      if (!ok)
        return fail(CWC_ERR_INVALID_ARG, rj + ": Michaelis-Menten rules are LOCAL rules of flat models with one or two "
                                              "reactant species of multiplicity 1, the substrate among them");
      const double K = d->rate_par ? d->rate_par[j] : 0.0;
      if (!(K > 0.0) || !std::isfinite(K))
        return fail(CWC_ERR_INVALID_ARG, rj + ": Michaelis-Menten rules need rate_par (K) > 0 and finite");
    }
  }
  cwc_model* m = new cwc_model();
  m->S = S;
  m->L = L;
  m->C = C;
  m->M = M;
  m->flat = (L == 1 && C == 1);
  cudaError_t e = cudaGetDevice(&m->device);
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "cudaGetDevice");
  }
  m->O = m->flat ? S : (L * S + (L - 1) * S + L);
  m->B = (M + 31) / 32;
  if (!m->flat) {
    if (C > CWC_MAX_SLOTS) {
      delete m;
      return fail(CWC_ERR_UNSUPPORTED, "compartmentalised models need max_compartments <= 64");
    }
    // ---- compartmentalised compilation ----
    std::vector<int32_t>& tb = m->h_ctables;
    tb.assign((size_t)M * CWC_RULE_WORDS, 0);
    // read and write sets: location key = ((role * L) + label) * S + species, role 0 content, 1 wrap
    auto key = [&](int role, int lab, int sp) { return ((long long)role * L + lab) * S + sp; };
    std::vector<std::vector<long long>> reads(M), writes(M);
    std::vector<std::pair<int, std::vector<int32_t>>> nested_ext;
    for (int j = 0; j < M; ++j) {
      const int kind = d->kind[j], ctx = d->ctx_label[j], ch = d->child_label[j];
      const int gr = kind == CWC_RULE_NESTED ? d->grand_label[j] : 0;
      m->general |= kind == CWC_RULE_FUSION || kind == CWC_RULE_NESTED || kind == CWC_RULE_PAIR;
      int32_t* rec = tb.data() + (size_t)j * CWC_RULE_WORDS;
      rec[CR_KIND] = kind;
      rec[CR_CTX] = ctx;
      rec[CR_CHILD] = kind == CWC_RULE_LOCAL ? 0 : ch;
      rec[CR_GRAND] = gr;   // the extension offset is added below
      // the (role, label) each pattern row reads
      const int row_role[5] = {0, 1, 0, 1, 0};
      const int row_label[5] = {ctx, ch, ch, kind == CWC_RULE_NESTED ? gr : ch, kind == CWC_RULE_NESTED ? gr : ch};
      int nr = 0;
      for (int row = 0; row < 5; ++row) {
        const int32_t* lo = lrow(j, row);
        if (lo == nullptr) continue;
        for (int sp = 0; sp < S; ++sp)
          if (lo[sp] > 0) {
            rec[CR_REAC + nr++] = sp | (lo[sp] << 16) | (row << 24);
            reads[j].push_back(key(row_role[row], row_label[row], sp));
          }
      }
      rec[CR_NREAC] = nr;
      // change lists: species | delta << 16 (values = the rhs row itself)
      // a change list at dst: count at dst[base_n], entries from dst[base_d]
      auto put = [&](int32_t* dst, int base_n, int base_d, const int32_t* lo, const int32_t* hi, bool values) -> bool {
        int k = 0;
        for (int sp = 0; sp < S; ++sp) {
          const int dv = values ? (hi ? hi[sp] : 0) : (hi ? hi[sp] : 0) - (lo ? lo[sp] : 0);
          if (dv == 0) continue;
          if (k == MAX_DELTA) return false;
          dst[base_d + k++] = (int32_t)((uint32_t)sp | ((uint32_t)(dv & 0xffff) << 16));
        }
        dst[base_n] = k;
        return true;
      };
      bool ok = put(rec, CR_ND0, CR_D0, lrow(j, 0), rrow(j, 0), false);
      if (kind == CWC_RULE_PARENT_CHILD || kind == CWC_RULE_NESTED || kind == CWC_RULE_PAIR) {
        ok = ok && put(rec, CR_ND1, CR_D1, lrow(j, 1), rrow(j, 1), false) &&
             put(rec, CR_ND2, CR_D2, lrow(j, 2), rrow(j, 2), false);
      } else if (kind == CWC_RULE_CREATE || kind == CWC_RULE_FUSION) {
        ok = ok && put(rec, CR_ND1, CR_D1, nullptr, rrow(j, 1), true) && put(rec, CR_ND2, CR_D2, nullptr, rrow(j, 2), true);
      }
      if (kind == CWC_RULE_NESTED || kind == CWC_RULE_PAIR) {
        // rows 3-4 of NESTED and PAIR go to an extension record after the
        // dependency list; its offset is known once the list is, so keep it
        // aside.  PAIR's low byte says whether the two compartments' right-
        // hand patterns are identical (with identical left-hand patterns the
        // pairs are then unordered)
        if (kind == CWC_RULE_PAIR) {
          bool rsym = true;
          for (int x = 0; x < S; ++x) {
            const int32_t* r1 = rrow(j, 1);
            const int32_t* r2 = rrow(j, 2);
            const int32_t* r3 = rrow(j, 3);
            const int32_t* r4 = rrow(j, 4);
            rsym = rsym && r1[x] == r3[x] && r2[x] == r4[x];
          }
          rec[CR_GRAND] = rsym ? 1 : 0;
        }
        nested_ext.emplace_back(j, std::vector<int32_t>(XR_WORDS, 0));
        int32_t* xr = nested_ext.back().second.data();
        ok = ok && put(xr, XR_ND3, XR_D3, lrow(j, 3), rrow(j, 3), false) &&
             put(xr, XR_ND4, XR_D4, lrow(j, 4), rrow(j, 4), false);
      }
      if (!ok) {
        delete m;
        return fail(CWC_ERR_UNSUPPORTED, "rule " + std::to_string(j) + ": more than 8 species change in one pattern");
      }
      for (int k = 0; k < rec[CR_ND0]; ++k) writes[j].push_back(key(0, ctx, rec[CR_D0 + k] & 0xffff));
      if (kind == CWC_RULE_PARENT_CHILD) {
        for (int k = 0; k < rec[CR_ND1]; ++k) writes[j].push_back(key(1, ch, rec[CR_D1 + k] & 0xffff));
        for (int k = 0; k < rec[CR_ND2]; ++k) writes[j].push_back(key(0, ch, rec[CR_D2 + k] & 0xffff));
      }
    }
    std::vector<int32_t> deps_all;
    auto general = [&](int kind) { return kind == CWC_RULE_FUSION || kind == CWC_RULE_NESTED || kind == CWC_RULE_PAIR; };
    for (int j = 0; j < M; ++j) {
      int32_t* rec = tb.data() + (size_t)j * CWC_RULE_WORDS;
      rec[CR_DEPOFF] = (int32_t)deps_all.size();
      uint32_t leafmask = 0, nodemask = 0;
      int cnt = 0;
      // rule i depends on rule j when j writes a location i reads, or when j
      // adds, removes or re-parents a compartment that can be a context of i.
      // FUSION and NESTED rules are recounted after every event, and after a
      // FUSION or NESTED event every rule is recounted.
      const int kj = d->kind[j], lj = d->ctx_label[j], cj = d->child_label[j];
      {
        for (int i = 0; i < M; ++i) {
          const int ki = d->kind[i], li = d->ctx_label[i], ci = d->child_label[i];
          const bool local_i = ki == CWC_RULE_LOCAL || ki == CWC_RULE_CREATE;
          bool hit = general(kj) || general(ki);
          for (long long w : writes[j])
            for (long long r : reads[i]) hit |= (w == r);
          if (kj == CWC_RULE_CREATE)   // a new compartment of label cj under one of label lj
            hit |= local_i ? li == cj : (ci == cj && li == lj);
          if (kj == CWC_RULE_DISSOLVE) {
            // any species of the parent content (label lj) may change
            for (long long r : reads[i]) hit |= (r / S) == (long long)lj;   // key(0, lj, *)
            // the dissolved compartment was a context; its children get a new parent
            hit |= local_i ? li == cj : (ci == cj || li == cj || li == lj);
          }
          if (!hit) continue;
          deps_all.push_back(i);
          ++cnt;
          const int l = i / m->B;
          leafmask |= 1u << l;
          nodemask |= (1u << (l >> 1)) | (1u << (16 + (l >> 2))) | (1u << (24 + (l >> 3))) |
                      (1u << (28 + (l >> 4))) | (1u << TREE_ROOT);
        }
      }
      rec[CR_DEPCNT] = cnt;
      rec[CR_LEAFMASK] = (int32_t)leafmask;
      rec[CR_NODEMASK] = (int32_t)nodemask;
    }
    for (auto& ne : nested_ext) {
      int32_t* rec = tb.data() + (size_t)ne.first * CWC_RULE_WORDS;
      const long long off = (long long)M * CWC_RULE_WORDS + (long long)deps_all.size();
      rec[CR_GRAND] = (rec[CR_GRAND] & 0xff) | (int32_t)(off << 8);
      deps_all.insert(deps_all.end(), ne.second.begin(), ne.second.end());
    }
    m->c_n_deps = (int)deps_all.size();   // the dependency lists, then the NESTED extensions
    tb.insert(tb.end(), deps_all.begin(), deps_all.end());
    if ((size_t)cwc_table_bytes_host(M, m->c_n_deps) + 32ull * (32 + TREE_NODES + M) * 8 > 220 * 1024) {
      delete m;
      return fail(CWC_ERR_UNSUPPORTED, "model too large for one block of 32 trajectories in shared memory");
    }
    e = cudaMalloc(&m->d_ctables, tb.size() * sizeof(int32_t));
    if (e != cudaSuccess) {
      delete m;
      return cuda_fail(e, "cudaMalloc(model tables)");
    }
    e = cudaMemcpy(m->d_ctables, tb.data(), tb.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(m->d_ctables);
      delete m;
      return cuda_fail(e, "cudaMemcpy(model tables)");
    }
    *out = m;
    return CWC_OK;
  }
  // ---- flat compilation ----
  for (int j = 0; j < M; ++j) {
    int order = 0;
    for (int s = 0; s < S; ++s) order += d->lhs[(size_t)j * 3 * S + s];
    if (order >= 3) m->checked_counts = 1;
  }
  std::vector<std::vector<int>> reac(M), delta(M);
  for (int j = 0; j < M; ++j) {
    const int32_t* lhs = d->lhs + (size_t)j * 3 * S;
    const int32_t* rhs = d->rhs + (size_t)j * 3 * S;
    for (int s = 0; s < S; ++s) {
      if (lhs[s] > 0) reac[j].push_back(s);
      if (rhs[s] != lhs[s]) delta[j].push_back(s);
    }
    if ((int)delta[j].size() > MAX_DELTA) {
      delete m;
      return fail(CWC_ERR_UNSUPPORTED, "rule " + std::to_string(j) + ": more than 8 species change");
    }
  }
  // dependents of j: rules with a reactant species whose count j changes
  std::vector<std::vector<int>> deps(M);
  std::vector<std::vector<int>> readers(S);
  for (int i = 0; i < M; ++i)
    for (int s : reac[i]) readers[s].push_back(i);
  for (int j = 0; j < M; ++j) {
    std::vector<char> mark(M, 0);
    for (int s : delta[j])
      for (int i : readers[s]) mark[i] = 1;
    for (int i = 0; i < M; ++i)
      if (mark[i]) deps[j].push_back(i);
  }
  int n_deps = 0;
  for (int j = 0; j < M; ++j) n_deps += (int)deps[j].size();
  m->n_deps = n_deps;
  std::vector<int32_t>& tb = m->h_tables;
  tb.assign((size_t)M * RULE_WORDS + n_deps, 0);
  int off = 0;
  for (int j = 0; j < M; ++j) {
    int32_t* rec = tb.data() + (size_t)j * RULE_WORDS;
    const int32_t* lhs = d->lhs + (size_t)j * 3 * S;
    const int32_t* rhs = d->rhs + (size_t)j * 3 * S;
    rec[R_NREAC] = (int32_t)reac[j].size();
    for (size_t a = 0; a < reac[j].size(); ++a) rec[R_REAC + a] = reac[j][a] | (lhs[reac[j][a]] << 16);
    rec[R_NDELTA] = (int32_t)delta[j].size();
    for (size_t a = 0; a < delta[j].size(); ++a) {
      const int s = delta[j][a];
      const int dv = rhs[s] - lhs[s];
      rec[R_DELTA + a] = (int32_t)((uint32_t)s | ((uint32_t)(dv & 0xffff) << 16));
    }
    rec[R_DEPOFF] = off;
    rec[R_DEPCNT] = (int32_t)deps[j].size();
    uint32_t leafmask = 0, nodemask = 0;
    for (int i : deps[j]) {
      tb[(size_t)M * RULE_WORDS + off++] = i;
      const int l = i / m->B;
      leafmask |= 1u << l;
      nodemask |= 1u << (l >> 1);
      nodemask |= 1u << (16 + (l >> 2));
      nodemask |= 1u << (24 + (l >> 3));
      nodemask |= 1u << (28 + (l >> 4));
      nodemask |= 1u << TREE_ROOT;
    }
    rec[R_LEAFMASK] = (int32_t)leafmask;
    rec[R_NODEMASK] = (int32_t)nodemask;
  }
  // reactant descriptors (used when every rule has order <= 2)
  for (int j = 0; j < M; ++j) {
    uint32_t kind = 0, s0 = 0, s1 = 0;
    const int32_t* lhs = d->lhs + (size_t)j * 3 * S;
    if (reac[j].size() == 1) {
      s0 = s1 = (uint32_t)reac[j][0];
      kind = lhs[s0] == 1 ? 1u : 2u;
    } else if (reac[j].size() == 2) {
      s0 = (uint32_t)reac[j][0];
      s1 = (uint32_t)reac[j][1];
      kind = 3u;
    }
    tb.push_back((int32_t)(kind | (s0 << 2) | (s1 << 16)));
  }
  // the logarithm's per-prefix tables (u64, low word first), 16-byte aligned
  {
    while (tb.size() % 4) tb.push_back(0);
    const LogConstants lct = make_log_constants();
    for (int i = 0; i < 64; ++i) {
      tb.push_back((int32_t)(uint32_t)lct.rj[i]);
      tb.push_back((int32_t)(uint32_t)(lct.rj[i] >> 32));
    }
    for (int i = 0; i < 64; ++i) {
      tb.push_back((int32_t)(uint32_t)lct.tj[i]);
      tb.push_back((int32_t)(uint32_t)(lct.tj[i] >> 32));
    }
  }
  // The warp rebuilds its lanes' dirty leaves together when a leaf holds more
  // than one rule and an event dirties three leaves or more on average over
  // the rules (or the leaves hold Michaelis-Menten divisions); measured +9 %
  // at 4.5 leaves (64 rules), -11 % at 2 (33 rules).
  {
    long long dirty = 0;
    for (int j = 0; j < M; ++j) dirty += __builtin_popcount((unsigned)tb[(size_t)j * RULE_WORDS + R_LEAFMASK]);
    bool law = false;
    for (int j = 0; j < M; ++j) law |= d->rate_law != nullptr && d->rate_law[j] != 0;
    m->pool = m->B > 1 && (law || dirty >= 3LL * M) ? 1 : 0;
  }
  // Michaelis-Menten tables (only when some rule has that law), after the
  // logarithm's tables (16-byte aligned): K_j as doubles [M] (0 = mass
  // action), then [M] int32 words substrate | (enzyme + 1) << 16 (0: none)
  bool any_mm = false;
  for (int j = 0; j < M; ++j) any_mm |= d->rate_law != nullptr && d->rate_law[j] != 0;
  if (any_mm) {
    m->mm_off = (int)tb.size();
    for (int j = 0; j < M; ++j) {
      const double K = d->rate_law[j] != 0 ? d->rate_par[j] : 0.0;
      uint64_t kb;
      std::memcpy(&kb, &K, 8);
      tb.push_back((int32_t)(uint32_t)kb);
      tb.push_back((int32_t)(uint32_t)(kb >> 32));
    }
    for (int j = 0; j < M; ++j) {
      uint32_t w = 0;
      if (d->rate_law[j] != 0) {
        const int sub = d->rate_law[j] - 1;
        w = (uint32_t)sub;
        for (int s : reac[j])
          if (s != sub) w |= (uint32_t)(s + 1) << 16;
      }
      tb.push_back((int32_t)w);
    }
  }
  // one trajectory's state must fit: 32 threads per block at least
  {
    FlatParams prm;
    std::memset(&prm, 0, sizeof(prm));
    prm.S = S;
    prm.M = M;
    prm.B = m->B;
    prm.smem_table_bytes = flat_table_bytes_host(M, n_deps);
    if (flat_smem_bytes(prm, 32, true) > 220 * 1024) {
      delete m;
      return fail(CWC_ERR_UNSUPPORTED, "model too large for one block of 32 trajectories in shared memory");
    }
  }
  e = cudaMalloc(&m->d_tables, tb.size() * sizeof(int32_t));
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "cudaMalloc(model tables)");
  }
  e = cudaMemcpy(m->d_tables, tb.data(), tb.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(m->d_tables);
    delete m;
    return cuda_fail(e, "cudaMemcpy(model tables)");
  }
  *out = m;
  return CWC_OK;
}

void cwc_model_destroy(cwc_model* m) {
  if (m == nullptr) return;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (auto it = g_tune_cache.begin(); it != g_tune_cache.end();)
      it = std::get<0>(it->first) == (const void*)m ? g_tune_cache.erase(it) : std::next(it);
  }
  if (m->d_tables) cudaFree(m->d_tables);
  if (m->d_ctables) cudaFree(m->d_ctables);
  delete m;
}

int32_t cwc_checkpoint_words(const cwc_model* m) {
  if (m == nullptr) return -1;
  return m->flat ? m->S + CKPT_HEADER_WORDS : CKPT_HEADER_WORDS + m->C * (3 + 2 * m->S);
}

int32_t cwc_model_num_observables(const cwc_model* m) {
  if (m == nullptr) return -1;
  return m->O;
}

cwc_status cwc_simulate_workspace_size(const cwc_model* m, const cwc_sim_args* a, size_t* bytes) {
  g_last_error.clear();
  if (bytes == nullptr) return fail(CWC_ERR_INVALID_ARG, "bytes must not be NULL");
  cwc_status st = check_sim_args(m, a);
  if (st != CWC_OK) return st;
  const cwc_sim_args b = resolve_auto(m, a);
  *bytes = ws_layout(m, &b, false, false).total;
  return CWC_OK;
}

cwc_status cwc_sensitivity_workspace_size(const cwc_model* m, const cwc_sim_args* a, const cwc_sens_args* s,
                                          size_t* bytes) {
  g_last_error.clear();
  if (bytes == nullptr || s == nullptr) return fail(CWC_ERR_INVALID_ARG, "sens and bytes must not be NULL");
  cwc_status st = check_sim_args(m, a);
  if (st != CWC_OK) return st;
  *bytes = ws_layout(m, a, true, s->partials != nullptr).total;
  return CWC_OK;
}

static cwc_status run_flat(const cwc_model* m, const cwc_sim_args* a, const cwc_sens_args* sens, cudaStream_t st) {
  const bool is_sens = sens != nullptr;
  const WsLayout w = ws_layout(m, a, is_sens, is_sens && sens->partials != nullptr);
  if (w.total > 0) {
    if (a->workspace == nullptr || a->workspace_bytes < w.total)
      return fail(CWC_ERR_WORKSPACE, "workspace of " + std::to_string(w.total) + " bytes required");
    if ((reinterpret_cast<uintptr_t>(a->workspace) & 255) != 0)
      return fail(CWC_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  }
  unsigned char* ws = static_cast<unsigned char*>(a->workspace);
  FlatParams prm = make_flat_params(m, a);
  const int O = m->S;
  cudaError_t e;
  if (w.need_header) {
    prm.ws = reinterpret_cast<WorkspaceHeader*>(ws + w.header);
    e = cudaMemsetAsync(prm.ws, 0, sizeof(WorkspaceHeader), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(workspace)");
  }
  if (!is_sens) {
    const cwc_status sst = states_ptr(a->states, st, &prm.states);
    if (sst != CWC_OK) return sst;
    unsigned long long* sums = reinterpret_cast<unsigned long long*>(a->sums);
    if (w.need_sums) sums = reinterpret_cast<unsigned long long*>(ws + w.sums);
    prm.sums = sums;
    if (sums != nullptr) {
      e = cudaMemsetAsync(sums, 0, (size_t)a->P * a->G * O * sizeof(long long), st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(sums)");
    }
    unsigned long long* sumsq = reinterpret_cast<unsigned long long*>(a->sumsq);
    if (w.need_sumsq) sumsq = reinterpret_cast<unsigned long long*>(ws + w.sumsq);
    prm.sumsq = sumsq;
    if (sumsq != nullptr) {
      e = cudaMemsetAsync(sumsq, 0, (size_t)a->P * a->G * O * 2 * sizeof(unsigned long long), st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(sumsq)");
    }
    prm.traj_status = a->traj_status;
    prm.traj_events = reinterpret_cast<long long*>(a->traj_events);
    prm.traj_hash = reinterpret_cast<unsigned long long*>(a->traj_hash);
    prm.traj_final_t = a->traj_final_t;
    prm.log_cap = a->log_cap;
    prm.log_rule = a->log_rule;
    prm.log_slot = a->log_slot;
    prm.log_t = a->log_t;
  } else {
    prm.means = sens->means;
    prm.grad_means = sens->grad_means;
    prm.partials = sens->partials != nullptr ? sens->partials : reinterpret_cast<double*>(ws + w.partials);
    prm.sens_acc = reinterpret_cast<double*>(ws + w.sens_acc);
    double* inv = reinterpret_cast<double*>(ws + w.inv_rates);
    e = launch_reciprocal(a->rates, inv, (long long)a->P * m->M, st);
    if (e != cudaSuccess) return cuda_fail(e, "reciprocal kernel launch");
    prm.inv_rates = inv;
  }
  const LogConstants lc = make_log_constants();
  const bool queue = queue_layout(a);
  int32_t* tail_list = nullptr;
  double* tail_est = nullptr;
  int32_t* tail_order = nullptr;
  if (w.need_tail) {
    // the thread kernel's checkpoints (the handed-over state), then the
    // warp kernel's list, predictions and order
    const size_t Q = (size_t)a->P * a->R;
    unsigned char* base = ws + w.tail;
    prm.ckpt = reinterpret_cast<int32_t*>(base);
    base += align256(Q * (size_t)(m->S + CKPT_HEADER_WORDS) * 4);
    tail_est = reinterpret_cast<double*>(base);
    tail_list = reinterpret_cast<int32_t*>(tail_est + Q);
    tail_order = tail_list + Q;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // default measured on the 256 x 256 uneven sweep with 16 lanes per handed-
    // over trajectory (4104 / 8192 / 16384 trajectories: 6.71 / 6.40 / 6.09 s;
    // the queue layout 7.91 s): 108 per SM
    prm.handoff = a->tail_threshold > 0 ? a->tail_threshold : 108LL * sms;
  }
  if (w.need_order) {
    double* est = reinterpret_cast<double*>(ws + w.order);
    int32_t* order = reinterpret_cast<int32_t*>(est + a->P);
    e = launch_flat_order(prm, est, order, st);
    if (e != cudaSuccess) return cuda_fail(e, "queue order kernels");
    prm.order = order;
  }
  const int T = pick_threads(m, a, prm, queue, is_sens);
  if (flat_smem_bytes(prm, T, is_sens) > 227 * 1024)
    return fail(CWC_ERR_INVALID_ARG, "block_threads too large for this model's shared-memory state");
  e = launch_flat(prm, lc, queue, is_sens, T, 0, st, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "flat SSA kernel launch");
  if (w.need_tail) {
    e = launch_flat_tail(prm, lc, tail_list, tail_est, tail_order, st);
    if (e != cudaSuccess) return cuda_fail(e, "tail kernels launch");
  }
  if (!is_sens && a->means != nullptr) {
    e = launch_means(prm.sums, a->means, (long long)a->P * a->G * O, a->R, st);
    if (e != cudaSuccess) return cuda_fail(e, "means kernel launch");
  }
  if (!is_sens && (a->variance != nullptr || a->ci90 != nullptr)) {
    e = launch_stats(prm.sums, prm.sumsq, a->variance, a->ci90, (long long)a->P * a->G * O, a->R, st);
    if (e != cudaSuccess) return cuda_fail(e, "statistics kernel launch");
  }
  if (is_sens) {
    e = launch_reduce_partials(prm.partials, sens->grad_rates, a->P, a->R, m->M, st);
    if (e != cudaSuccess) return cuda_fail(e, "reduce kernel launch");
  }
  return CWC_OK;
}

static cwc_status run_cwc(const cwc_model* m, const cwc_sim_args* a, const cwc_sens_args* sens, cudaStream_t st,
                          bool allow_narrow = true);

// Scratch of cwc_simulate_noalloc: one statically sized array per device that
// loads the library.  In host code its name is only a stand-in; the device
// address comes from cudaGetSymbolAddress, looked up once per device with
// that device current and cached here.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CWC_NOALLOC_SCRATCH_BYTES];
static std::mutex g_noalloc_mutex;
static void* g_noalloc_addr[256];

static cwc_status noalloc_scratch_address(int device, void** addr) {
  if (device < 0 || device >= 256) return fail(CWC_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_addr[device] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_noalloc_addr[device] = p;
  }
  *addr = g_noalloc_addr[device];
  return CWC_OK;
}

cwc_status cwc_simulate_noalloc(const cwc_model* m, const cwc_sim_args* a, void* stream) {
  g_last_error.clear();
  cwc_status st = check_sim_args(m, a);  // also checks that m's device is the current one
  if (st != CWC_OK) return st;
  const cwc_sim_args ra = resolve_auto(m, a);
  const WsLayout w = ws_layout(m, &ra, false, false, false);
  if (w.total > CWC_NOALLOC_SCRATCH_BYTES)
    return fail(CWC_ERR_INVALID_ARG, "this call needs " + std::to_string(w.total) +
                                         " bytes of scratch; cwc_simulate_noalloc holds " +
                                         std::to_string(CWC_NOALLOC_SCRATCH_BYTES) +
                                         " (request sums, or use cwc_simulate with a workspace)");
  void* scratch = nullptr;
  st = noalloc_scratch_address(m->device, &scratch);
  if (st != CWC_OK) return st;
  cwc_sim_args b = ra;
  b.workspace = scratch;
  b.workspace_bytes = CWC_NOALLOC_SCRATCH_BYTES;
  if (!m->flat) return run_cwc(m, &b, nullptr, static_cast<cudaStream_t>(stream), false);
  return run_flat(m, &b, nullptr, static_cast<cudaStream_t>(stream));
}

static cwc_status run_cwc(const cwc_model* m, const cwc_sim_args* a, const cwc_sens_args* sens, cudaStream_t st,
                          bool allow_narrow) {
  const bool is_sens = sens != nullptr;
  const WsLayout w = ws_layout(m, a, is_sens, is_sens && sens->partials != nullptr, allow_narrow);
  if (w.blocks < 1) return fail(CWC_ERR_CUDA, "could not size the compartmentalised launch");
  if (a->workspace == nullptr || a->workspace_bytes < w.total)
    return fail(CWC_ERR_WORKSPACE, "workspace of " + std::to_string(w.total) + " bytes required");
  if ((reinterpret_cast<uintptr_t>(a->workspace) & 255) != 0)
    return fail(CWC_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  unsigned char* ws = static_cast<unsigned char*>(a->workspace);
  CwcParams prm = cwc_shape_params(m, a, is_sens);
  prm.rules = m->d_ctables;
  prm.P = a->P;
  prm.R = a->R;
  prm.G = a->G;
  prm.Pi = a->Pi;
  prm.r_offset = a->replica_offset;
  prm.rates = a->rates;
  prm.init = a->init;
  prm.grid = a->grid;
  prm.key0 = (uint32_t)a->seed;
  prm.key1 = (uint32_t)(a->seed >> 32);
  prm.max_events = a->max_events;
  prm.deadline_ns = a->deadline_ns;
  prm.ckpt = is_sens ? nullptr : a->checkpoint;
  prm.resume = is_sens ? 0 : a->resume;
  if (!is_sens) {
    const cwc_status sst = states_ptr(a->states, st, &prm.states);
    if (sst != CWC_OK) return sst;
    prm.traj_status = a->traj_status;
    prm.traj_events = reinterpret_cast<long long*>(a->traj_events);
    prm.traj_hash = reinterpret_cast<unsigned long long*>(a->traj_hash);
    prm.traj_final_t = a->traj_final_t;
    prm.log_cap = a->log_cap;
    prm.log_rule = a->log_rule;
    prm.log_slot = a->log_slot;
    prm.log_t = a->log_t;
  } else {
    prm.means = sens->means;
    prm.grad_means = sens->grad_means;
    prm.partials = sens->partials != nullptr ? sens->partials : reinterpret_cast<double*>(ws + w.partials);
  }
  prm.slabs = reinterpret_cast<int32_t*>(ws + w.slabs);
  cudaError_t e;
  if (w.need_header) {
    prm.ws = reinterpret_cast<WorkspaceHeader*>(ws + w.header);
    e = cudaMemsetAsync(prm.ws, 0, sizeof(WorkspaceHeader), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(workspace)");
  }
  unsigned long long* sums = is_sens ? nullptr : reinterpret_cast<unsigned long long*>(a->sums);
  if (w.need_sums) sums = reinterpret_cast<unsigned long long*>(ws + w.sums);
  prm.sums = sums;
  if (sums != nullptr) {
    e = cudaMemsetAsync(sums, 0, (size_t)a->P * a->G * m->O * sizeof(long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(sums)");
  }
  unsigned long long* sumsq = is_sens ? nullptr : reinterpret_cast<unsigned long long*>(a->sumsq);
  if (w.need_sumsq) sumsq = reinterpret_cast<unsigned long long*>(ws + w.sumsq);
  prm.sumsq = sumsq;
  if (sumsq != nullptr) {
    e = cudaMemsetAsync(sumsq, 0, (size_t)a->P * a->G * m->O * 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(sumsq)");
  }
  const LogConstants lc = make_log_constants();
  const bool queue = chosen_layout(a) == CWC_LAYOUT_QUEUE;
  if (w.narrow) {
    // 16-bit terms first; then the 32-bit launch resumes the trajectories it
    // handed over (every other record carries its final status and is
    // skipped), adding to the same sums
    prm.narrow = 1;
    prm.ckpt = reinterpret_cast<int32_t*>(ws + w.narrow_ckpt);
    prm.resume = 0;
    e = launch_cwc(prm, lc, queue, w.lanes, w.T, w.blocks, st);
    if (e != cudaSuccess) return cuda_fail(e, "CWC SSA kernel launch (16-bit terms)");
    if (w.need_header) {
      e = cudaMemsetAsync(prm.ws, 0, sizeof(WorkspaceHeader), st);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(workspace)");
    }
    prm.narrow = 0;
    prm.resume = 1;
  }
  e = launch_cwc(prm, lc, queue, w.lanes, w.T, w.blocks, st);
  if (e != cudaSuccess) return cuda_fail(e, "CWC SSA kernel launch");
  if (is_sens) {
    e = launch_reduce_partials(prm.partials, sens->grad_rates, a->P, a->R, m->M, st);
    if (e != cudaSuccess) return cuda_fail(e, "reduce kernel launch");
    return CWC_OK;
  }
  if (a->means != nullptr) {
    e = launch_means(sums, a->means, (long long)a->P * a->G * m->O, a->R, st);
    if (e != cudaSuccess) return cuda_fail(e, "means kernel launch");
  }
  if (a->variance != nullptr || a->ci90 != nullptr) {
    e = launch_stats(sums, sumsq, a->variance, a->ci90, (long long)a->P * a->G * m->O, a->R, st);
    if (e != cudaSuccess) return cuda_fail(e, "statistics kernel launch");
  }
  return CWC_OK;
}

cwc_status cwc_simulate(const cwc_model* m, const cwc_sim_args* a, void* stream) {
  g_last_error.clear();
  cwc_status st = check_sim_args(m, a);
  if (st != CWC_OK) return st;
  const cwc_sim_args b = resolve_auto(m, a);
  if (!m->flat) return run_cwc(m, &b, nullptr, static_cast<cudaStream_t>(stream));
  return run_flat(m, &b, nullptr, static_cast<cudaStream_t>(stream));
}

cwc_status cwc_autotune(const cwc_model* m, const cwc_sim_args* a, int64_t tune_events, void* stream,
                        int32_t* best_layout, int32_t* best_threads, double* best_ms, int32_t* best_lanes) {
  g_last_error.clear();
  cwc_status st = check_sim_args(m, a);
  if (st != CWC_OK) return st;
  if (tune_events < 0) return fail(CWC_ERR_INVALID_ARG, "tune_events must be >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(CWC_ERR_CUDA, "cudaEventCreate");
  cwc_sim_args c = *a;
  c.states = nullptr;
  c.sums = nullptr;
  c.means = nullptr;
  c.sumsq = nullptr;
  c.variance = nullptr;
  c.ci90 = nullptr;
  c.traj_status = nullptr;
  c.traj_events = nullptr;
  c.traj_hash = nullptr;
  c.traj_final_t = nullptr;
  c.log_cap = 0;
  c.log_rule = nullptr;
  c.log_slot = nullptr;
  c.log_t = nullptr;
  c.checkpoint = nullptr;
  c.resume = 0;
  c.deadline_ns = 0;
  const int64_t cap = tune_events == 0 ? 2048 : tune_events;
  c.max_events = std::min<int64_t>(a->max_events, cap);
  float best = -1.0f;
  int bl = 0, bt = 0, bn = 1;
  for (int lanes : {1, 4, 8})
  for (int lay : {CWC_LAYOUT_STATIC, CWC_LAYOUT_QUEUE}) {
    if (m->flat && lanes != 1) continue;
    for (int T = 32; T <= 256; T += 32) {
      c.layout = lay;
      c.block_threads = T;
      c.lanes = lanes;
      if (m->flat) {
        FlatParams prm = make_flat_params(m, &c);
        if (flat_smem_bytes(prm, T, false) > 227 * 1024) continue;
      } else if ((size_t)cwc_table_bytes_host(m->M, m->c_n_deps) + (size_t)(T / lanes) * cwc_thread_bytes_host(m->M) >
                 227 * 1024) {
        continue;
      }
      const WsLayout w = ws_layout(m, &c, false, false);
      if (!m->flat && w.blocks < 1) continue;
      if (w.total > 0 && (c.workspace == nullptr || c.workspace_bytes < w.total)) continue;
      float ms_best = -1.0f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, s);
        st = m->flat ? run_flat(m, &c, nullptr, s) : run_cwc(m, &c, nullptr, s);
        cudaEventRecord(e1, s);
        if (st != CWC_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return fail(CWC_ERR_CUDA, "autotune candidate failed");
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep == 1) ms_best = ms;
      }
      if (st != CWC_OK) {
        st = CWC_OK;
        continue;
      }
      if (ms_best >= 0.0f && (best < 0.0f || ms_best < best)) {
        best = ms_best;
        bl = lay;
        bt = T;
        bn = lanes;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0.0f) return fail(CWC_ERR_INTERNAL, "no autotune candidate could run (workspace too small?)");
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[std::make_tuple((const void*)m, a->P, a->R, a->G, a->Pi)] = std::make_tuple(bl, bt, bn);
  }
  if (best_layout) *best_layout = bl;
  if (best_threads) *best_threads = bt;
  if (best_lanes) *best_lanes = bn;
  if (best_ms) *best_ms = best;
  g_last_error.clear();
  return CWC_OK;
}

cwc_status cwc_sensitivity(const cwc_model* m, const cwc_sim_args* a, const cwc_sens_args* s, void* stream) {
  g_last_error.clear();
  cwc_status st = check_sim_args(m, a);
  if (st != CWC_OK) return st;
  if (s == nullptr || s->means == nullptr || s->grad_means == nullptr || s->grad_rates == nullptr)
    return fail(CWC_ERR_INVALID_ARG, "means, grad_means and grad_rates must not be NULL");
  if (a->checkpoint != nullptr || a->resume != 0)
    return fail(CWC_ERR_INVALID_ARG, "sensitivities do not take checkpoints");
  if (!m->flat) return run_cwc(m, a, s, static_cast<cudaStream_t>(stream));
  return run_flat(m, a, s, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
