/*
 * cwc_oracle.c -- plain, sequential CPU oracle for Gillespie direct-method
 * simulation of restricted CWC rewrite systems (flat mass-action networks are
 * the one-compartment case), run over replicas x parameter-sweep points.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  It shares no code, header,
 * table or constant generator with the CUDA library, and the CUDA library
 * never loads it.
 *
 * It is deliberately slow and literal: every step re-matches every rule in
 * every compartment and rebuilds the whole propensity tree, in the order of
 * the simulation step of Sec. 5.1 (Fig. "CWC simulator pseudo-code": Match,
 * Resolve = Gillespie + stochastic choice of the context, Update, clock).
 *
 * Build (see build.py): gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math.
 * With contraction off, every floating-point expression below is evaluated
 * as separate IEEE-754 double operations rounded to nearest-even, in the
 * order written.
 *
 * Parity is pinned per function by the tests (tests/test_oracle_*.py):
 *   philox4x32_10   statistical tests on the CPU; cuRAND's Philox4_32_10 on
 *                   the GPU (library routine).
 *   u52             exhaustive boundary words, exactness.
 *   log_spec        < 0.55 ulp against 50-digit decimal logarithms; <= 1 ulp
 *                   against the C library log on 10^6 points + edges.
 *   tree_sum        error bound against an exactly rounded sum (math.fsum).
 *   select_rule     never picks a zero entry; frequencies vs a_j / a0.
 *   propensities    Sec. 2.2 worked example (rate 4k); brute-force counting
 *                   of distinct reactant tuples on small terms, and of
 *                   distinct occurrences of FUSION / PAIR / NESTED left-hand
 *                   sides (identified atoms and compartments) on random terms.
 *   context choice  chi-square laws where the chosen compartment changes the
 *                   outcome; exact recomputation of the integer draw.
 *   simulate        closed-form laws (birth-death Poisson / binomial mixture,
 *                   isomerisation binomial, depth-two transport binomial,
 *                   sibling transport as the Ehrenfest model),
 *                   chemical master equation via matrix exponential (incl.
 *                   fusion of empty compartments), conservation invariants.
 *   sensitivities   analytic birth-death gradient; central finite
 *                   differences with common random numbers.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Status codes of one trajectory.                                          */
/* ------------------------------------------------------------------------ */
enum {
  ST_OK = 0,             /* reached the end of the grid                     */
  ST_ABSORBED = 1,       /* total propensity became zero (not an error)     */
  ST_INT_OVERFLOW = 2,   /* a count would exceed INT32_MAX; event not applied */
  ST_PROP_OVERFLOW = 3,  /* an int64 combinatorial count overflowed, or a0 = inf */
  ST_CAPACITY = 4,       /* CREATE found no free compartment slot           */
  ST_EVENT_LIMIT = 5,    /* max_events events were applied                  */
  ST_BAD_INPUT = 6       /* rates, initial term or grid invalid             */
};

/* Rule kinds.  A rule's left-hand side is matched in the content of a
 * compartment of its label l (Sec. 2.1); with the compartment patterns it may
 * contain, the kinds are
 *   LOCAL         l: p X -> p' X
 *   PARENT_CHILD  l: p X (w x | q Y)^l' -> p' X (w' x | q' Y)^l'
 *   CREATE        l: p X -> p' X (w' | q')^l'
 *   DISSOLVE      l: p X (w x | q Y)^l' -> p' X x Y
 *   FUSION        l: p X (w1 x1 | q1 Y1)^l' (w2 x2 | q2 Y2)^l'
 *                      -> p' X (w' x1 x2 | q' Y1 Y2)^l'      (two compartments)
 *   NESTED        l: p X (w x | q Y (v z | u Z)^l'')^l'
 *                      -> p' X (w' x | q' Y (v' z | u' Z)^l'')^l'   (depth two)
 *   PAIR          l: p X (w1 x1 | q1 Y1)^l' (w2 x2 | q2 Y2)^l'
 *                      -> p' X (w1' x1 | q1' Y1)^l' (w2' x2 | q2' Y2)^l'
 *                                         (two compartments, both kept) */
enum { K_LOCAL = 0, K_PARENT_CHILD = 1, K_CREATE = 2, K_DISSOLVE = 3, K_FUSION = 4, K_NESTED = 5, K_PAIR = 6 };

/* Pattern rows of lhs / rhs ([M][ROWS][S]):
 *   0  the context's content (the parent's, for rules with a compartment)
 *   1  wrap of the (first) child      2  content of the (first) child
 *   3  FUSION, PAIR: wrap of the second child, NESTED: wrap of the grandchild
 *   4  FUSION, PAIR: content of the second child, NESTED: content of the grandchild
 * CREATE's rhs rows 1, 2 are the new compartment's wrap and content; FUSION's
 * rhs rows 1, 2 are added to the merged wrap and content. */
#define ROWS 5

/* Rate laws (Sec. 2.2: mass action, "but more flexible approaches are also
 * considered"): rate_law[j] = 0 for mass action, where h_j is the number of
 * reactant combinations; rate_law[j] = 1 + s for Michaelis-Menten kinetics
 * of substrate s with constant K_j = rate_par[j] > 0 (flat models, LOCAL
 * rules with one or two reactant species of multiplicity 1, the other one
 * the enzyme E):  h_j = RN(RN(n_E * n_s) / RN(K_j + n_s)), or
 * RN(n_s / RN(K_j + n_s)) without an enzyme, each an IEEE double operation
 * in this order.  Both arrays may be NULL (all mass action). */
typedef struct {
  int32_t S, L, C, M;
  const int32_t *kind, *ctx_label, *child_label, *grand_label;
  const int32_t *lhs; /* [M][ROWS][S] */
  const int32_t *rhs; /* [M][ROWS][S] */
  const int32_t *rate_law; /* [M] or NULL */
  const double *rate_par;  /* [M] or NULL */
} oracle_model;

/* Michaelis-Menten value of rule j at a flat term's counts x (see above). */
static double mm_value(const oracle_model* m, int j, const int32_t* x) {
  const int32_t* lhs = m->lhs + (size_t)j * ROWS * m->S;
  const int sub = m->rate_law[j] - 1;
  double num = (double)x[sub];
  for (int s = 0; s < m->S; s++)
    if (lhs[s] != 0 && s != sub) num = num * (double)x[s];   /* the enzyme, if any */
  const double den = m->rate_par[j] + (double)x[sub];
  return num / den;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications,    */
/* a key schedule bumped by two Weyl constants between rounds.               */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Draw for event n, purpose (0: tau and rule, 1: context), replica r, point p. */
static void draw(uint64_t seed, uint32_t n, uint32_t purpose, uint32_t r, uint32_t p,
                 uint32_t out[4]) {
  uint32_t ctr[4] = {n, purpose, r, p};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  oracle_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Uniform in (0,1): 52 random bits k, u = (k + 1/2) 2^-52.  Exact.          */
/* ------------------------------------------------------------------------ */
double oracle_u52(uint32_t wa, uint32_t wb) {
  uint64_t k = ((uint64_t)(wa >> 6) << 26) | (uint64_t)(wb >> 6);
  return ((double)k + 0.5) * 0x1p-52;
}

/* ------------------------------------------------------------------------ */
/* Natural logarithm of the time step, for u in [2^-53, 1), evaluated in     */
/* exact integer arithmetic with one final rounding to nearest (both sides   */
/* of the parity check compute the same integers).  Write u = F 2^(E-52),     */
/* F the 53-bit significand, f = F 2^-52 in [1, 2), E in [-53, -1].           */
/*  * near one (E = -1 and D = 2^53 - F < 2^46, so d = 1 - u < 2^-7):        */
/*    -ln u = -ln(1 - d) = d (1 + d/2 + d^2/3 + ... + d^8/9), the Mercator    */
/*    series (Abramowitz & Stegun 4.1.24), Horner in Q63 with d in Q64.       */
/*  * otherwise, with j the top 6 fraction bits of f and c_j = 1 + j/64:      */
/*    -ln u = -E ln2 - ln c_j - ln(1 + y),  y = f R_j - 1 in [0, 2^-6),       */
/*    R_j = ceil(2^69 / (64 + j)) (1/c_j in Q63, rounded up so that y >= 0),  */
/*    ln(1 + y) = y (1 - y/2 + y^2/3 - ... + y^10/11) by Horner in Q63, and   */
/*    the sum formed in Q120.                                                 */
/* Tables and constants (integers, the same definitions on both sides):     */
/*    C_n = floor(2^63 / n);  LN2_Q120 = sum_{k=1..120} floor(2^(120-k) / k)  */
/*    (the series ln 2 = sum 1/(k 2^k));  T_j = ln c_j in Q64 from the atanh  */
/*    series (A&S 4.1.27): s = floor(2^64 j / (128 + j)), z = floor(s^2/2^64),*/
/*    P = 1 + z/3 + ... + z^19/39 by Horner in Q63, T_j = floor(s P / 2^62). */
/* Every product is truncated (floor) to the width stated.  Error < 0.55 ulp.*/
/* ------------------------------------------------------------------------ */
typedef unsigned __int128 u128;

static uint64_t cq[40];    /* cq[n] = floor(2^63 / n) */
static uint64_t rj[64];    /* ceil(2^69 / (64 + j)) */
static uint64_t tj[64];    /* ln(1 + j/64) in Q64 */
static u128 ln2_q120;
static int log_ready = 0;

static uint64_t mulhi64(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a * (u128)b) >> 64); }

static void init_log(void) {
  if (log_ready) return;
  for (int n = 1; n < 40; n++) cq[n] = (uint64_t)((((u128)1) << 63) / (u128)n);
  u128 acc = 0;
  for (int k = 1; k <= 120; k++) acc += (((u128)1) << (120 - k)) / (u128)k;
  ln2_q120 = acc;
  for (int j = 0; j < 64; j++) {
    const u128 num = ((u128)1) << 69;
    rj[j] = (uint64_t)((num + (u128)(63 + j)) / (u128)(64 + j));
    const uint64_t sq = (uint64_t)((((u128)j) << 64) / (u128)(128 + j));
    const uint64_t zq = mulhi64(sq, sq);
    uint64_t p = cq[39];
    for (int k = 37; k >= 3; k -= 2) p = cq[k] + mulhi64(p, zq);
    p = (1ull << 63) + mulhi64(p, zq);
    tj[j] = (uint64_t)(((u128)sq * (u128)p) >> 62);
  }
  log_ready = 1;
}

/* x * 2^scale rounded to the nearest double (ties to even); x > 0, result normal */
static double round_u128(u128 x, int scale) {
  int lead = 127;
  while (!((x >> lead) & 1)) lead--;
  uint64_t mant;
  if (lead <= 52) {
    mant = (uint64_t)x << (52 - lead);
  } else {
    int sh = lead - 52;
    mant = (uint64_t)(x >> sh);
    u128 rem = x & ((((u128)1) << sh) - 1);
    u128 half = ((u128)1) << (sh - 1);
    if (rem > half || (rem == half && (mant & 1))) mant++;
    if (mant == (1ull << 53)) {
      mant >>= 1;
      lead++;
    }
  }
  return ldexp((double)mant, lead - 52 + scale);
}

double oracle_log_spec(double u) {
  init_log();
  uint64_t bits;
  memcpy(&bits, &u, 8);
  const int E = (int)((bits >> 52) & 0x7ff) - 1023;
  const uint64_t F = (bits & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
  if (E == -1 && (1ull << 53) - F < (1ull << 46)) {
    const uint64_t D = (1ull << 53) - F;
    const uint64_t dq = D << 11;                      /* d in Q64 */
    uint64_t q = cq[9];
    for (int n = 8; n >= 1; n--) q = cq[n] + mulhi64(q, dq);
    return -round_u128((u128)D * (u128)q, -116);      /* d q = D 2^-53 q 2^-63 */
  }
  const int j = (int)((F >> 46) & 63);
  const uint64_t X = F << 11;                         /* f in Q63 */
  const u128 fr = (u128)X * (u128)rj[j];             /* f R_j in Q126 */
  const uint64_t yq = (uint64_t)((fr >> 62) - (((u128)1) << 64));   /* y in Q64 */
  uint64_t p = cq[11];
  for (int k = 10; k >= 2; k--) p = cq[k] - mulhi64(p, yq);
  p = (1ull << 63) - mulhi64(p, yq);                  /* ln(1+y)/y in Q63 */
  const u128 l1 = ((u128)yq * (u128)p) >> 7;          /* ln(1+y) in Q120 */
  const u128 y = (u128)(uint64_t)(-E) * ln2_q120 - (((u128)tj[j]) << 56) - l1;
  return -round_u128(y, -120);
}

/* ------------------------------------------------------------------------ */
/* 32-lane blocked tree over a[0..M-1]: block size B = ceil(M/32); leaf l is */
/* the left-to-right sum of a[lB .. min((l+1)B, M)-1] (empty: +0); then five */
/* levels of pairwise sums, node(k,i) = node(k-1,2i) + node(k-1,2i+1).       */
/* nodes[0..31] = leaves, [32..47] level 1, [48..55] level 2, [56..59]       */
/* level 3, [60..61] level 4, [62] root.                                      */
/* ------------------------------------------------------------------------ */
static const int LEVEL_BASE[6] = {0, 32, 48, 56, 60, 62};

static void build_tree(const double* a, int M, double nodes[63]) {
  int B = (M + 31) / 32;
  for (int l = 0; l < 32; l++) {
    double s = 0.0;
    for (int j = l * B; j < (l + 1) * B && j < M; j++) s = s + a[j];
    nodes[l] = s;
  }
  for (int k = 1; k <= 5; k++) {
    int width = 32 >> k;
    for (int i = 0; i < width; i++)
      nodes[LEVEL_BASE[k] + i] = nodes[LEVEL_BASE[k - 1] + 2 * i] + nodes[LEVEL_BASE[k - 1] + 2 * i + 1];
  }
}

double oracle_tree_sum(const double* a, int32_t M) {
  double nodes[63];
  build_tree(a, M, nodes);
  return nodes[62];
}

/* Guarded descent: at a node go left if x < S_left or S_right == 0, else    */
/* x -= S_left and go right; in the leaf pick the first j whose running sum  */
/* exceeds x, else the last positive entry.  Never returns a zero entry.     */
int32_t oracle_select(const double* a, int32_t M, double x) {
  double nodes[63];
  build_tree(a, M, nodes);
  int B = (M + 31) / 32;
  int i = 0; /* index within the level */
  for (int k = 5; k >= 1; k--) {
    double SL = nodes[LEVEL_BASE[k - 1] + 2 * i];
    double SR = nodes[LEVEL_BASE[k - 1] + 2 * i + 1];
    if (x < SL || SR == 0.0) {
      i = 2 * i;
    } else {
      x = x - SL;
      i = 2 * i + 1;
    }
  }
  double s = 0.0;
  int last = -1;
  for (int j = i * B; j < (i + 1) * B && j < M; j++) {
    if (a[j] > 0.0) {
      last = j;
      s = s + a[j];
      if (x < s) return j;
    }
  }
  return last;
}

/* ------------------------------------------------------------------------ */
/* Terms: per trajectory, C compartment slots.                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t S, C;
  int32_t* alive;   /* [C] */
  int32_t* label;   /* [C] */
  int32_t* parent;  /* [C] */
  int32_t* wrap;    /* [C][S] */
  int32_t* content; /* [C][S] */
} term_t;

/* binomial(n, k) for k in {0,1,2}, n >= 0; the Match_Populations count. */
static int binom(int64_t n, int32_t k, int64_t* out) {
  if (k == 0) { *out = 1; return 0; }
  if (n < k) { *out = 0; return 0; }
  if (k == 1) { *out = n; return 0; }
  /* k == 2: n (n-1) / 2, exact in int64 for n < 2^31 */
  *out = n * (n - 1) / 2;
  return 0;
}

/* product of binomials of one pattern over one multiset; -1 on int64 overflow */
static int pattern_count(const int32_t* pattern, const int32_t* multiset, int32_t S, int64_t* acc) {
  for (int x = 0; x < S; x++) {
    if (pattern[x] == 0) continue;
    int64_t b;
    binom(multiset[x], pattern[x], &b);
    int64_t prod;
    if (__builtin_mul_overflow(*acc, b, &prod)) return -1;
    *acc = prod;
  }
  return 0;
}

/* Is slot c a context of rule j?  LOCAL/CREATE: slot of the rule's label.    */
/* PARENT_CHILD/DISSOLVE: a child slot of label child_label whose parent has  */
/* the rule's label.                                                          */
/* NESTED: a grandchild slot of label grand_label whose parent has label     */
/* child_label and whose grandparent has the rule's label.  FUSION's and     */
/* PAIR's contexts are pairs of slots (is_pair below), never single slots.   */
static int is_context(const oracle_model* m, const term_t* t, int j, int c) {
  if (!t->alive[c]) return 0;
  int kind = m->kind[j];
  if (kind == K_LOCAL || kind == K_CREATE) return t->label[c] == m->ctx_label[j];
  if (kind == K_FUSION || kind == K_PAIR) return 0;
  if (c == 0) return 0;
  int q = t->parent[c];
  if (kind == K_NESTED) {
    if (t->label[c] != m->grand_label[j] || q == 0) return 0;
    return t->label[q] == m->child_label[j] && t->label[t->parent[q]] == m->ctx_label[j];
  }
  return t->label[c] == m->child_label[j] && t->label[q] == m->ctx_label[j];
}

/* FUSION: are the two compartment patterns identical?  Then the occurrences */
/* (d1, d2) and (d2, d1) are the same subterm and only d1 < d2 counts (the    */
/* merged result is the same either way).  PAIR: the two compartments keep   */
/* their own right-hand sides, so (d1, d2) and (d2, d1) are the same rewrite  */
/* only when the right-hand patterns are identical too.                       */
static int pair_symmetric(const oracle_model* m, int j) {
  const int S = m->S;
  const int32_t* lhs = m->lhs + (size_t)j * ROWS * S;
  const int32_t* rhs = m->rhs + (size_t)j * ROWS * S;
  for (int x = 0; x < S; x++)
    if (lhs[S + x] != lhs[3 * S + x] || lhs[2 * S + x] != lhs[4 * S + x]) return 0;
  if (m->kind[j] == K_PAIR)
    for (int x = 0; x < S; x++)
      if (rhs[S + x] != rhs[3 * S + x] || rhs[2 * S + x] != rhs[4 * S + x]) return 0;
  return 1;
}

/* Is the ordered pair (d1, d2) an occurrence context of FUSION / PAIR rule j: two */
/* distinct alive children of label child_label under the same parent, whose */
/* label is the rule's?                                                        */
static int is_pair(const oracle_model* m, const term_t* t, int j, int d1, int d2) {
  if (d1 == d2 || d1 == 0 || d2 == 0 || !t->alive[d1] || !t->alive[d2]) return 0;
  if (t->label[d1] != m->child_label[j] || t->label[d2] != m->child_label[j]) return 0;
  if (t->parent[d1] != t->parent[d2]) return 0;
  if (t->label[t->parent[d1]] != m->ctx_label[j]) return 0;
  if (d1 > d2 && pair_symmetric(m, j)) return 0;
  return 1;
}

/* Match(rule, term, context): number of distinct reactant combinations of   */
/* rule j at context c (Sec. 2.2).  -1 on overflow.                           */
static int match_count(const oracle_model* m, const term_t* t, int j, int c, int64_t* h) {
  const int32_t S = m->S;
  const int32_t* lhs = m->lhs + (size_t)j * ROWS * S;
  int kind = m->kind[j];
  int64_t acc = 1;
  if (kind == K_LOCAL || kind == K_CREATE) {
    if (pattern_count(lhs, t->content + (size_t)c * S, S, &acc)) return -1;
  } else if (kind == K_NESTED) {
    /* c is the grandchild; rows: grandparent content, child wrap and content, */
    /* grandchild wrap and content                                            */
    int q = t->parent[c], a = t->parent[q];
    if (pattern_count(lhs, t->content + (size_t)a * S, S, &acc)) return -1;
    if (pattern_count(lhs + S, t->wrap + (size_t)q * S, S, &acc)) return -1;
    if (pattern_count(lhs + 2 * S, t->content + (size_t)q * S, S, &acc)) return -1;
    if (pattern_count(lhs + 3 * S, t->wrap + (size_t)c * S, S, &acc)) return -1;
    if (pattern_count(lhs + 4 * S, t->content + (size_t)c * S, S, &acc)) return -1;
  } else {
    int q = t->parent[c];
    if (pattern_count(lhs, t->content + (size_t)q * S, S, &acc)) return -1;
    if (pattern_count(lhs + S, t->wrap + (size_t)c * S, S, &acc)) return -1;
    if (pattern_count(lhs + 2 * S, t->content + (size_t)c * S, S, &acc)) return -1;
  }
  *h = acc;
  return 0;
}

/* FUSION, PAIR: occurrences at the pair (d1, d2): parent content x first child's */
/* wrap and content x second child's wrap and content.                        */
static int pair_count(const oracle_model* m, const term_t* t, int j, int d1, int d2, int64_t* h) {
  const int32_t S = m->S;
  const int32_t* lhs = m->lhs + (size_t)j * ROWS * S;
  int64_t acc = 1;
  int q = t->parent[d1];
  if (pattern_count(lhs, t->content + (size_t)q * S, S, &acc)) return -1;
  if (pattern_count(lhs + S, t->wrap + (size_t)d1 * S, S, &acc)) return -1;
  if (pattern_count(lhs + 2 * S, t->content + (size_t)d1 * S, S, &acc)) return -1;
  if (pattern_count(lhs + 3 * S, t->wrap + (size_t)d2 * S, S, &acc)) return -1;
  if (pattern_count(lhs + 4 * S, t->content + (size_t)d2 * S, S, &acc)) return -1;
  *h = acc;
  return 0;
}

/* H_j = sum over contexts of the combinatorial counts (int64, -1 overflow). */
static int rule_total(const oracle_model* m, const term_t* t, int j, int64_t* H) {
  int64_t total = 0;
  if (m->kind[j] == K_FUSION || m->kind[j] == K_PAIR) {
    for (int d1 = 0; d1 < t->C; d1++)
      for (int d2 = 0; d2 < t->C; d2++) {
        if (!is_pair(m, t, j, d1, d2)) continue;
        int64_t h, s;
        if (pair_count(m, t, j, d1, d2, &h)) return -1;
        if (__builtin_add_overflow(total, h, &s)) return -1;
        total = s;
      }
    *H = total;
    return 0;
  }
  for (int c = 0; c < t->C; c++) {
    if (!is_context(m, t, j, c)) continue;
    int64_t h;
    if (match_count(m, t, j, c, &h)) return -1;
    int64_t s;
    if (__builtin_add_overflow(total, h, &s)) return -1;
    total = s;
  }
  *H = total;
  return 0;
}

/* Observables: flat models give the root content; otherwise content totals  */
/* per label [L][S], wrap totals per label 1..L-1 [L-1][S], alive count per  */
/* label [L].  Totals are summed in int64 and saturate at INT32_MAX.         */
static int num_obs(const oracle_model* m) {
  if (m->L == 1 && m->C == 1) return m->S;
  return m->L * m->S + (m->L - 1) * m->S + m->L;
}

static void observe(const oracle_model* m, const term_t* t, int32_t* out) {
  const int S = m->S, L = m->L;
  if (L == 1 && m->C == 1) {
    for (int x = 0; x < S; x++) out[x] = t->content[x];
    return;
  }
  int O = num_obs(m);
  int64_t tot[4096];
  int64_t* acc = O <= 4096 ? tot : malloc(sizeof(int64_t) * O);
  for (int o = 0; o < O; o++) acc[o] = 0;
  for (int c = 0; c < t->C; c++) {
    if (!t->alive[c]) continue;
    int l = t->label[c];
    for (int x = 0; x < S; x++) acc[l * S + x] += t->content[(size_t)c * S + x];
    if (l > 0)
      for (int x = 0; x < S; x++) acc[L * S + (l - 1) * S + x] += t->wrap[(size_t)c * S + x];
    acc[L * S + (L - 1) * S + l] += 1;
  }
  for (int o = 0; o < O; o++) out[o] = acc[o] > 2147483647LL ? 2147483647 : (int32_t)acc[o];
  if (acc != tot) free(acc);
}

/* Check that a new value fits int32. */
static int fits(int64_t v) { return v >= 0 && v <= 2147483647LL; }

/* Update step: delete P sigma and add O sigma at the chosen context.        */
/* Returns ST_OK, ST_CAPACITY or ST_INT_OVERFLOW (then nothing changed).     */
static int apply_rule(const oracle_model* m, term_t* t, int j, int c) {
  const int S = m->S;
  const int32_t* lhs = m->lhs + (size_t)j * ROWS * S;
  const int32_t* rhs = m->rhs + (size_t)j * ROWS * S;
  int kind = m->kind[j];
  if (kind == K_NESTED) {
    /* c is the grandchild: rewrite the five matched multisets in place */
    int q = t->parent[c], a = t->parent[q];
    int32_t* ms[5] = {t->content + (size_t)a * S, t->wrap + (size_t)q * S, t->content + (size_t)q * S,
                      t->wrap + (size_t)c * S, t->content + (size_t)c * S};
    for (int row = 0; row < 5; row++)
      for (int s = 0; s < S; s++)
        if (!fits((int64_t)ms[row][s] + rhs[row * S + s] - lhs[row * S + s])) return ST_INT_OVERFLOW;
    for (int row = 0; row < 5; row++)
      for (int s = 0; s < S; s++) ms[row][s] = ms[row][s] + rhs[row * S + s] - lhs[row * S + s];
    return ST_OK;
  }
  if (kind == K_PAIR) {
    /* c encodes the pair (d1, d2): the parent content and both compartments' */
    /* wraps and contents are rewritten in place                              */
    int d1 = c & 0xffff, d2 = c >> 16, q = t->parent[d1];
    int32_t* ms[5] = {t->content + (size_t)q * S, t->wrap + (size_t)d1 * S, t->content + (size_t)d1 * S,
                      t->wrap + (size_t)d2 * S, t->content + (size_t)d2 * S};
    for (int row = 0; row < 5; row++)
      for (int s = 0; s < S; s++)
        if (!fits((int64_t)ms[row][s] + rhs[row * S + s] - lhs[row * S + s])) return ST_INT_OVERFLOW;
    for (int row = 0; row < 5; row++)
      for (int s = 0; s < S; s++) ms[row][s] = ms[row][s] + rhs[row * S + s] - lhs[row * S + s];
    return ST_OK;
  }
  if (kind == K_FUSION) {
    /* c encodes the pair (d1, d2); the merged compartment keeps the lower   */
    /* slot, the higher one is freed and its children move to the survivor. */
    int d1 = c & 0xffff, d2 = c >> 16;
    int q = t->parent[d1];
    int keep = d1 < d2 ? d1 : d2, gone = d1 < d2 ? d2 : d1;
    int32_t* xp = t->content + (size_t)q * S;
    const int32_t *w1 = t->wrap + (size_t)d1 * S, *x1 = t->content + (size_t)d1 * S;
    const int32_t *w2 = t->wrap + (size_t)d2 * S, *x2 = t->content + (size_t)d2 * S;
    for (int s = 0; s < S; s++) {
      if (!fits((int64_t)xp[s] + rhs[s] - lhs[s])) return ST_INT_OVERFLOW;
      if (!fits((int64_t)w1[s] - lhs[S + s] + (int64_t)w2[s] - lhs[3 * S + s] + rhs[S + s])) return ST_INT_OVERFLOW;
      if (!fits((int64_t)x1[s] - lhs[2 * S + s] + (int64_t)x2[s] - lhs[4 * S + s] + rhs[2 * S + s]))
        return ST_INT_OVERFLOW;
    }
    for (int s = 0; s < S; s++) {
      int32_t wm = w1[s] - lhs[S + s] + w2[s] - lhs[3 * S + s] + rhs[S + s];
      int32_t xm = x1[s] - lhs[2 * S + s] + x2[s] - lhs[4 * S + s] + rhs[2 * S + s];
      xp[s] = xp[s] + rhs[s] - lhs[s];
      t->wrap[(size_t)keep * S + s] = wm;
      t->content[(size_t)keep * S + s] = xm;
      t->wrap[(size_t)gone * S + s] = 0;
      t->content[(size_t)gone * S + s] = 0;
    }
    for (int d = 0; d < t->C; d++)
      if (t->alive[d] && t->parent[d] == gone) t->parent[d] = keep;
    t->alive[gone] = 0;
    t->label[gone] = 0;
    t->parent[gone] = -1;
    return ST_OK;
  }
  if (kind == K_LOCAL) {
    int32_t* x = t->content + (size_t)c * S;
    for (int s = 0; s < S; s++)
      if (!fits((int64_t)x[s] + rhs[s] - lhs[s])) return ST_INT_OVERFLOW;
    for (int s = 0; s < S; s++) x[s] = x[s] + rhs[s] - lhs[s];
    return ST_OK;
  }
  if (kind == K_PARENT_CHILD) {
    int q = t->parent[c];
    int32_t* xp = t->content + (size_t)q * S;
    int32_t* w = t->wrap + (size_t)c * S;
    int32_t* xc = t->content + (size_t)c * S;
    for (int s = 0; s < S; s++) {
      if (!fits((int64_t)xp[s] + rhs[s] - lhs[s])) return ST_INT_OVERFLOW;
      if (!fits((int64_t)w[s] + rhs[S + s] - lhs[S + s])) return ST_INT_OVERFLOW;
      if (!fits((int64_t)xc[s] + rhs[2 * S + s] - lhs[2 * S + s])) return ST_INT_OVERFLOW;
    }
    for (int s = 0; s < S; s++) {
      xp[s] = xp[s] + rhs[s] - lhs[s];
      w[s] = w[s] + rhs[S + s] - lhs[S + s];
      xc[s] = xc[s] + rhs[2 * S + s] - lhs[2 * S + s];
    }
    return ST_OK;
  }
  if (kind == K_CREATE) {
    int e = -1;
    for (int d = 1; d < t->C; d++)
      if (!t->alive[d]) { e = d; break; }
    if (e < 0) return ST_CAPACITY;
    int32_t* x = t->content + (size_t)c * S;
    for (int s = 0; s < S; s++)
      if (!fits((int64_t)x[s] + rhs[s] - lhs[s])) return ST_INT_OVERFLOW;
    for (int s = 0; s < S; s++) x[s] = x[s] + rhs[s] - lhs[s];
    t->alive[e] = 1;
    t->label[e] = m->child_label[j];
    t->parent[e] = c;
    for (int s = 0; s < S; s++) {
      t->wrap[(size_t)e * S + s] = rhs[S + s];
      t->content[(size_t)e * S + s] = rhs[2 * S + s];
    }
    return ST_OK;
  }
  /* K_DISSOLVE */
  {
    int q = t->parent[c];
    int32_t* xp = t->content + (size_t)q * S;
    int32_t* w = t->wrap + (size_t)c * S;
    int32_t* xc = t->content + (size_t)c * S;
    for (int s = 0; s < S; s++) {
      int64_t v = (int64_t)xp[s] + rhs[s] - lhs[s] + ((int64_t)w[s] - lhs[S + s]) +
                  ((int64_t)xc[s] - lhs[2 * S + s]);
      if (!fits(v)) return ST_INT_OVERFLOW;
    }
    for (int s = 0; s < S; s++)
      xp[s] = xp[s] + rhs[s] - lhs[s] + (w[s] - lhs[S + s]) + (xc[s] - lhs[2 * S + s]);
    for (int d = 0; d < t->C; d++)
      if (t->alive[d] && d != c && t->parent[d] == c) t->parent[d] = q;
    t->alive[c] = 0;
    t->label[c] = 0;
    t->parent[c] = -1;
    for (int s = 0; s < S; s++) {
      w[s] = 0;
      xc[s] = 0;
    }
    return ST_OK;
  }
}

/* FNV-1a 64-bit over the little-endian bytes of (uint32 rule, uint32 slot). */
static uint64_t fnv_event(uint64_t h, uint32_t rule, uint32_t slot) {
  uint8_t bytes[8];
  for (int i = 0; i < 4; i++) bytes[i] = (uint8_t)(rule >> (8 * i));
  for (int i = 0; i < 4; i++) bytes[4 + i] = (uint8_t)(slot >> (8 * i));
  for (int i = 0; i < 8; i++) {
    h ^= bytes[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

/* Load the initial term for sweep point p; returns 0 if valid.              */
static int load_init(const oracle_model* m, const int32_t* init, int p, int Pi, term_t* t) {
  const int S = m->S, C = m->C;
  int ip = Pi == 1 ? 0 : p;
  for (int c = 0; c < C; c++) {
    t->alive[c] = 0;
    t->label[c] = 0;
    t->parent[c] = -1;
  }
  memset(t->wrap, 0, sizeof(int32_t) * (size_t)C * S);
  memset(t->content, 0, sizeof(int32_t) * (size_t)C * S);
  if (m->L == 1 && C == 1) {
    const int32_t* x = init + (size_t)ip * S;
    t->alive[0] = 1;
    for (int s = 0; s < S; s++) {
      if (x[s] < 0) return -1;
      t->content[s] = x[s];
    }
    return 0;
  }
  const int W = 3 + 2 * S;
  const int32_t* img = init + (size_t)ip * C * W;
  for (int c = 0; c < C; c++) {
    const int32_t* row = img + (size_t)c * W;
    if (row[0] != 0 && row[0] != 1) return -1;
    t->alive[c] = row[0];
    if (!row[0]) continue;
    t->label[c] = row[1];
    t->parent[c] = row[2];
    for (int s = 0; s < S; s++) {
      t->wrap[(size_t)c * S + s] = row[3 + s];
      t->content[(size_t)c * S + s] = row[3 + S + s];
      if (row[3 + s] < 0 || row[3 + S + s] < 0) return -1;
    }
  }
  /* the root: slot 0, alive, label 0, no parent, empty wrap */
  if (!t->alive[0] || t->label[0] != 0 || t->parent[0] != -1) return -1;
  for (int s = 0; s < S; s++)
    if (t->wrap[s] != 0) return -1;
  for (int c = 1; c < C; c++) {
    if (!t->alive[c]) continue;
    if (t->label[c] < 1 || t->label[c] >= m->L) return -1;
    /* the parent chain must reach the root through alive slots */
    int q = c, steps = 0;
    while (q != 0) {
      q = t->parent[q];
      if (q < 0 || q >= C || !t->alive[q] || ++steps > C) return -1;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One trajectory.  The score part (partials != NULL) follows the same path  */
/* and accumulates, per grid point g, c(g) * S_j(g) with                      */
/*   c(g)   = sum_o grad_means[g][o] * (X_o(g) - means[g][o])                */
/*   S_j(g) = N_j(g) / k_j - I_j(g),  I_j(g) = int_0^{g} H_j(X(s)) ds        */
/* (the likelihood-ratio score of a CTMC path, a_j = k_j H_j).               */
/* ------------------------------------------------------------------------ */
typedef struct {
  const oracle_model* m;
  const double* k;
  const double* grid;
  int G, O, M;
  int32_t* states;        /* [G][O] or NULL */
  const double* means;    /* [G][O] or NULL */
  const double* gmeans;   /* [G][O] or NULL */
  double* partial;        /* [M] or NULL */
  int64_t* N;             /* [M] */
  double* I;              /* [M] */
  int64_t* H;             /* [M] combinatorial counts (mass action) */
  double* Hs;             /* [M] h_j as a double: (double)H_j, or the rate-law value */
  int32_t* obs;           /* [O] */
} traj_ctx;

static void record(traj_ctx* x, const term_t* t, int g, double now) {
  observe(x->m, t, x->obs);
  if (x->states) memcpy(x->states + (size_t)g * x->O, x->obs, sizeof(int32_t) * x->O);
  if (x->partial) {
    double cg = 0.0;
    for (int o = 0; o < x->O; o++)
      cg = cg + x->gmeans[(size_t)g * x->O + o] * ((double)x->obs[o] - x->means[(size_t)g * x->O + o]);
    double dt = x->grid[g] - now;
    for (int j = 0; j < x->M; j++) {
      double Ig = x->I[j] + x->Hs[j] * dt;
      double Sj = (double)x->N[j] / x->k[j] - Ig;
      x->partial[j] = x->partial[j] + cg * Sj;
    }
  }
}

static int valid_grid(const double* grid, int G) {
  if (G < 1) return 0;
  if (!(grid[0] >= 0.0) || !isfinite(grid[0])) return 0;
  for (int g = 1; g < G; g++)
    if (!(grid[g] > grid[g - 1]) || !isfinite(grid[g])) return 0;
  return 1;
}

int32_t oracle_num_observables(const oracle_model* m) { return num_obs(m); }

/*
 * Simulate trajectories q in [q_begin, q_end), q = p*R + r.
 * Output arrays are indexed by (q - q_begin); any of them may be NULL.
 *   states   [nq][G][O] int32     status [nq] int32    events [nq] int64
 *   hash     [nq] uint64          final_t [nq] double
 *   log_*    [nq][log_cap]: rule, slot and time of the first log_cap events
 *   means/grad_means [P][G][O], partials [nq][M]: score accumulation
 * Returns 0, or -1 if the model is malformed.
 */
int oracle_simulate(const oracle_model* m, const double* rates, int32_t P, int32_t R,
                    const int32_t* init, int32_t Pi, const double* grid, int32_t G,
                    uint64_t seed, int64_t max_events, int64_t q_begin, int64_t q_end,
                    int32_t* states, int32_t* status, int64_t* events, uint64_t* hash,
                    double* final_t, int32_t log_cap, int32_t* log_rule, int32_t* log_slot,
                    double* log_t, const double* means, const double* grad_means,
                    double* partials) {
  const int S = m->S, C = m->C, M = m->M, O = num_obs(m);
  if (S < 1 || C < 1 || M < 1 || m->L < 1) return -1;
  for (int j = 0; j < M; j++) {
    if (m->kind[j] < 0 || m->kind[j] > 6) return -1;
    if (m->rate_law != NULL && m->rate_law[j] != 0) {
      /* Michaelis-Menten: flat models, LOCAL, one or two reactant species of
         multiplicity 1 among which the substrate, K > 0 finite */
      const int sub = m->rate_law[j] - 1;
      const int32_t* lhs = m->lhs + (size_t)j * ROWS * m->S;
      int nreac = 0, bad = 0;
      for (int r = 0; r < ROWS; r++)
        for (int x = 0; x < m->S; x++)
          if (lhs[r * m->S + x] != 0) {
            nreac++;
            if (r != 0 || lhs[x] != 1) bad = 1;
          }
      if (m->L != 1 || m->C != 1 || m->kind[j] != K_LOCAL || sub < 0 || sub >= m->S || lhs[sub] != 1 ||
          nreac < 1 || nreac > 2 || bad || m->rate_par == NULL || !(m->rate_par[j] > 0.0) || !isfinite(m->rate_par[j]))
        return -1;
    }
    if (m->ctx_label[j] < 0 || m->ctx_label[j] >= m->L) return -1;
    if (m->kind[j] != K_LOCAL && (m->child_label[j] < 1 || m->child_label[j] >= m->L)) return -1;
    if (m->kind[j] == K_NESTED && (m->grand_label == NULL || m->grand_label[j] < 1 || m->grand_label[j] >= m->L))
      return -1;
  }
  term_t t;
  t.S = S;
  t.C = C;
  t.alive = malloc(sizeof(int32_t) * C);
  t.label = malloc(sizeof(int32_t) * C);
  t.parent = malloc(sizeof(int32_t) * C);
  t.wrap = malloc(sizeof(int32_t) * (size_t)C * S);
  t.content = malloc(sizeof(int32_t) * (size_t)C * S);
  double* a = malloc(sizeof(double) * M);
  traj_ctx x;
  x.m = m;
  x.grid = grid;
  x.G = G;
  x.O = O;
  x.M = M;
  x.N = malloc(sizeof(int64_t) * M);
  x.I = malloc(sizeof(double) * M);
  x.H = malloc(sizeof(int64_t) * M);
  x.Hs = malloc(sizeof(double) * M);
  x.obs = malloc(sizeof(int32_t) * O);
  const double T = grid[G - 1];
  const int grid_ok = valid_grid(grid, G);

  for (int64_t q = q_begin; q < q_end; q++) {
    const int64_t lq = q - q_begin;
    const int p = (int)(q / R), r = (int)(q % R);
    x.k = rates + (size_t)p * M;
    x.states = states ? states + (size_t)lq * G * O : NULL;
    x.means = means ? means + (size_t)p * G * O : NULL;
    x.gmeans = grad_means ? grad_means + (size_t)p * G * O : NULL;
    x.partial = partials ? partials + (size_t)lq * M : NULL;
    for (int j = 0; j < M; j++) {
      x.N[j] = 0;
      x.I[j] = 0.0;
      x.H[j] = 0;
      x.Hs[j] = 0.0;
      if (x.partial) x.partial[j] = 0.0;
    }
    double tnow = 0.0;
    int64_t n = 0;
    uint64_t h = 0xcbf29ce484222325ull;
    int st = ST_OK;
    int gi = 0;
    int rates_ok = 1;
    for (int j = 0; j < M; j++)
      if (!(x.k[j] > 0.0) || !isfinite(x.k[j])) rates_ok = 0;
    if (!rates_ok || !grid_ok || load_init(m, init, p, Pi, &t) != 0) {
      st = ST_BAD_INPUT;
      if (x.states) memset(x.states, 0, sizeof(int32_t) * (size_t)G * O);
      goto done;
    }
    for (;;) {
      /* 1. Match: every rule at every compartment. */
      int overflow = 0;
      for (int j = 0; j < M; j++) {
        if (m->rate_law != NULL && m->rate_law[j] > 0) {
          x.H[j] = 0;
          x.Hs[j] = mm_value(m, j, t.content);
        } else {
          if (rule_total(m, &t, j, &x.H[j])) { overflow = 1; break; }
          x.Hs[j] = (double)x.H[j];
        }
        a[j] = x.k[j] * x.Hs[j];
      }
      double a0 = 0.0;
      if (!overflow) {
        a0 = oracle_tree_sum(a, M);
        if (!isfinite(a0)) overflow = 1;
      }
      if (overflow) {
        /* H of the current term is unusable: record states, keep the score unchanged */
        st = ST_PROP_OVERFLOW;
        for (int j = 0; j < M; j++) {
          x.H[j] = 0;
          x.Hs[j] = 0.0;
        }
        for (; gi < G; gi++) record(&x, &t, gi, tnow);
        break;
      }
      if (n == max_events) {
        st = ST_EVENT_LIMIT;
        for (; gi < G; gi++) record(&x, &t, gi, tnow);
        break;
      }
      if (a0 == 0.0) {
        st = ST_ABSORBED;
        for (; gi < G; gi++) record(&x, &t, gi, tnow);
        break;
      }
      /* 2. Resolve: tau ~ Exp(a0), rule j with probability a_j / a0. */
      uint32_t w[4];
      draw(seed, (uint32_t)n, 0, (uint32_t)r, (uint32_t)p, w);
      double u_tau = oracle_u52(w[0], w[1]);
      double u_sel = oracle_u52(w[2], w[3]);
      double tau = (-oracle_log_spec(u_tau)) / a0;
      double tnext = tnow + tau;
      while (gi < G && grid[gi] < tnext) {
        record(&x, &t, gi, tnow);
        gi++;
      }
      if (tnext > T) break; /* the event falls past the horizon: not applied */
      int j = oracle_select(a, M, u_sel * a0);
      /* stochastic choice of the context within rule j: x in [0, H_j) */
      uint32_t wc[4];
      draw(seed, (uint32_t)n, 1, (uint32_t)r, (uint32_t)p, wc);
      uint64_t W = (uint64_t)wc[0] | ((uint64_t)wc[1] << 32);
      uint64_t xc = (uint64_t)(((unsigned __int128)W * (unsigned __int128)(uint64_t)x.H[j]) >> 64);
      if (m->rate_law != NULL && m->rate_law[j] > 0) xc = 0; /* flat: the root is the only context */
      int ctx = -1;
      uint64_t cum = 0;
      if (m->kind[j] == K_FUSION || m->kind[j] == K_PAIR) {
        /* pairs in ascending (d1, d2) order; the context id is d1 | d2 << 16 */
        for (int d1 = 0; d1 < C && ctx < 0; d1++)
          for (int d2 = 0; d2 < C; d2++) {
            if (!is_pair(m, &t, j, d1, d2)) continue;
            int64_t hc;
            pair_count(m, &t, j, d1, d2, &hc);
            cum += (uint64_t)hc;
            if (xc < cum) { ctx = d1 | (d2 << 16); break; }
          }
      }
      for (int c = 0; c < C && m->kind[j] != K_FUSION && m->kind[j] != K_PAIR; c++) {
        if (!is_context(m, &t, j, c)) continue;
        int64_t hc;
        match_count(m, &t, j, c, &hc);
        cum += (uint64_t)hc;
        if (xc < cum) { ctx = c; break; }
      }
      /* 3. Update. */
      int ast = apply_rule(m, &t, j, ctx);
      if (ast != ST_OK) {
        st = ast;
        for (; gi < G; gi++) record(&x, &t, gi, tnow);
        break;
      }
      if (x.partial) {
        for (int i = 0; i < M; i++) x.I[i] = x.I[i] + x.Hs[i] * (tnext - tnow);
        x.N[j] += 1;
      }
      if (log_cap > 0 && n < log_cap) {
        if (log_rule) log_rule[lq * log_cap + n] = j;
        if (log_slot) log_slot[lq * log_cap + n] = ctx;
        if (log_t) log_t[lq * log_cap + n] = tnext;
      }
      tnow = tnext;
      n = n + 1;
      h = fnv_event(h, (uint32_t)j, (uint32_t)ctx);
    }
  done:
    if (status) status[lq] = st;
    if (events) events[lq] = n;
    if (hash) hash[lq] = h;
    if (final_t) final_t[lq] = tnow;
  }
  free(t.alive);
  free(t.label);
  free(t.parent);
  free(t.wrap);
  free(t.content);
  free(a);
  free(x.N);
  free(x.I);
  free(x.H);
  free(x.Hs);
  free(x.obs);
  return 0;
}

/* Combinatorial count H_j of every rule at a given term (for the pins).     */
/* term: flat counts [S] or slot image [C][3+2S].  Returns -1 on overflow or */
/* invalid term.                                                              */
int oracle_rule_totals(const oracle_model* m, const int32_t* init, int64_t* H_out) {
  const int S = m->S, C = m->C;
  term_t t;
  t.S = S;
  t.C = C;
  t.alive = malloc(sizeof(int32_t) * C);
  t.label = malloc(sizeof(int32_t) * C);
  t.parent = malloc(sizeof(int32_t) * C);
  t.wrap = malloc(sizeof(int32_t) * (size_t)C * S);
  t.content = malloc(sizeof(int32_t) * (size_t)C * S);
  int rc = load_init(m, init, 0, 1, &t);
  for (int j = 0; rc == 0 && j < m->M; j++)
    if (rule_total(m, &t, j, &H_out[j])) rc = -1;
  free(t.alive);
  free(t.label);
  free(t.parent);
  free(t.wrap);
  free(t.content);
  return rc;
}

/* h_j as a double of every rule at a flat term's counts [S]: the number of
 * reactant combinations, or the Michaelis-Menten value (for the pins).
 * Returns -1 on an int64 overflow. */
int oracle_rule_h(const oracle_model* m, const int32_t* counts, double* h_out) {
  term_t t;
  int32_t alive = 1, label = 0, parent = -1, wrap0 = 0;
  int32_t* wrap = calloc((size_t)m->S, sizeof(int32_t));
  t.S = m->S;
  t.C = 1;
  t.alive = &alive;
  t.label = &label;
  t.parent = &parent;
  t.wrap = wrap;
  t.content = (int32_t*)counts;
  (void)wrap0;
  int rc = 0;
  for (int j = 0; j < m->M && rc == 0; j++) {
    if (m->rate_law != NULL && m->rate_law[j] > 0) {
      h_out[j] = mm_value(m, j, counts);
    } else {
      int64_t H;
      if (rule_total(m, &t, j, &H)) rc = -1;
      else h_out[j] = (double)H;
    }
  }
  free(wrap);
  return rc;
}

/* Vector helpers for the pins (plain loops over the scalar routines). */
void oracle_log_spec_array(const double* u, double* out, int64_t n) {
  for (int64_t i = 0; i < n; i++) out[i] = oracle_log_spec(u[i]);
}

void oracle_philox_array(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, int64_t n) {
  for (int64_t i = 0; i < n; i++) oracle_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}
