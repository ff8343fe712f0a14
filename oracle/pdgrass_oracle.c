/*
 * pdGRASS off-tree edge recovery -- plain single-threaded CPU ORACLE.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load this file.  It shares no code,
 * header, table or helper with the CUDA library: it is the slow, literal
 * statement of what the recovery step computes, against which the GPU path is
 * checked.
 *
 * Steps, in the order of Algorithm 1 (pdGRASS) and Sec. 4 of the paper:
 *   1. Split the edges of G into tree and off-tree edges (Sec. 2.2, after
 *      Eq. RT).  Canonical edge id = rank of the CSR entry (u, v), u < v,
 *      among all such entries in row-major order.
 *   2. For every off-tree edge (u, v): l = LCA_T(u, v); the resistance
 *      distance of Eq. RT, the sum of 1/w over the tree path u -> l -> v,
 *      computed EXACTLY and rounded once to nearest-even FP64; the
 *      criticality score; and the density-aware step
 *      beta* = min(hops(u,l), hops(v,l), c) (Eq. beta-new).  Two methods
 *      that must agree bit for bit:
 *        WALK  -- the definition: naive ancestor walk, path sum in a wide
 *                 exact accumulator (slow on deep trees);
 *        DISTS -- Algorithm 1 step 1: exact root distances "dists" (multi-
 *                 limb integers) and a skip table for the LCA query, then
 *                 R_T = D(u) + D(v) - 2 D(l) exactly.  Used by orc_recover.
 *   3. Order: score descending, ties by the smaller edge id (a stable sort of
 *      the id-ordered edge list, Algorithm 1 step 2).
 *   4. Subtasks: one index-linked list per LCA, in that order (Algorithm 1
 *      step 3; Lemma "share LCA" makes the lists independent).
 *   5. Greedy (Sec. 4.1 marking with the "continue" branch): walk the global
 *      order; a marked edge is skipped; an unmarked edge is recovered, and
 *      every later edge of its subtask that is strictly similar to it
 *      (Def. "Similar edge (Strict)") is marked.  Strict similarity is tested
 *      with the explicit beta*-hop BFS neighbourhoods S_{u,b}, S_{v,b} in the
 *      spanning tree T (Def. "BFS step size").  Stop after alpha*|V| edges
 *      (Sec. 2.2 budget).
 *
 * Also here: spanning-tree generation, the step before recovery (Sec. 2.2;
 * Kruskal for the maximum-weight and the effective-weight trees of Eq. weff,
 * orc_spanning_tree at the end of this file).
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *   - R_T is the exact real path sum, rounded once (the paper gives no
 *     rounding rule; this is the only reading that is order-independent).
 *   - score = fl(w_e * R_T(e)) in STRETCH mode (default) or R_T in
 *     RESISTANCE mode; larger score = more critical = earlier.
 *   - "dist" in Eq. beta-new and the BFS neighbourhoods are hop counts in T.
 *   - k = floor(alpha * |V|) in IEEE double unless k_override >= 0; if fewer
 *     than k edges survive one pass, all survivors are returned and the
 *     status is ORC_UNDER_BUDGET (one pass, Sec. 5 "Runtime").
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_UNDER_BUDGET 1
#define ORC_E_ARG (-1)
#define ORC_E_NOT_A_TREE (-3)
#define ORC_E_OOM (-7)

#define ORC_SCORE_STRETCH 0
#define ORC_SCORE_RESISTANCE 1

#define ORC_METHOD_WALK 0  /* explicit path walk: the definition of Eq. RT */
#define ORC_METHOD_DISTS 1 /* Algorithm 1: dists + skip-table LCA, exact */

/* ------------------------------------------------------------------------ */
/* Exact sum of positive doubles: an integer N in units of 2^-1074 held in   */
/* 64-bit limbs (least significant first).  Every finite double is an exact  */
/* multiple of 2^-1074, so adds are exact; one rounding happens at the end.  */

#define ACC_LIMBS 36 /* 2304 bits: 2^1024 * 2^1074 needs 2098 bits + carries */

typedef struct {
  uint64_t limb[ACC_LIMBS];
} exact_acc;

static void acc_zero(exact_acc* a) { memset(a->limb, 0, sizeof(a->limb)); }

static void acc_add_at(exact_acc* a, int idx, uint64_t v) {
  while (v != 0 && idx < ACC_LIMBS) {
    uint64_t old = a->limb[idx];
    a->limb[idx] = old + v;
    v = (a->limb[idx] < old) ? 1u : 0u; /* carry */
    idx++;
  }
}

/* x must be finite and >= 0 */
static void acc_add_double(exact_acc* a, double x) {
  uint64_t bits;
  memcpy(&bits, &x, 8);
  uint64_t ef = (bits >> 52) & 0x7ffu;
  uint64_t frac = bits & ((1ull << 52) - 1);
  uint64_t mant;
  int64_t pos; /* bit position of mant's lowest bit, in units of 2^-1074 */
  if (ef == 0) {
    mant = frac;
    pos = 0;
  } else {
    mant = frac | (1ull << 52);
    pos = (int64_t)ef - 1; /* value = mant * 2^(ef-1075) = mant * 2^(ef-1) * 2^-1074 */
  }
  if (mant == 0) return;
  int idx = (int)(pos / 64);
  int sh = (int)(pos % 64);
  uint64_t lo = mant << sh;
  uint64_t hi = sh ? (mant >> (64 - sh)) : 0;
  acc_add_at(a, idx, lo);
  if (hi) acc_add_at(a, idx + 1, hi);
}

static int acc_bit(const exact_acc* a, int64_t i) {
  if (i < 0) return 0;
  return (int)((a->limb[i / 64] >> (i % 64)) & 1u);
}

/* round-to-nearest, ties-to-even conversion of N * 2^-1074 to double */
static double acc_to_double(const exact_acc* a) {
  int64_t p = -1; /* index of the most significant set bit */
  for (int i = ACC_LIMBS - 1; i >= 0 && p < 0; i--) {
    if (a->limb[i]) {
      for (int b = 63; b >= 0; b--) {
        if ((a->limb[i] >> b) & 1u) {
          p = (int64_t)i * 64 + b;
          break;
        }
      }
    }
  }
  if (p < 0) return 0.0;
  if (p <= 52) { /* N < 2^53: exactly representable */
    uint64_t q = 0;
    for (int64_t i = p; i >= 0; i--) q = (q << 1) | (uint64_t)acc_bit(a, i);
    return ldexp((double)q, -1074);
  }
  uint64_t q = 0; /* the 53 leading bits */
  for (int64_t i = p; i >= p - 52; i--) q = (q << 1) | (uint64_t)acc_bit(a, i);
  int round_bit = acc_bit(a, p - 53);
  int sticky = 0;
  for (int64_t i = p - 54; i >= 0 && !sticky; i--) sticky = acc_bit(a, i);
  if (round_bit && (sticky || (q & 1u))) {
    q += 1;
    if (q == (1ull << 53)) {
      q >>= 1;
      p += 1;
    }
  }
  return ldexp((double)q, (int)(p - 52 - 1074));
}

/* Exposed for the oracle's own pins: exact sum of cnt non-negative doubles,
 * rounded once. */
double orc_exact_sum(const double* xs, int64_t cnt) {
  exact_acc a;
  acc_zero(&a);
  for (int64_t i = 0; i < cnt; i++) acc_add_double(&a, xs[i]);
  return acc_to_double(&a);
}

/* ------------------------------------------------------------------------ */
/* Tree facts: hop depth and r(v) = fl(1/w(v, parent v))                     */

typedef struct {
  int64_t n;
  const int64_t* row_ptr;
  const int32_t* col;
  const double* w;
  const int32_t* parent;
  int64_t* depth;   /* hops from the root */
  double* r;        /* resistance of the tree edge (v, parent v) */
  int64_t* ch_ptr;  /* children of each vertex in T (CSR) */
  int32_t* ch;
} tree_t;

static void tree_free(tree_t* t) {
  free(t->depth);
  free(t->r);
  free(t->ch_ptr);
  free(t->ch);
}

static int tree_build(tree_t* t, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w,
                      const int32_t* parent) {
  memset(t, 0, sizeof(*t));
  t->n = n;
  t->row_ptr = row_ptr;
  t->col = col;
  t->w = w;
  t->parent = parent;
  t->depth = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  t->r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  t->ch_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  t->ch = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  if (!t->depth || !t->r || !t->ch_ptr || !t->ch) return ORC_E_OOM;
  int64_t roots = 0;
  for (int64_t v = 0; v < n; v++) {
    int32_t p = parent[v];
    if (p < 0) {
      roots++;
      t->r[v] = 0.0;
      continue;
    }
    if (p >= n || p == v) return ORC_E_NOT_A_TREE;
    /* weight of the tree edge: scan v's row for p */
    int found = 0;
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
      if (col[e] == p) {
        t->r[v] = 1.0 / w[e];
        found = 1;
        break;
      }
    }
    if (!found) return ORC_E_NOT_A_TREE;
    t->ch_ptr[p + 1]++;
  }
  if (roots != 1) return ORC_E_NOT_A_TREE;
  /* hop depth: walk to the root, memoised; -1 = unknown, -2 = on the stack */
  for (int64_t v = 0; v < n; v++) t->depth[v] = -1;
  int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!stack) return ORC_E_OOM;
  for (int64_t v = 0; v < n; v++) {
    int64_t sp = 0, x = v;
    while (x >= 0 && t->depth[x] == -1) {
      t->depth[x] = -2;
      stack[sp++] = x;
      x = parent[x];
    }
    if (x >= 0 && t->depth[x] == -2) {
      free(stack);
      return ORC_E_NOT_A_TREE; /* cycle */
    }
    int64_t d = (x < 0) ? -1 : t->depth[x];
    while (sp > 0) {
      int64_t y = stack[--sp];
      t->depth[y] = ++d;
    }
  }
  free(stack);
  for (int64_t v = 0; v < n; v++) t->ch_ptr[v + 1] += t->ch_ptr[v];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!fill) return ORC_E_OOM;
  for (int64_t v = 0; v < n; v++) fill[v] = t->ch_ptr[v];
  for (int64_t v = 0; v < n; v++)
    if (parent[v] >= 0) t->ch[fill[parent[v]]++] = (int32_t)v;
  free(fill);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Step 1: tree / off-tree split with canonical ids                          */

typedef struct {
  int64_t count;
  int32_t* u;
  int32_t* v;
  int32_t* id;
  double* w;
} offtree_t;

static void offtree_free(offtree_t* o) {
  free(o->u);
  free(o->v);
  free(o->id);
  free(o->w);
}

static int offtree_build(offtree_t* o, const tree_t* t) {
  memset(o, 0, sizeof(*o));
  int64_t nnz = t->row_ptr[t->n];
  int64_t cap = nnz / 2 + 1;
  o->u = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  o->v = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  o->id = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  o->w = (double*)malloc(sizeof(double) * (size_t)cap);
  if (!o->u || !o->v || !o->id || !o->w) return ORC_E_OOM;
  int64_t next_id = 0;
  for (int64_t u = 0; u < t->n; u++) {
    for (int64_t e = t->row_ptr[u]; e < t->row_ptr[u + 1]; e++) {
      int32_t v = t->col[e];
      if (u >= v) continue;
      int64_t id = next_id++;
      int is_tree = (t->parent[v] == u) || (t->parent[u] == v);
      if (is_tree) continue;
      o->u[o->count] = (int32_t)u;
      o->v[o->count] = v;
      o->id[o->count] = (int32_t)id;
      o->w[o->count] = t->w[e];
      o->count++;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Step 2: LCA (naive walk), exact R_T, score and beta*                       */

static void score_one(const tree_t* t, int32_t u, int32_t v, double w, int32_t c, int score_mode,
                      int32_t* lca_out, double* res_out, double* score_out, int32_t* beta_out) {
  exact_acc acc;
  acc_zero(&acc);
  int64_t a = u, b = v;
  int64_t hu = 0, hv = 0; /* hops walked from u and from v */
  while (t->depth[a] > t->depth[b]) {
    acc_add_double(&acc, t->r[a]);
    a = t->parent[a];
    hu++;
  }
  while (t->depth[b] > t->depth[a]) {
    acc_add_double(&acc, t->r[b]);
    b = t->parent[b];
    hv++;
  }
  while (a != b) {
    acc_add_double(&acc, t->r[a]);
    acc_add_double(&acc, t->r[b]);
    a = t->parent[a];
    b = t->parent[b];
    hu++;
    hv++;
  }
  double R = acc_to_double(&acc);
  *lca_out = (int32_t)a;
  *res_out = R;
  *score_out = (score_mode == ORC_SCORE_RESISTANCE) ? R : w * R;
  int64_t bs = hu < hv ? hu : hv;
  if (bs > c) bs = c;
  *beta_out = (int32_t)bs;
}

/* ------------------------------------------------------------------------ */
/* Step 2 via Algorithm 1's own data: "dists" (exact root distances) and the */
/* skip table S (binary lifting).  D(v) is an integer of `limbs` 64-bit words */
/* in units of 2^(e_min - 52), where e_min is the smallest binary exponent of */
/* any r(v): every r(v) is then an exact multiple of that unit, so sums are   */
/* exact and R_T = D(u) + D(v) - 2 D(l) equals the path sum exactly.  The     */
/* width adapts to the exponent range and the tree depth, so no input that    */
/* the walk can handle is refused.                                            */

typedef struct {
  int limbs;
  int e_min;
  uint64_t* D;    /* n * limbs */
  int levels;
  int32_t* skip;  /* levels * n: skip[j*n + v] = 2^j-th ancestor or -1 */
} dists_t;

static void dists_free(dists_t* d) {
  free(d->D);
  free(d->skip);
}

static int exp_of(double x) {
  uint64_t b;
  memcpy(&b, &x, 8);
  return (int)((b >> 52) & 0x7ff) - 1023;
}

static int dists_build(dists_t* d, const tree_t* t) {
  memset(d, 0, sizeof(*d));
  int64_t n = t->n, maxdep = 0;
  int e_min = 1 << 30, e_max = -(1 << 30);
  for (int64_t v = 0; v < n; v++) {
    if (t->depth[v] > maxdep) maxdep = t->depth[v];
    if (t->parent[v] < 0) continue;
    int e = exp_of(t->r[v]);
    if (e < e_min) e_min = e;
    if (e > e_max) e_max = e;
  }
  if (e_min > e_max) e_min = e_max = 0; /* single vertex */
  int dep_bits = 0;
  while ((1ll << dep_bits) <= maxdep) dep_bits++;
  int bits = (e_max - e_min + 53) + dep_bits + 2; /* +1 for 2*D(l), +1 spare */
  d->limbs = (bits + 63) / 64;
  d->e_min = e_min;
  d->D = (uint64_t*)calloc((size_t)n * (size_t)d->limbs, sizeof(uint64_t));
  d->levels = dep_bits > 0 ? dep_bits : 1;
  d->skip = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * (size_t)d->levels);
  if (!d->D || !d->skip) return ORC_E_OOM;
  /* vertices by increasing depth (counting sort) so parents come first */
  int64_t* cnt = (int64_t*)calloc((size_t)maxdep + 2, sizeof(int64_t));
  int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!cnt || !ord) {
    free(cnt);
    free(ord);
    return ORC_E_OOM;
  }
  for (int64_t v = 0; v < n; v++) cnt[t->depth[v] + 1]++;
  for (int64_t i = 0; i <= maxdep; i++) cnt[i + 1] += cnt[i];
  for (int64_t v = 0; v < n; v++) ord[cnt[t->depth[v]]++] = v;
  int L = d->limbs;
  for (int64_t i = 0; i < n; i++) {
    int64_t v = ord[i];
    int32_t p = t->parent[v];
    if (p < 0) continue; /* root: D = 0 */
    uint64_t* dv = d->D + (size_t)v * L;
    const uint64_t* dp = d->D + (size_t)p * L;
    for (int k = 0; k < L; k++) dv[k] = dp[k];
    /* add r(v) = mant * 2^(e - 52) = (mant << (e - e_min)) units */
    uint64_t b;
    memcpy(&b, &t->r[v], 8);
    uint64_t mant = (b & ((1ull << 52) - 1)) | (1ull << 52);
    int sh = exp_of(t->r[v]) - e_min;
    int idx = sh / 64, off = sh % 64;
    uint64_t lo = mant << off, hi = off ? (mant >> (64 - off)) : 0;
    uint64_t carry = 0;
    for (int k = idx; k < L; k++) {
      uint64_t add = (k == idx) ? lo : (k == idx + 1 ? hi : 0);
      uint64_t old = dv[k];
      uint64_t s1 = old + add;
      uint64_t c1 = s1 < old;
      uint64_t s2 = s1 + carry;
      uint64_t c2 = s2 < s1;
      dv[k] = s2;
      carry = c1 | c2;
    }
  }
  free(cnt);
  free(ord);
  /* skip table: level 0 = parent, level j = level j-1 applied twice */
  for (int64_t v = 0; v < n; v++) d->skip[v] = t->parent[v];
  for (int j = 1; j < d->levels; j++)
    for (int64_t v = 0; v < n; v++) {
      int32_t a = d->skip[(size_t)(j - 1) * n + v];
      d->skip[(size_t)j * n + v] = (a < 0) ? -1 : d->skip[(size_t)(j - 1) * n + a];
    }
  return ORC_OK;
}

static int32_t lca_query(const tree_t* t, const dists_t* d, int32_t u, int32_t v) {
  int64_t n = t->n;
  if (t->depth[u] < t->depth[v]) {
    int32_t x = u;
    u = v;
    v = x;
  }
  int64_t diff = t->depth[u] - t->depth[v];
  for (int j = 0; diff; j++, diff >>= 1)
    if (diff & 1) u = d->skip[(size_t)j * n + u];
  if (u == v) return u;
  for (int j = d->levels - 1; j >= 0; j--) {
    int32_t a = d->skip[(size_t)j * n + u], b = d->skip[(size_t)j * n + v];
    if (a != b) {
      u = a;
      v = b;
    }
  }
  return t->parent[u];
}

static void score_one_dists(const tree_t* t, const dists_t* d, int32_t u, int32_t v, double w, int32_t c,
                            int score_mode, int32_t* lca_out, double* res_out, double* score_out,
                            int32_t* beta_out) {
  int32_t l = lca_query(t, d, u, v);
  int L = d->limbs;
  const uint64_t* du = d->D + (size_t)u * L;
  const uint64_t* dv = d->D + (size_t)v * L;
  const uint64_t* dl = d->D + (size_t)l * L;
  /* (D(u) - D(l)) + (D(v) - D(l)), limb by limb */
  uint64_t r[64];
  uint64_t borrow1 = 0, borrow2 = 0, carry = 0;
  for (int k = 0; k < L; k++) {
    uint64_t a = du[k] - dl[k] - borrow1;
    borrow1 = (du[k] < dl[k]) || (du[k] - dl[k] < borrow1);
    uint64_t b = dv[k] - dl[k] - borrow2;
    borrow2 = (dv[k] < dl[k]) || (dv[k] - dl[k] < borrow2);
    uint64_t s1 = a + b;
    uint64_t c1 = s1 < a;
    uint64_t s2 = s1 + carry;
    uint64_t c2 = s2 < s1;
    r[k] = s2;
    carry = c1 | c2;
  }
  /* into units of 2^-1074: shift left by 1074 + (e_min - 52) = 1022 + e_min */
  exact_acc acc;
  acc_zero(&acc);
  int sh = 1022 + d->e_min;
  for (int k = 0; k < L; k++) {
    if (!r[k]) continue;
    int64_t pos = (int64_t)k * 64 + sh;
    int idx = (int)(pos / 64), off = (int)(pos % 64);
    acc_add_at(&acc, idx, r[k] << off);
    if (off) acc_add_at(&acc, idx + 1, r[k] >> (64 - off));
  }
  double R = acc_to_double(&acc);
  *lca_out = l;
  *res_out = R;
  *score_out = (score_mode == ORC_SCORE_RESISTANCE) ? R : w * R;
  int64_t hu = t->depth[u] - t->depth[l], hv = t->depth[v] - t->depth[l];
  int64_t bs = hu < hv ? hu : hv;
  if (bs > c) bs = c;
  *beta_out = (int32_t)bs;
}

/* ------------------------------------------------------------------------ */
/* Step 3: order (score descending, id ascending)                             */

typedef struct {
  double score;
  int32_t id;
  int64_t idx; /* index into the off-tree arrays */
} order_item;

static int cmp_order(const void* x, const void* y) {
  const order_item* a = (const order_item*)x;
  const order_item* b = (const order_item*)y;
  if (a->score > b->score) return -1;
  if (a->score < b->score) return 1;
  return (a->id < b->id) ? -1 : (a->id > b->id);
}

/* ------------------------------------------------------------------------ */
/* beta-hop neighbourhood in T by BFS, recorded as stamp[x] = tag            */

static void bfs_stamp(const tree_t* t, int32_t src, int32_t hops, int64_t* stamp, int64_t tag, int32_t* queue,
                      int32_t* qdist) {
  int64_t head = 0, tail = 0;
  stamp[src] = tag;
  queue[tail] = src;
  qdist[tail++] = 0;
  while (head < tail) {
    int32_t x = queue[head];
    int32_t d = qdist[head++];
    if (d == hops) continue;
    int32_t p = t->parent[x];
    if (p >= 0 && stamp[p] != tag) {
      stamp[p] = tag;
      queue[tail] = p;
      qdist[tail++] = d + 1;
    }
    for (int64_t i = t->ch_ptr[x]; i < t->ch_ptr[x + 1]; i++) {
      int32_t y = t->ch[i];
      if (stamp[y] != tag) {
        stamp[y] = tag;
        queue[tail] = y;
        qdist[tail++] = d + 1;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Public entry points                                                        */

static int64_t budget_k(int64_t n, double alpha, int64_t k_override) {
  if (k_override >= 0) return k_override;
  double kd = floor(alpha * (double)n);
  if (kd < 0) kd = 0;
  return (int64_t)kd;
}

/* Per-off-tree-edge scores, in canonical id order.  All output arrays hold
 * m - n + 1 entries (caller-allocated). */
int orc_offtree_scores(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w, const int32_t* parent,
                       int32_t c, int score_mode, int method, int64_t* n_off, int32_t* off_u, int32_t* off_v,
                       int32_t* off_id, int32_t* lca, double* resistance, double* score, int32_t* beta) {
  if (n <= 0 || !row_ptr || !col || !w || !parent || c < 0 || !n_off) return ORC_E_ARG;
  tree_t t;
  int st = tree_build(&t, n, row_ptr, col, w, parent);
  if (st != ORC_OK) {
    tree_free(&t);
    return st;
  }
  offtree_t o;
  st = offtree_build(&o, &t);
  if (st != ORC_OK) {
    offtree_free(&o);
    tree_free(&t);
    return st;
  }
  dists_t d;
  memset(&d, 0, sizeof(d));
  if (method == ORC_METHOD_DISTS && (st = dists_build(&d, &t)) != ORC_OK) {
    dists_free(&d);
    offtree_free(&o);
    tree_free(&t);
    return st;
  }
  for (int64_t i = 0; i < o.count; i++) {
    off_u[i] = o.u[i];
    off_v[i] = o.v[i];
    off_id[i] = o.id[i];
    if (method == ORC_METHOD_DISTS)
      score_one_dists(&t, &d, o.u[i], o.v[i], o.w[i], c, score_mode, &lca[i], &resistance[i], &score[i], &beta[i]);
    else
      score_one(&t, o.u[i], o.v[i], o.w[i], c, score_mode, &lca[i], &resistance[i], &score[i], &beta[i]);
  }
  *n_off = o.count;
  dists_free(&d);
  offtree_free(&o);
  tree_free(&t);
  return ORC_OK;
}

/* Recovery: the first k recovered off-tree edge ids in recovery order.
 * out_full_count (nullable) receives the number of edges one full pass would
 * recover (the greedy is then run to the end of the order instead of
 * stopping at k).  Returns ORC_OK, ORC_UNDER_BUDGET or a negative error. */
int orc_recover(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w, const int32_t* parent,
                double alpha, int32_t c, int score_mode, int64_t k_override, int32_t* out_ids, double* out_scores,
                int64_t out_capacity, int64_t* out_count, int64_t* out_full_count) {
  if (n <= 0 || !row_ptr || !col || !w || !parent || c < 0 || !out_count) return ORC_E_ARG;
  if (!(alpha >= 0.0) && k_override < 0) return ORC_E_ARG;
  int64_t k = budget_k(n, alpha, k_override);
  tree_t t;
  int st = tree_build(&t, n, row_ptr, col, w, parent);
  if (st != ORC_OK) {
    tree_free(&t);
    return st;
  }
  offtree_t o;
  st = offtree_build(&o, &t);
  if (st != ORC_OK) {
    offtree_free(&o);
    tree_free(&t);
    return st;
  }
  int64_t E = o.count;
  size_t E1 = (size_t)(E > 0 ? E : 1);
  int32_t* lca = (int32_t*)malloc(sizeof(int32_t) * E1);
  double* res = (double*)malloc(sizeof(double) * E1);
  double* sc = (double*)malloc(sizeof(double) * E1);
  int32_t* beta = (int32_t*)malloc(sizeof(int32_t) * E1);
  order_item* ord = (order_item*)malloc(sizeof(order_item) * E1);
  int64_t* next_in_task = (int64_t*)malloc(sizeof(int64_t) * E1); /* linked list, by position in ord */
  int64_t* task_tail = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  unsigned char* marked = (unsigned char*)calloc(E1, 1);
  int64_t* stamp_u = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* stamp_v = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* qdist = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!lca || !res || !sc || !beta || !ord || !next_in_task || !task_tail || !marked || !stamp_u || !stamp_v ||
      !queue || !qdist) {
    st = ORC_E_OOM;
    goto done;
  }
  /* step 2: scores (dists + skip table, Algorithm 1 step 1) */
  {
    dists_t d;
    st = dists_build(&d, &t);
    if (st != ORC_OK) {
      dists_free(&d);
      goto done;
    }
    for (int64_t i = 0; i < E; i++)
      score_one_dists(&t, &d, o.u[i], o.v[i], o.w[i], c, score_mode, &lca[i], &res[i], &sc[i], &beta[i]);
    dists_free(&d);
  }
  /* step 3: global order */
  for (int64_t i = 0; i < E; i++) {
    ord[i].score = sc[i];
    ord[i].id = o.id[i];
    ord[i].idx = i;
  }
  qsort(ord, (size_t)E, sizeof(order_item), cmp_order);
  /* Steps 4-5 run on a prefix [0, P) of the global order: the greedy decides
   * every edge from earlier edges only, so its decisions inside a prefix do
   * not depend on what follows.  If the prefix yields fewer than k recovered
   * edges it is enlarged and the greedy restarts. */
  int run_full = (out_full_count != NULL);
  int64_t P = run_full ? E : (2 * k + 1024 < E ? 2 * k + 1024 : E);
  int64_t taken = 0, full = 0;
restart:
  /* step 4: subtasks = index-linked lists per LCA, in global order */
  for (int64_t x = 0; x < n; x++) task_tail[x] = -1;
  for (int64_t pos = P - 1; pos >= 0; pos--) {
    int32_t l = lca[ord[pos].idx];
    next_in_task[pos] = task_tail[l]; /* built back to front: head is the earliest */
    task_tail[l] = pos;
  }
  for (int64_t x = 0; x < n; x++) {
    stamp_u[x] = -1;
    stamp_v[x] = -1;
  }
  if (P > 0) memset(marked, 0, (size_t)P);
  taken = 0;
  full = 0;
  /* step 5: greedy over the global order */
  for (int64_t pos = 0; pos < P; pos++) {
    if (marked[pos]) continue; /* the "continue" branch */
    int64_t i = ord[pos].idx;
    if (taken < k) {
      if (taken < out_capacity) {
        if (out_ids) out_ids[taken] = o.id[i];
        if (out_scores) out_scores[taken] = sc[i];
      }
      taken++;
    }
    full++;
    if (taken >= k && !run_full) break;
    /* mark later edges of the same subtask that are strictly similar */
    int32_t b = beta[i];
    bfs_stamp(&t, o.u[i], b, stamp_u, pos, queue, qdist);
    bfs_stamp(&t, o.v[i], b, stamp_v, pos, queue, qdist);
    for (int64_t q = next_in_task[pos]; q >= 0; q = next_in_task[q]) {
      if (marked[q]) continue;
      int64_t j = ord[q].idx;
      int32_t uu = o.u[j], vv = o.v[j];
      int sim = (stamp_u[uu] == pos && stamp_v[vv] == pos) || (stamp_v[uu] == pos && stamp_u[vv] == pos);
      if (sim) marked[q] = 1;
    }
  }
  if (taken < k && P < E) {
    P = (4 * P < E) ? 4 * P : E;
    goto restart;
  }
  *out_count = taken;
  if (out_full_count) *out_full_count = full;
  st = (taken < k) ? ORC_UNDER_BUDGET : ORC_OK;
  if (taken > out_capacity) st = ORC_E_ARG;
done:
  free(lca);
  free(res);
  free(sc);
  free(beta);
  free(ord);
  free(next_in_task);
  free(task_tail);
  free(marked);
  free(stamp_u);
  free(stamp_v);
  free(queue);
  free(qdist);
  offtree_free(&o);
  tree_free(&t);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Spanning-tree generation, the step before recovery (Sec. 2.2: feGRASS     */
/* first builds a spanning tree from the effective weight of Eq. weff).      */
/*                                                                            */
/* Kruskal: visit the edges in the order (key descending, canonical edge id  */
/* ascending) and keep every edge that joins two different trees of the      */
/* forest built so far (union-find).  Keys:                                   */
/*   ORC_TREE_MAX_WEIGHT  key = w(e)                                          */
/*   ORC_TREE_FEGRASS     key = W_eff(e) = (w * log(max(deg u, deg v)))       */
/*                        / (d(u) + d(v)), each operation rounded to double,  */
/*                        d = BFS hop distance in G from the vertex of        */
/*                        maximum degree (ties: smaller id); G connected.     */
/* Rooting: every component is rooted at its maximum-degree vertex (ties:    */
/* smaller id) and parents come from a BFS over the tree edges.              */
/* Returns ORC_OK or ORC_E_ARG (FEGRASS on a disconnected graph).            */

#define ORC_TREE_MAX_WEIGHT 0
#define ORC_TREE_FEGRASS 1

typedef struct {
  double key;
  int32_t id;
} orc_kedge;

static int kedge_order(const void* a, const void* b) {
  const orc_kedge* x = (const orc_kedge*)a;
  const orc_kedge* y = (const orc_kedge*)b;
  if (x->key > y->key) return -1;
  if (x->key < y->key) return 1;
  return (x->id < y->id) ? -1 : (x->id > y->id);
}

static int32_t uf_find(int32_t* up, int32_t x) {
  while (up[x] != x) {
    up[x] = up[up[x]];
    x = up[x];
  }
  return x;
}

/* better root: larger degree, then smaller id */
static int better_root(const int64_t* rp, int32_t a, int32_t b) {
  const int64_t da = rp[a + 1] - rp[a], db = rp[b + 1] - rp[b];
  return da > db || (da == db && a < b);
}

int orc_spanning_tree(int64_t n, const int64_t* rp, const int32_t* col, const double* w, int kind,
                      int32_t* parent) {
  const int64_t m = rp[n] / 2;
  int32_t *eu = malloc(sizeof(int32_t) * (m + 1)), *ev = malloc(sizeof(int32_t) * (m + 1));
  double* ew = malloc(sizeof(double) * (m + 1));
  orc_kedge* ord = malloc(sizeof(orc_kedge) * (m + 1));
  int32_t* up = malloc(sizeof(int32_t) * n);
  int32_t* dist = malloc(sizeof(int32_t) * n);
  int32_t* queue = malloc(sizeof(int32_t) * n);
  uint8_t* in_tree = calloc((size_t)m + 1, 1);
  int64_t* tptr = calloc((size_t)n + 1, sizeof(int64_t));
  int32_t* tadj = malloc(sizeof(int32_t) * (2 * n + 1));
  int32_t* best = malloc(sizeof(int32_t) * n);
  int st = ORC_OK;
  if (!eu || !ev || !ew || !ord || !up || !dist || !queue || !in_tree || !tptr || !tadj || !best) {
    st = ORC_E_OOM;
    goto done;
  }
  /* canonical edges: entries (u, v) with u < v in row-major order */
  int64_t e = 0;
  for (int64_t u = 0; u < n; u++)
    for (int64_t p = rp[u]; p < rp[u + 1]; p++)
      if (col[p] > u) {
        eu[e] = (int32_t)u;
        ev[e] = col[p];
        ew[e] = w[p];
        e++;
      }
  /* keys */
  if (kind == ORC_TREE_FEGRASS) {
    int32_t root = 0;
    for (int32_t v = 1; v < n; v++)
      if (better_root(rp, v, root)) root = v;
    for (int64_t v = 0; v < n; v++) dist[v] = -1;
    int64_t head = 0, tail = 0;
    dist[root] = 0;
    queue[tail++] = root;
    while (head < tail) {
      const int32_t x = queue[head++];
      for (int64_t p = rp[x]; p < rp[x + 1]; p++)
        if (dist[col[p]] < 0) {
          dist[col[p]] = dist[x] + 1;
          queue[tail++] = col[p];
        }
    }
    if (tail != n) {
      st = ORC_E_ARG;
      goto done;
    }
    for (int64_t i = 0; i < m; i++) {
      const int64_t du = rp[eu[i] + 1] - rp[eu[i]], dv = rp[ev[i] + 1] - rp[ev[i]];
      const double lg = log((double)(du > dv ? du : dv));
      const double num = ew[i] * lg;
      ord[i].key = num / (double)(dist[eu[i]] + dist[ev[i]]);
      ord[i].id = (int32_t)i;
    }
  } else {
    for (int64_t i = 0; i < m; i++) {
      ord[i].key = ew[i];
      ord[i].id = (int32_t)i;
    }
  }
  /* Kruskal */
  qsort(ord, (size_t)m, sizeof(orc_kedge), kedge_order);
  for (int64_t v = 0; v < n; v++) up[v] = (int32_t)v;
  for (int64_t i = 0; i < m; i++) {
    const int32_t id = ord[i].id;
    const int32_t a = uf_find(up, eu[id]), b = uf_find(up, ev[id]);
    if (a == b) continue;
    up[a] = b;
    in_tree[id] = 1;
  }
  /* tree adjacency */
  for (int64_t i = 0; i < m; i++)
    if (in_tree[i]) {
      tptr[eu[i] + 1]++;
      tptr[ev[i] + 1]++;
    }
  for (int64_t v = 0; v < n; v++) tptr[v + 1] += tptr[v];
  for (int64_t v = 0; v < n; v++) best[v] = -1;
  {
    int64_t* fill = calloc((size_t)n, sizeof(int64_t));
    if (!fill) {
      st = ORC_E_OOM;
      goto done;
    }
    for (int64_t i = 0; i < m; i++)
      if (in_tree[i]) {
        tadj[tptr[eu[i]] + fill[eu[i]]++] = ev[i];
        tadj[tptr[ev[i]] + fill[ev[i]]++] = eu[i];
      }
    free(fill);
  }
  /* root of every component, then BFS over the tree from it */
  for (int64_t v = 0; v < n; v++) {
    const int32_t r = uf_find(up, (int32_t)v);
    if (best[r] < 0 || better_root(rp, (int32_t)v, best[r])) best[r] = (int32_t)v;
  }
  for (int64_t v = 0; v < n; v++) {
    parent[v] = -1;
    dist[v] = -1;
  }
  for (int64_t v = 0; v < n; v++) {
    if (best[v] < 0) continue; /* v is not a union-find root */
    const int32_t root = best[v];
    int64_t head = 0, tail = 0;
    dist[root] = 0;
    queue[tail++] = root;
    while (head < tail) {
      const int32_t x = queue[head++];
      for (int64_t p = tptr[x]; p < tptr[x + 1]; p++) {
        const int32_t y = tadj[p];
        if (dist[y] < 0) {
          dist[y] = dist[x] + 1;
          parent[y] = x;
          queue[tail++] = y;
        }
      }
    }
  }
done:
  free(eu);
  free(ev);
  free(ew);
  free(ord);
  free(up);
  free(dist);
  free(queue);
  free(in_tree);
  free(tptr);
  free(tadj);
  free(best);
  return st;
}
