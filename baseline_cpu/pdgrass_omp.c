/*
 * The paper's multi-threaded CPU method (Sec. 4.1, Algorithm 1, Sec. 5
 * setup), written with OpenMP: a CONTEXT implementation that the benchmark
 * times on the host's cores beside the GPU path.  It is not the oracle (the
 * oracle is the single-threaded reference in oracle/) and nothing of the GPU
 * library runs here; the test-suite checks that it returns exactly the
 * oracle's recovery.
 *
 * Steps (Algorithm 1):
 *   1. resistance of every off-tree edge: LCA by a skip table (binary
 *      lifting over the tree), root distances summed exactly in 128-bit
 *      fixed point (every r = fl(1/w) is a multiple of 2^-S with
 *      S = 52 - min exponent), R_T = D(u) + D(v) - 2 D(l) rounded once,
 *      score = fl(w R_T) (or R_T), beta* = min(hops(u, l), hops(v, l), c)
 *      (Eq. RT, Eq. beta-new); a parallel loop over the edges;
 *   2. parallel stable sort by score (descending; equal scores keep the
 *      canonical id order): chunks sorted by the threads, then merged pairwise
 *      in parallel;
 *   3. subtasks: one index-linked list per LCA over the order (Lemma "share
 *      LCA"), sorted by size;
 *   4. recovery with the mixed strategy: subtasks with at least CUTOFF edges
 *      (1e5, or 10 % of the off-tree edges if that is smaller) one after the
 *      other with inner parallelism -- blocks of p unmarked edges (the marked
 *      ones are skipped before the parallel region: judge-before-parallel),
 *      every thread finding the later edges of the subtask strictly similar to
 *      its edge, then a serial pass over the block that recovers an edge unless
 *      an earlier recovered edge marked it and applies the marks of the
 *      recovered ones; all other subtasks in parallel, one thread each, in the
 *      sequential greedy (largest first, dynamic schedule).
 *   Strict similarity (Def. "Similar edge (Strict)"): e' = (u', v') of the same
 *   subtask is similar to a recovered e = (u, v) when u' and v' lie in the
 *   beta*(e)-hop BFS neighbourhoods of u and v in T, in either orientation.
 * The budget: k = floor(alpha |V|) recovered edges in the global order (Sec.
 * 2.2).  Steps 3-4 run on a prefix of the order (2k + 1024 edges, then four
 * times longer while fewer than k are recovered); the greedy decides an edge
 * from earlier edges only, so a prefix holding the first k recovered edges
 * gives the same set.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OMP_OK 0
#define OMP_UNDER_BUDGET 1
#define OMP_E_ARG (-1)
#define OMP_E_NOT_A_TREE (-3)
#define OMP_E_RANGE (-4)
#define OMP_E_OOM (-5)

typedef unsigned __int128 u128;

typedef struct {
  double key;  /* score */
  int32_t id;  /* canonical edge id (position in the edge list) */
  int32_t off; /* index among the off-tree edges */
} item_t;

static int item_before(const item_t* a, const item_t* b) {
  if (a->key != b->key) return a->key > b->key;
  return a->id < b->id;
}

static int cmp_item(const void* x, const void* y) {
  const item_t* a = (const item_t*)x;
  const item_t* b = (const item_t*)y;
  return item_before(a, b) ? -1 : (item_before(b, a) ? 1 : 0);
}

static int cmp_pair_i64(const void* x, const void* y) {
  const int64_t* a = (const int64_t*)x;
  const int64_t* b = (const int64_t*)y;
  if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
  return (a[1] > b[1]) - (a[1] < b[1]);
}

/* merge two sorted runs [a, a + na) and [b, b + nb) into out */
static void merge_runs(const item_t* a, int64_t na, const item_t* b, int64_t nb, item_t* out) {
  int64_t i = 0, j = 0, o = 0;
  while (i < na && j < nb) out[o++] = item_before(&b[j], &a[i]) ? b[j++] : a[i++];
  while (i < na) out[o++] = a[i++];
  while (j < nb) out[o++] = b[j++];
}

/* parallel sort: thread chunks by qsort, then rounds of pairwise merges */
static int parallel_sort(item_t* x, int64_t N, int T) {
  if (N <= 1) return OMP_OK;
  int R = 1;
  while (R < T) R <<= 1;
  if ((int64_t)R > N) R = 1;
  item_t* tmp = (item_t*)malloc(sizeof(item_t) * (size_t)N);
  if (!tmp) return OMP_E_OOM;
#pragma omp parallel for schedule(static, 1)
  for (int r = 0; r < R; r++) {
    const int64_t lo = N * r / R, hi = N * (r + 1) / R;
    qsort(x + lo, (size_t)(hi - lo), sizeof(item_t), cmp_item);
  }
  item_t *src = x, *dst = tmp;
  for (int width = 1; width < R; width <<= 1) {
#pragma omp parallel for schedule(static, 1)
    for (int r = 0; r < R; r += 2 * width) {
      const int64_t lo = N * r / R, mid = N * (r + width) / R, hi = N * (r + 2 * width) / R;
      merge_runs(src + lo, mid - lo, src + mid, hi - mid, dst + lo);
    }
    item_t* t = src;
    src = dst;
    dst = t;
  }
  if (src != x) memcpy(x, src, sizeof(item_t) * (size_t)N);
  free(tmp);
  return OMP_OK;
}

/* tree: children lists, preorder, depth, exact root distances, skip table */
typedef struct {
  int64_t n;
  int32_t root;
  const int32_t* parent;
  int64_t* cptr;   /* children CSR */
  int32_t* child;
  int32_t* depth;
  u128* D;         /* root distance in units of 2^-S */
  int S;
  int levels;      /* skip-table levels */
  int32_t* up;     /* up[j * n + v] = 2^j-th ancestor (root maps to itself) */
} tree_t;

static void tree_free(tree_t* t) {
  free(t->cptr);
  free(t->child);
  free(t->depth);
  free(t->D);
  free(t->up);
}

static int tree_build(tree_t* t, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w,
                      const int32_t* parent) {
  memset(t, 0, sizeof(*t));
  t->n = n;
  t->parent = parent;
  t->root = -1;
  for (int64_t v = 0; v < n; v++) {
    if (parent[v] < 0) {
      if (t->root >= 0) return OMP_E_NOT_A_TREE;
      t->root = (int32_t)v;
    } else if (parent[v] >= n) {
      return OMP_E_NOT_A_TREE;
    }
  }
  if (t->root < 0) return OMP_E_NOT_A_TREE;
  t->cptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  t->child = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 1 ? n - 1 : 1));
  t->depth = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  t->D = (u128*)malloc(sizeof(u128) * (size_t)n);
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!t->cptr || !t->child || !t->depth || !t->D || !r || !order || !fill) {
    free(r);
    free(order);
    free(fill);
    return OMP_E_OOM;
  }
  for (int64_t v = 0; v < n; v++)
    if (parent[v] >= 0) t->cptr[parent[v] + 1]++;
  for (int64_t v = 0; v < n; v++) t->cptr[v + 1] += t->cptr[v];
  memcpy(fill, t->cptr, sizeof(int64_t) * (size_t)n);
  for (int64_t v = 0; v < n; v++)
    if (parent[v] >= 0) t->child[fill[parent[v]]++] = (int32_t)v;
  /* r(x) = fl(1 / w(x, parent x)) from the CSR row of x, and the exponent range */
  int e_min = 1 << 30, e_max = -(1 << 30);
  int bad = 0;
#pragma omp parallel for reduction(min : e_min) reduction(max : e_max) reduction(| : bad)
  for (int64_t x = 0; x < n; x++) {
    r[x] = 0.0;
    const int32_t p = parent[x];
    if (p < 0) continue;
    int found = 0;
    for (int64_t q = row_ptr[x]; q < row_ptr[x + 1]; q++)
      if (col[q] == p) {
        r[x] = 1.0 / w[q];
        found = 1;
        break;
      }
    if (!found || !(r[x] > 0) || !isfinite(r[x])) {
      bad = 1;
      continue;
    }
    int e;
    frexp(r[x], &e);
    e -= 1; /* r = m 2^e with 1 <= m < 2 */
    if (e < e_min) e_min = e;
    if (e > e_max) e_max = e;
  }
  if (bad) {
    free(r);
    free(order);
    free(fill);
    return OMP_E_NOT_A_TREE;
  }
  /* BFS order from the root (a parent before its children): depth */
  int64_t head = 0, tail = 0;
  order[tail++] = t->root;
  int32_t max_depth = 0;
  t->S = (e_min == (1 << 30)) ? 0 : 52 - e_min;
  t->depth[t->root] = 0;
  t->D[t->root] = 0;
  while (head < tail) {
    const int32_t x = order[head++];
    for (int64_t q = t->cptr[x]; q < t->cptr[x + 1]; q++) {
      const int32_t y = t->child[q];
      t->depth[y] = t->depth[x] + 1;
      if (t->depth[y] > max_depth) max_depth = t->depth[y];
      order[tail++] = y;
    }
  }
  if (tail != n) { /* a cycle through the parent links leaves vertices unreached */
    free(r);
    free(order);
    free(fill);
    return OMP_E_NOT_A_TREE;
  }
  /* D must fit 128 bits: 2^(e_max - e_min + 53) per edge, at most max_depth edges on a path */
  int dep_bits = 0;
  while ((1ll << dep_bits) <= max_depth) dep_bits++;
  if (e_min != (1 << 30) && e_max - e_min + 53 + dep_bits > 126) {
    free(r);
    free(order);
    free(fill);
    return OMP_E_RANGE;
  }
  for (int64_t i = 0; i < n; i++) {
    const int32_t x = order[i];
    if (x == t->root) continue;
    int e;
    const double m = frexp(r[x], &e); /* r = m 2^e, 1/2 <= m < 1 */
    const uint64_t mant = (uint64_t)ldexp(m, 53);
    const int sh = (e - 1 - 52) + t->S; /* r = mant 2^(e - 53); times 2^S */
    t->D[x] = t->D[parent[x]] + ((u128)mant << sh);
  }
  free(r);
  free(order);
  free(fill);
  /* skip table */
  t->levels = 1;
  while ((1ll << t->levels) <= max_depth) t->levels++;
  t->up = (int32_t*)malloc(sizeof(int32_t) * (size_t)n * (size_t)t->levels);
  if (!t->up) return OMP_E_OOM;
#pragma omp parallel for
  for (int64_t v = 0; v < n; v++) t->up[v] = parent[v] >= 0 ? parent[v] : (int32_t)v;
  for (int j = 1; j < t->levels; j++) {
    const int32_t* a = t->up + (size_t)(j - 1) * n;
    int32_t* b = t->up + (size_t)j * n;
#pragma omp parallel for
    for (int64_t v = 0; v < n; v++) b[v] = a[a[v]];
  }
  return OMP_OK;
}

static int32_t lca_query(const tree_t* t, int32_t u, int32_t v) {
  if (t->depth[u] < t->depth[v]) {
    const int32_t s = u;
    u = v;
    v = s;
  }
  int32_t diff = t->depth[u] - t->depth[v];
  for (int j = 0; diff; j++, diff >>= 1)
    if (diff & 1) u = t->up[(size_t)j * t->n + u];
  if (u == v) return u;
  for (int j = t->levels - 1; j >= 0; j--) {
    const int32_t a = t->up[(size_t)j * t->n + u], b = t->up[(size_t)j * t->n + v];
    if (a != b) {
      u = a;
      v = b;
    }
  }
  return t->parent[u];
}

/* BFS ball of radius b around x in T, stamped with tag; returns nothing (the stamps are the set) */
static void ball(const tree_t* t, int32_t x, int b, int32_t* stamp, int32_t tag, int32_t* q, int32_t* qd) {
  int64_t h = 0, e = 0;
  q[e] = x;
  qd[e++] = 0;
  stamp[x] = tag;
  while (h < e) {
    const int32_t y = q[h], d = qd[h++];
    if (d == b) continue;
    const int32_t p = t->parent[y];
    if (p >= 0 && stamp[p] != tag) {
      stamp[p] = tag;
      q[e] = p;
      qd[e++] = d + 1;
    }
    for (int64_t k = t->cptr[y]; k < t->cptr[y + 1]; k++) {
      const int32_t z = t->child[k];
      if (stamp[z] != tag) {
        stamp[z] = tag;
        q[e] = z;
        qd[e++] = d + 1;
      }
    }
  }
}

/* per-thread scratch of the similarity checks */
typedef struct {
  int32_t* su; /* stamps of the two balls (a tag per recovered edge: at most 2^31 per thread) */
  int32_t* sv;
  int32_t* q;  /* BFS queue and hop counts */
  int32_t* qd;
  int32_t tag;
  int64_t* marks; /* inner parallelism: positions this thread's edge marks */
  int64_t nmarks, cap;
} scratch_t;

static int scratch_push(scratch_t* s, int64_t pos) {
  if (s->nmarks == s->cap) {
    const int64_t c = s->cap ? 2 * s->cap : 1024;
    int64_t* m = (int64_t*)realloc(s->marks, sizeof(int64_t) * (size_t)c);
    if (!m) return OMP_E_OOM;
    s->marks = m;
    s->cap = c;
  }
  s->marks[s->nmarks++] = pos;
  return OMP_OK;
}

typedef struct {
  const tree_t* t;
  const int32_t* ou;
  const int32_t* ov;
  const int32_t* beta;
  const item_t* ord;        /* global order */
  const int64_t* task_pos;  /* positions of each subtask's edges, in order */
  const int64_t* task_ptr;
  uint8_t* marked;          /* per position */
  uint8_t* recovered;       /* per position */
} recov_t;

/* marks set for the recovered edge at position pos: later edges of its subtask strictly similar to it */
static void stamp_edge(const recov_t* R, int64_t pos, scratch_t* s) {
  const int32_t i = R->ord[pos].off;
  const int b = R->beta[i];
  s->tag++;
  ball(R->t, R->ou[i], b, s->su, s->tag, s->q, s->qd);
  ball(R->t, R->ov[i], b, s->sv, s->tag, s->q, s->qd);
}

static int similar_to_stamped(const recov_t* R, int64_t pos, const scratch_t* s) {
  const int32_t j = R->ord[pos].off;
  const int32_t uu = R->ou[j], vv = R->ov[j];
  return (s->su[uu] == s->tag && s->sv[vv] == s->tag) || (s->sv[uu] == s->tag && s->su[vv] == s->tag);
}

/* sequential greedy over subtask x (outer parallelism) */
static void run_serial(const recov_t* R, int64_t x, scratch_t* s) {
  const int64_t lo = R->task_ptr[x], hi = R->task_ptr[x + 1];
  for (int64_t a = lo; a < hi; a++) {
    const int64_t pos = R->task_pos[a];
    if (R->marked[pos]) continue;
    R->recovered[pos] = 1;
    stamp_edge(R, pos, s);
    for (int64_t c = a + 1; c < hi; c++) {
      const int64_t q = R->task_pos[c];
      if (!R->marked[q] && similar_to_stamped(R, q, s)) R->marked[q] = 1;
    }
  }
}

/* inner parallelism over subtask x: blocks of p unmarked edges */
static int run_blocked(const recov_t* R, int64_t x, scratch_t* sc, int p) {
  const int64_t lo = R->task_ptr[x], hi = R->task_ptr[x + 1];
  int64_t* blk = (int64_t*)malloc(sizeof(int64_t) * (size_t)p);
  int err = OMP_OK;
  if (!blk) return OMP_E_OOM;
  int64_t a = lo;
  while (a < hi && err == OMP_OK) {
    /* judge before parallel: the next p unmarked edges (their subtask offsets) */
    int nb = 0;
    while (a < hi && nb < p) {
      if (!R->marked[R->task_pos[a]]) blk[nb++] = a;
      a++;
    }
    if (nb == 0) break;
#pragma omp parallel for num_threads(p) schedule(static, 1)
    for (int k = 0; k < nb; k++) {
      scratch_t* s = &sc[k];  /* one scratch (stamps and mark list) per block slot */
      s->nmarks = 0;
      stamp_edge(R, R->task_pos[blk[k]], s);
      for (int64_t c = blk[k] + 1; c < hi; c++) {
        const int64_t q = R->task_pos[c];
        if (!R->marked[q] && similar_to_stamped(R, q, s))
          if (scratch_push(s, q) != OMP_OK) {
#pragma omp atomic write
            err = OMP_E_OOM;
          }
      }
    }
    /* serial pass in order: an edge marked by an earlier recovered edge is not recovered */
    for (int k = 0; k < nb; k++) {
      const int64_t pos = R->task_pos[blk[k]];
      if (R->marked[pos]) continue; /* an earlier edge of this block, recovered, marked it */
      R->recovered[pos] = 1;
      const scratch_t* s = &sc[k];
      for (int64_t m = 0; m < s->nmarks; m++) R->marked[s->marks[m]] = 1;
    }
  }
  free(blk);
  return err;
}

/*
 * omp_recover -- the whole recovery.  n, row_ptr, col, w: the symmetric CSR
 * of G (host); parent: the spanning tree (-1 at the root).  alpha, c,
 * score_mode (0: fl(w R_T), 1: R_T), k_override (>= 0 replaces floor(alpha n)).
 * threads: p (0: the OpenMP default); cutoff: subtasks with at least this
 * many edges use inner parallelism (< 0: min(1e5, 10 % of the off-tree edges)).
 * out_ids / out_scores (capacity entries): the first k recovered edges, in
 * recovery order; *out_count: how many.  Returns OMP_OK, OMP_UNDER_BUDGET
 * (fewer than k exist: all are returned) or a negative error.
 */
int omp_recover(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w, const int32_t* parent,
                double alpha, int32_t c, int32_t score_mode, int64_t k_override, int32_t threads, int64_t cutoff,
                int32_t* out_ids, double* out_scores, int64_t capacity, int64_t* out_count) {
  if (n < 1 || !row_ptr || !col || !w || !parent || c < 0 || !out_count) return OMP_E_ARG;
  const int T = threads > 0 ? threads : omp_get_max_threads();
  omp_set_num_threads(T);
  int st;
  tree_t t;
  if ((st = tree_build(&t, n, row_ptr, col, w, parent)) != OMP_OK) {
    tree_free(&t);
    return st;
  }
  /* canonical edge list (row-major CSR entries with u < v): counts per row, offsets, fill */
  int64_t* eptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!eptr) {
    tree_free(&t);
    return OMP_E_OOM;
  }
#pragma omp parallel for
  for (int64_t u = 0; u < n; u++) {
    int64_t k = 0;
    for (int64_t q = row_ptr[u]; q < row_ptr[u + 1]; q++) k += col[q] > u;
    eptr[u + 1] = k;
  }
  for (int64_t u = 0; u < n; u++) eptr[u + 1] += eptr[u];
  const int64_t m = eptr[n];
  /* off-tree edges (a tree edge joins a vertex and its parent) */
  uint8_t* is_off = (uint8_t*)malloc((size_t)(m > 0 ? m : 1));
  int32_t *eu = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t *ev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  double* ew = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  int64_t* optr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!is_off || !eu || !ev || !ew || !optr) {
    st = OMP_E_OOM;
    goto out0;
  }
#pragma omp parallel for
  for (int64_t u = 0; u < n; u++) {
    int64_t e = eptr[u], k = 0;
    for (int64_t q = row_ptr[u]; q < row_ptr[u + 1]; q++) {
      const int32_t v = col[q];
      if (v <= u) continue;
      eu[e] = (int32_t)u;
      ev[e] = v;
      ew[e] = w[q];
      is_off[e] = !(parent[v] == u || parent[u] == v);
      k += is_off[e];
      e++;
    }
    optr[u + 1] = k;
  }
  for (int64_t u = 0; u < n; u++) optr[u + 1] += optr[u];
  const int64_t E = optr[n];
  int32_t *ou = NULL, *ov = NULL, *oid = NULL, *lca = NULL, *beta = NULL;
  double* ow = NULL;
  item_t* ord = NULL;
  ou = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  ov = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  oid = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  ow = (double*)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1));
  lca = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  beta = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  ord = (item_t*)malloc(sizeof(item_t) * (size_t)(E > 0 ? E : 1));
  if (!ou || !ov || !oid || !ow || !lca || !beta || !ord) {
    st = OMP_E_OOM;
    goto out1;
  }
#pragma omp parallel for
  for (int64_t u = 0; u < n; u++) {
    int64_t o = optr[u];
    for (int64_t e = eptr[u]; e < eptr[u + 1]; e++)
      if (is_off[e]) {
        ou[o] = eu[e];
        ov[o] = ev[e];
        ow[o] = ew[e];
        oid[o] = (int32_t)e;
        o++;
      }
  }
  /* step 1: LCA, exact R_T, score, beta* */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < E; i++) {
    const int32_t u = ou[i], v = ov[i];
    const int32_t l = lca_query(&t, u, v);
    const u128 Rf = (t.D[u] - t.D[l]) + (t.D[v] - t.D[l]);
    const double R = ldexp((double)Rf, -t.S); /* one rounding: the conversion (exact scaling after) */
    ord[i].key = score_mode == 1 ? R : ow[i] * R;
    ord[i].id = oid[i];
    ord[i].off = (int32_t)i;
    lca[i] = l;
    const int32_t hu = t.depth[u] - t.depth[l], hv = t.depth[v] - t.depth[l];
    int32_t b = hu < hv ? hu : hv;
    beta[i] = b > c ? c : b;
  }
  /* step 2: order */
  if ((st = parallel_sort(ord, E, T)) != OMP_OK) goto out1;
  {
    int64_t k = k_override >= 0 ? k_override : (int64_t)floor(alpha * (double)n);
    if (k < 0) k = 0;
    const int64_t cut = cutoff >= 0 ? cutoff : (E / 10 < 100000 ? E / 10 : 100000);
    int64_t P = 2 * k + 1024 < E ? 2 * k + 1024 : E;
    int64_t *task_ptr = NULL, *task_pos = NULL, *cnt = NULL, *tasks = NULL;
    uint8_t *marked = NULL, *recovered = NULL;
    scratch_t* sc = (scratch_t*)calloc((size_t)T, sizeof(scratch_t));
    int64_t taken = 0;
    st = OMP_OK;
    if (!sc) {
      st = OMP_E_OOM;
      goto out2;
    }
    for (int q = 0; q < T; q++) {
      sc[q].su = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
      sc[q].sv = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
      sc[q].q = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
      sc[q].qd = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
      if (!sc[q].su || !sc[q].sv || !sc[q].q || !sc[q].qd) {
        st = OMP_E_OOM;
        goto out2;
      }
      for (int64_t x = 0; x < n; x++) sc[q].su[x] = sc[q].sv[x] = -1;
    }
    cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    task_pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(E > 0 ? E : 1));
    marked = (uint8_t*)malloc((size_t)(E > 0 ? E : 1));
    recovered = (uint8_t*)malloc((size_t)(E > 0 ? E : 1));
    tasks = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!cnt || !task_pos || !marked || !recovered || !tasks) {
      st = OMP_E_OOM;
      goto out2;
    }
    for (;;) {
      /* step 3: subtasks over the prefix -- a counting sort of the positions by LCA (stable: in order) */
      memset(cnt, 0, sizeof(int64_t) * ((size_t)n + 1));
      for (int64_t pos = 0; pos < P; pos++) cnt[lca[ord[pos].off] + 1]++;
      for (int64_t x = 0; x < n; x++) cnt[x + 1] += cnt[x];
      task_ptr = cnt;
      {
        int64_t* fillp = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        if (!fillp) {
          st = OMP_E_OOM;
          goto out2;
        }
        memcpy(fillp, cnt, sizeof(int64_t) * (size_t)n);
        for (int64_t pos = 0; pos < P; pos++) task_pos[fillp[lca[ord[pos].off]]++] = pos;
        free(fillp);
      }
      /* subtasks by size, largest first */
      int64_t ntask = 0;
      for (int64_t x = 0; x < n; x++)
        if (cnt[x + 1] > cnt[x]) tasks[ntask++] = x;
      {
        /* sort tasks by size descending (ties: smaller LCA first) */
        int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ntask > 0 ? ntask : 1) * 2);
        if (!key) {
          st = OMP_E_OOM;
          goto out2;
        }
        for (int64_t i = 0; i < ntask; i++) {
          key[2 * i] = -(cnt[tasks[i] + 1] - cnt[tasks[i]]);
          key[2 * i + 1] = tasks[i];
        }
        qsort(key, (size_t)ntask, 2 * sizeof(int64_t), cmp_pair_i64);
        for (int64_t i = 0; i < ntask; i++) tasks[i] = key[2 * i + 1];
        free(key);
      }
      memset(marked, 0, (size_t)P);
      memset(recovered, 0, (size_t)P);
      const recov_t R = {&t, ou, ov, beta, ord, task_pos, task_ptr, marked, recovered};
      /* step 4: large subtasks one by one with inner parallelism, the rest in parallel */
      int64_t nlarge = 0;
      while (nlarge < ntask && cnt[tasks[nlarge] + 1] - cnt[tasks[nlarge]] >= cut && cut > 0) nlarge++;
      for (int64_t i = 0; i < nlarge && st == OMP_OK; i++) st = run_blocked(&R, tasks[i], sc, T);
      if (st != OMP_OK) goto out2;
#pragma omp parallel for schedule(dynamic, 1)
      for (int64_t i = nlarge; i < ntask; i++) run_serial(&R, tasks[i], &sc[omp_get_thread_num()]);
      /* budget: the first k recovered positions */
      taken = 0;
      for (int64_t pos = 0; pos < P; pos++) taken += recovered[pos];
      if (taken >= k || P >= E) break;
      P = 4 * P < E ? 4 * P : E;
    }
    {
      int64_t o = 0;
      for (int64_t pos = 0; pos < P && o < k; pos++) {
        if (!recovered[pos]) continue;
        if (o < capacity) {
          if (out_ids) out_ids[o] = ord[pos].id;
          if (out_scores) out_scores[o] = ord[pos].key;
        }
        o++;
      }
      *out_count = o;
      st = (o < k) ? OMP_UNDER_BUDGET : OMP_OK;
      if (o > capacity) st = OMP_E_ARG;
    }
  out2:
    if (sc) {
      for (int q = 0; q < T; q++) {
        free(sc[q].su);
        free(sc[q].sv);
        free(sc[q].q);
        free(sc[q].qd);
        free(sc[q].marks);
      }
      free(sc);
    }
    free(cnt);
    free(task_pos);
    free(marked);
    free(recovered);
    free(tasks);
  }
out1:
  free(ou);
  free(ov);
  free(oid);
  free(ow);
  free(lca);
  free(beta);
  free(ord);
out0:
  free(eptr);
  free(is_off);
  free(eu);
  free(ev);
  free(ew);
  free(optr);
  tree_free(&t);
  return st;
}
