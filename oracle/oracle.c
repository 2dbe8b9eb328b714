/*
 * CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, literal implementation of what the RP-Tuning hot path computes:
 *   - RobustPrune, sorted and unsorted (Algorithm 1; unsorted variant in §3,
 *     "RP-Tuning" paragraph),
 *   - RP-Tuning = RobustPrune(p, N_out(p), alpha2, R) for every node (§3),
 *   - the slow-preprocessing construction RobustPrune(p, P \ {p}, alpha, R)
 *     (§2.1, Lemma 2.2),
 *   - GreedySearch (Algorithm 2) from the medoid start vertex (§4.1),
 *   - brute-force exact k nearest neighbours (ground truth for recall, §4),
 *   - alpha-reachability alpha* of a graph (Definition 2.1).
 *
 * Only the test-suite, the package smoke check and the benchmark's CPU
 * baseline leg use this file.  It shares no code, header or constant with the
 * CUDA library and never calls it.
 *
 * Canonical arithmetic (the paper says "Euclidean distance", §4.1; it fixes no
 * precision, so these readings are ours):
 *   - uint8 vectors: d2 is the exact int64 sum of (x_i - y_i)^2; the domination
 *     test alpha * D(p*,p') <= D(p,p') is evaluated exactly as
 *     A*A*d2(p*,p') <= 1e6 * d2(p,p') in int64, alpha = A / 1000.
 *   - float32 vectors: t = (double)x_i - (double)y_i; s = s + t*t in index order,
 *     round-to-nearest binary64, no fused multiply-add (built with
 *     -ffp-contract=off).  Decision: (double)(A*A) * d2a <= 1e6 * d2b, each
 *     product rounded to binary64.
 *   - Squared distances stand in for distances: alpha*D(a,b) <= D(c,e) iff
 *     alpha^2 * d2(a,b) <= d2(c,e) over the reals.
 *   - argmin ties go to the smaller id; candidate sets are deduplicated and p
 *     itself is dropped (Algorithm 1 first step: V <- (V u N_out(p)) \ {p}).
 *   - R = INT32_MAX means "no degree bound" (RP-Tuning passes infinity, §3).
 */
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_U8 1
#define ORC_F32 2
#define ORC_SORTED 0
#define ORC_UNSORTED 1

/* ------------------------------------------------------------------ */
/* distances                                                           */
/* ------------------------------------------------------------------ */

static int64_t d2_u8(const uint8_t *a, const uint8_t *b, int d) {
  int64_t s = 0;
  for (int i = 0; i < d; i++) {
    int64_t t = (int64_t)a[i] - (int64_t)b[i];
    s += t * t;
  }
  return s;
}

static double d2_f32(const float *a, const float *b, int d) {
  double s = 0.0;
  for (int i = 0; i < d; i++) {
    double t = (double)a[i] - (double)b[i];
    s = s + t * t;
  }
  return s;
}

/* d2 between two base points as a double (exact for uint8: < 2^53). */
static double d2_pts(const void *X, int dtype, int d, int64_t a, int64_t b) {
  if (dtype == ORC_U8) {
    const uint8_t *U = (const uint8_t *)X;
    return (double)d2_u8(U + a * d, U + b * d, d);
  }
  const float *F = (const float *)X;
  return d2_f32(F + a * d, F + b * d, d);
}

/* d2 between a free vector q (same dtype as X) and base point b. */
static double d2_vec(const void *X, int dtype, int d, const void *q, int64_t b) {
  if (dtype == ORC_U8)
    return (double)d2_u8((const uint8_t *)q, (const uint8_t *)X + b * d, d);
  return d2_f32((const float *)q, (const float *)X + b * d, d);
}

/* ------------------------------------------------------------------ */
/* a tiny thread pool over independent items                           */
/* ------------------------------------------------------------------ */

typedef void (*item_fn)(void *arg, int64_t item, int tid);
typedef struct {
  atomic_llong next;
  int64_t total;
  item_fn fn;
  void *arg;
} pool_t;
typedef struct {
  pool_t *pool;
  int tid;
} worker_arg;

static void *pool_worker(void *a) {
  worker_arg *w = (worker_arg *)a;
  for (;;) {
    int64_t i = atomic_fetch_add(&w->pool->next, 1);
    if (i >= w->pool->total) break;
    w->pool->fn(w->pool->arg, i, w->tid);
  }
  return NULL;
}

static int resolve_threads(int nthreads) {
  if (nthreads > 0) return nthreads;
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}

static void parallel_for(int64_t total, int nthreads, item_fn fn, void *arg) {
  pool_t pool;
  atomic_init(&pool.next, 0);
  pool.total = total;
  pool.fn = fn;
  pool.arg = arg;
  if (nthreads <= 1 || total <= 1) {
    worker_arg w = {&pool, 0};
    pool_worker(&w);
    return;
  }
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  worker_arg *wa = (worker_arg *)malloc(sizeof(worker_arg) * (size_t)nthreads);
  for (int t = 0; t < nthreads; t++) {
    wa[t].pool = &pool;
    wa[t].tid = t;
    pthread_create(&th[t], NULL, pool_worker, &wa[t]);
  }
  for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  free(th);
  free(wa);
}

int orc_num_threads(int nthreads) { return resolve_threads(nthreads); }

/* ------------------------------------------------------------------ */
/* Algorithm 1, RobustPrune(p, V, alpha, R), written once over an      */
/* abstract distance oracle so that the Euclidean form (vectors) and  */
/* the general-metric form (an explicit distance matrix) share the    */
/* same loop.                                                          */
/* ------------------------------------------------------------------ */

typedef struct {
  /* vector form */
  const void *X;
  int dtype;
  int d;
  int32_t A; /* alpha in milli-units */
  /* matrix form */
  const double *D;
  int64_t n;
  double alpha;
  /* common */
  int64_t p;
} prune_env;

/* key(p, v): D(p, v) as used for the argmin (squared for vectors). */
static double piv_key(const prune_env *e, int64_t v) {
  if (e->D) return e->D[e->p * e->n + v];
  return d2_pts(e->X, e->dtype, e->d, e->p, v);
}

/* Does the newly kept point a remove candidate v?  alpha * D(a, v) <= D(p, v),
   where key_v = D(p, v) as returned by piv_key. */
static int dominates(const prune_env *e, int64_t a, int64_t v, double key_v) {
  if (e->D) return e->alpha * e->D[a * e->n + v] <= key_v;
  if (e->dtype == ORC_U8) {
    const uint8_t *U = (const uint8_t *)e->X;
    int64_t d2a = d2_u8(U + a * e->d, U + v * e->d, e->d);
    int64_t d2b = (int64_t)key_v; /* exact: an integer below 2^53 */
    return (int64_t)e->A * (int64_t)e->A * d2a <= (int64_t)1000000 * d2b;
  }
  const float *F = (const float *)e->X;
  double d2a = d2_f32(F + a * e->d, F + v * e->d, e->d);
  double A2 = (double)((int64_t)e->A * (int64_t)e->A);
  return A2 * d2a <= 1e6 * key_v;
}

typedef struct {
  int32_t id;
  int64_t pos;
} id_pos;

static int by_id_then_pos(const void *a, const void *b) {
  const id_pos *x = (const id_pos *)a, *y = (const id_pos *)b;
  if (x->id != y->id) return (x->id > y->id) - (x->id < y->id);
  return (x->pos > y->pos) - (x->pos < y->pos);
}

static int by_pos(const void *a, const void *b) {
  const id_pos *x = (const id_pos *)a, *y = (const id_pos *)b;
  return (x->pos > y->pos) - (x->pos < y->pos);
}

/*
 * The loop of Algorithm 1.  cand[0..m) is V in stored order (may hold
 * duplicates and p itself); out receives the new N_out(p) in the order points
 * were added.  Returns |N_out(p)|.
 */
static int64_t robust_prune_env(const prune_env *e, const int32_t *cand, int64_t m,
                                int32_t R, int variant, int32_t *out) {
  /* V <- (V u N_out(p)) \ {p}, as a set; first occurrence keeps its place. */
  int32_t *V = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  double *key = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  char *alive = (char *)malloc((size_t)(m > 0 ? m : 1));
  id_pos *ip = (id_pos *)malloc(sizeof(id_pos) * (size_t)(m > 0 ? m : 1));
  int64_t nip = 0, nv = 0;
  for (int64_t j = 0; j < m; j++)
    if ((int64_t)cand[j] != e->p) {
      ip[nip].id = cand[j];
      ip[nip].pos = j;
      nip++;
    }
  qsort(ip, (size_t)nip, sizeof(id_pos), by_id_then_pos);
  int64_t nu = 0;
  for (int64_t j = 0; j < nip; j++)
    if (j == 0 || ip[j].id != ip[j - 1].id) ip[nu++] = ip[j];
  qsort(ip, (size_t)nu, sizeof(id_pos), by_pos);
  for (int64_t j = 0; j < nu; j++) V[nv++] = ip[j].id;
  free(ip);
  for (int64_t j = 0; j < nv; j++) {
    key[j] = piv_key(e, V[j]);
    alive[j] = 1;
  }
  int64_t remaining = nv, kept = 0;
  while (remaining > 0) {
    /* p* <- argmin_{p' in V} D(p, p')  (sorted), or an arbitrary member of V:
       the first one still present in stored order (unsorted). */
    int64_t best = -1;
    for (int64_t j = 0; j < nv; j++) {
      if (!alive[j]) continue;
      if (best < 0) { best = j; if (variant == ORC_UNSORTED) break; continue; }
      if (key[j] < key[best] || (key[j] == key[best] && V[j] < V[best])) best = j;
    }
    int64_t ps = V[best];
    out[kept++] = (int32_t)ps;
    alive[best] = 0;
    remaining--;
    if (kept == (int64_t)R) break;
    for (int64_t j = 0; j < nv; j++) {
      if (!alive[j]) continue;
      if (dominates(e, ps, V[j], key[j])) { alive[j] = 0; remaining--; }
    }
  }
  free(V);
  free(key);
  free(alive);
  return kept;
}

int64_t orc_robust_prune(const void *X, int dtype, int64_t n, int d, int64_t p,
                         const int32_t *cand, int64_t m, int32_t A, int32_t R, int variant,
                         int32_t *out) {
  (void)n;
  prune_env e;
  memset(&e, 0, sizeof e);
  e.X = X; e.dtype = dtype; e.d = d; e.A = A; e.p = p;
  return robust_prune_env(&e, cand, m, R, variant, out);
}

int64_t orc_robust_prune_dmat(const double *D, int64_t n, int64_t p, const int32_t *cand,
                              int64_t m, double alpha, int32_t R, int variant, int32_t *out) {
  prune_env e;
  memset(&e, 0, sizeof e);
  e.D = D; e.n = n; e.alpha = alpha; e.p = p;
  return robust_prune_env(&e, cand, m, R, variant, out);
}

/* ------------------------------------------------------------------ */
/* RP-Tuning over a whole graph (§3), or over a list of nodes          */
/* ------------------------------------------------------------------ */

typedef struct {
  const void *X;
  int dtype, d;
  int64_t n;
  const int64_t *row_ptr;
  const int32_t *col;
  int32_t A, R;
  int variant;
  const int64_t *nodes;
  int32_t *out_cnt;
  int32_t *out_col;
  int64_t cap;
  int slow; /* 1: V = P \ {p} (slow preprocessing) */
  int32_t **scratch;
} tune_job;

static void tune_item(void *arg, int64_t i, int tid) {
  tune_job *J = (tune_job *)arg;
  int64_t p = J->nodes ? J->nodes[i] : i;
  int32_t *tmp = J->scratch[tid];
  int64_t kept;
  if (J->slow) {
    int32_t *all = tmp + J->n; /* second half of the scratch */
    int64_t m = 0;
    for (int64_t v = 0; v < J->n; v++)
      if (v != p) all[m++] = (int32_t)v;
    kept = orc_robust_prune(J->X, J->dtype, J->n, J->d, p, all, m, J->A, J->R, J->variant, tmp);
  } else {
    int64_t a = J->row_ptr[p], b = J->row_ptr[p + 1];
    kept = orc_robust_prune(J->X, J->dtype, J->n, J->d, p, J->col + a, b - a, J->A, J->R,
                            J->variant, tmp);
  }
  if (kept > J->cap) kept = J->cap; /* caller sized cap >= max possible; never hit */
  J->out_cnt[i] = (int32_t)kept;
  memcpy(J->out_col + i * J->cap, tmp, sizeof(int32_t) * (size_t)kept);
}

static int run_tune(tune_job *J, int64_t count, int nthreads, int64_t scratch_len) {
  int T = resolve_threads(nthreads);
  J->scratch = (int32_t **)malloc(sizeof(int32_t *) * (size_t)T);
  for (int t = 0; t < T; t++)
    J->scratch[t] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(scratch_len > 0 ? scratch_len : 1));
  parallel_for(count, T, tune_item, J);
  for (int t = 0; t < T; t++) free(J->scratch[t]);
  free(J->scratch);
  return 0;
}

/* out_cnt[i], out_col[i*cap ..] for node nodes[i] (or i when nodes == NULL). */
int orc_rp_tune(const void *X, int dtype, int64_t n, int d, const int64_t *row_ptr,
                const int32_t *col, int32_t A, int32_t R, int variant, const int64_t *nodes,
                int64_t n_nodes, int nthreads, int32_t *out_cnt, int32_t *out_col, int64_t cap) {
  tune_job J;
  memset(&J, 0, sizeof J);
  J.X = X; J.dtype = dtype; J.d = d; J.n = n; J.row_ptr = row_ptr; J.col = col;
  J.A = A; J.R = R; J.variant = variant; J.nodes = nodes; J.out_cnt = out_cnt;
  J.out_col = out_col; J.cap = cap;
  int64_t maxdeg = 0;
  for (int64_t p = 0; p < n; p++)
    if (row_ptr[p + 1] - row_ptr[p] > maxdeg) maxdeg = row_ptr[p + 1] - row_ptr[p];
  return run_tune(&J, nodes ? n_nodes : n, nthreads, maxdeg);
}

/* Slow preprocessing (§2.1, Lemma 2.2): RobustPrune(p, P \ {p}, alpha, R). */
int orc_slow_base(const void *X, int dtype, int64_t n, int d, int32_t A, int32_t R, int variant,
                  const int64_t *nodes, int64_t n_nodes, int nthreads, int32_t *out_cnt,
                  int32_t *out_col, int64_t cap) {
  tune_job J;
  memset(&J, 0, sizeof J);
  J.X = X; J.dtype = dtype; J.d = d; J.n = n; J.A = A; J.R = R; J.variant = variant;
  J.nodes = nodes; J.out_cnt = out_cnt; J.out_col = out_col; J.cap = cap; J.slow = 1;
  return run_tune(&J, nodes ? n_nodes : n, nthreads, 2 * n);
}

/* ------------------------------------------------------------------ */
/* exact k nearest neighbours, ordered by (d2, id)                     */
/* ------------------------------------------------------------------ */

typedef struct {
  const void *X;
  int dtype, d;
  int64_t n;
  const void *Q;
  const int64_t *qid;
  int k;
  int32_t *out_ids;
  double *out_d2;
} knn_job;

static void knn_item(void *arg, int64_t i, int tid) {
  (void)tid;
  knn_job *J = (knn_job *)arg;
  int32_t *ids = J->out_ids + i * J->k;
  double *dd = J->out_d2 + i * J->k;
  int cnt = 0;
  size_t esz = J->dtype == ORC_U8 ? 1 : 4;
  const void *q = J->qid ? (const char *)J->X + (size_t)J->qid[i] * (size_t)J->d * esz
                         : (const char *)J->Q + (size_t)i * (size_t)J->d * esz;
  int64_t self = J->qid ? J->qid[i] : -1;
  for (int64_t v = 0; v < J->n; v++) {
    if (v == self) continue;
    double x = d2_vec(J->X, J->dtype, J->d, q, v);
    /* keep the k smallest (d2, id) pairs seen so far, in order */
    if (cnt == J->k) {
      if (!(x < dd[cnt - 1])) continue; /* equal d2: larger id loses */
      cnt--;
    }
    int pos = cnt;
    while (pos > 0 && x < dd[pos - 1]) {
      dd[pos] = dd[pos - 1];
      ids[pos] = ids[pos - 1];
      pos--;
    }
    dd[pos] = x;
    ids[pos] = (int32_t)v;
    cnt++;
  }
  for (int j = cnt; j < J->k; j++) {
    ids[j] = -1;
    dd[j] = INFINITY;
  }
}

/* Queries are Q[i] (qid == NULL) or base points qid[i] with themselves excluded. */
int orc_knn(const void *X, int dtype, int64_t n, int d, const void *Q, const int64_t *qid,
            int64_t nq, int k, int nthreads, int32_t *out_ids, double *out_d2) {
  knn_job J = {X, dtype, d, n, Q, qid, k, out_ids, out_d2};
  parallel_for(nq, resolve_threads(nthreads), knn_item, &J);
  return 0;
}

/* ------------------------------------------------------------------ */
/* start vertex: the point nearest to the mean (§4.1 "medoid")         */
/* ------------------------------------------------------------------ */

int64_t orc_medoid(const void *X, int dtype, int64_t n, int d) {
  if (n <= 0) return -1;
  double *mean = (double *)calloc((size_t)d, sizeof(double));
  for (int j = 0; j < d; j++) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++)
      s = s + (dtype == ORC_U8 ? (double)((const uint8_t *)X)[i * d + j]
                               : (double)((const float *)X)[i * d + j]);
    mean[j] = s / (double)n;
  }
  int64_t best = -1;
  double bd = 0.0;
  for (int64_t i = 0; i < n; i++) {
    double s = 0.0;
    for (int j = 0; j < d; j++) {
      double x = dtype == ORC_U8 ? (double)((const uint8_t *)X)[i * d + j]
                                 : (double)((const float *)X)[i * d + j];
      double t = x - mean[j];
      s = s + t * t;
    }
    if (best < 0 || s < bd) { best = i; bd = s; }
  }
  free(mean);
  return best;
}

/* ------------------------------------------------------------------ */
/* Algorithm 2, GreedySearch(s, q, k, L)                               */
/* ------------------------------------------------------------------ */

typedef struct {
  const void *X;
  int dtype, d;
  int64_t n;
  const int64_t *row_ptr;
  const int32_t *col;
  int64_t start;
  const void *Q;
  int L, k;
  int32_t *out_ids;
  double *out_d2;
  int64_t *out_expansions;
  int64_t maxdeg;
  /* per-thread scratch */
  char **seen;
  char **in_list;
  char **visited;
  int64_t **touched;
} search_job;

typedef struct {
  double dist;
  int32_t id;
} entry;

static int entry_cmp(const void *a, const void *b) {
  const entry *x = (const entry *)a, *y = (const entry *)b;
  if (x->dist < y->dist) return -1;
  if (x->dist > y->dist) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

static void search_item(void *arg, int64_t qi, int tid) {
  search_job *J = (search_job *)arg;
  size_t esz = J->dtype == ORC_U8 ? 1 : 4;
  const void *q = (const char *)J->Q + (size_t)qi * (size_t)J->d * esz;
  char *seen = J->seen[tid];
  char *inL = J->in_list[tid];
  char *vis = J->visited[tid];
  int64_t *touched = J->touched[tid]; /* every node marked during this query, once */
  int64_t ntouched = 0;
  entry *Lst = (entry *)malloc(sizeof(entry) * (size_t)(J->L + J->maxdeg + 1));
  int64_t ls = 0, expansions = 0;
  /* L <- {s}, V <- {} */
  Lst[ls].dist = d2_vec(J->X, J->dtype, J->d, q, J->start);
  Lst[ls].id = (int32_t)J->start;
  ls++;
  inL[J->start] = 1;
  seen[J->start] = 1;
  touched[ntouched++] = J->start;
  for (;;) {
    /* p* <- argmin over L \ V of D(p, q); ties to the smaller id */
    int64_t best = -1;
    for (int64_t j = 0; j < ls; j++) {
      if (vis[Lst[j].id]) continue;
      if (best < 0 || entry_cmp(&Lst[j], &Lst[best]) < 0) best = j;
    }
    if (best < 0) break; /* L \ V is empty */
    int32_t ps = Lst[best].id;
    expansions++;
    /* L <- L u N_out(p*), V <- V u {p*} */
    vis[ps] = 1;
    for (int64_t e = J->row_ptr[ps]; e < J->row_ptr[ps + 1]; e++) {
      int32_t v = J->col[e];
      if (inL[v]) continue;
      inL[v] = 1;
      if (!seen[v]) { seen[v] = 1; touched[ntouched++] = v; }
      Lst[ls].dist = d2_vec(J->X, J->dtype, J->d, q, v);
      Lst[ls].id = v;
      ls++;
    }
    /* if |L| > L, keep the L closest to q */
    if (ls > J->L) {
      qsort(Lst, (size_t)ls, sizeof(entry), entry_cmp);
      for (int64_t j = J->L; j < ls; j++) inL[Lst[j].id] = 0;
      ls = J->L;
    }
  }
  qsort(Lst, (size_t)ls, sizeof(entry), entry_cmp);
  for (int j = 0; j < J->k; j++) {
    J->out_ids[qi * J->k + j] = j < ls ? Lst[j].id : -1;
    J->out_d2[qi * J->k + j] = j < ls ? Lst[j].dist : INFINITY;
  }
  if (J->out_expansions) J->out_expansions[qi] = expansions;
  /* reset this thread's marks for the next query */
  for (int64_t j = 0; j < ntouched; j++) {
    seen[touched[j]] = 0;
    inL[touched[j]] = 0;
    vis[touched[j]] = 0;
  }
  free(Lst);
}

int orc_greedy_search(const void *X, int dtype, int64_t n, int d, const int64_t *row_ptr,
                      const int32_t *col, int64_t start, const void *Q, int64_t nq, int L, int k,
                      int nthreads, int32_t *out_ids, double *out_d2, int64_t *out_expansions) {
  if (L < k || k <= 0 || start < 0 || start >= n) return -1;
  int T = resolve_threads(nthreads);
  search_job J;
  memset(&J, 0, sizeof J);
  J.X = X; J.dtype = dtype; J.d = d; J.n = n; J.row_ptr = row_ptr; J.col = col;
  J.start = start; J.Q = Q; J.L = L; J.k = k; J.out_ids = out_ids; J.out_d2 = out_d2;
  J.out_expansions = out_expansions;
  for (int64_t p = 0; p < n; p++)
    if (row_ptr[p + 1] - row_ptr[p] > J.maxdeg) J.maxdeg = row_ptr[p + 1] - row_ptr[p];
  J.seen = (char **)malloc(sizeof(char *) * (size_t)T);
  J.in_list = (char **)malloc(sizeof(char *) * (size_t)T);
  J.visited = (char **)malloc(sizeof(char *) * (size_t)T);
  J.touched = (int64_t **)malloc(sizeof(int64_t *) * (size_t)T);
  for (int t = 0; t < T; t++) {
    J.seen[t] = (char *)calloc((size_t)n, 1);
    J.in_list[t] = (char *)calloc((size_t)n, 1);
    J.visited[t] = (char *)calloc((size_t)n, 1);
    J.touched[t] = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  }
  parallel_for(nq, T, search_item, &J);
  for (int t = 0; t < T; t++) {
    free(J.seen[t]);
    free(J.in_list[t]);
    free(J.visited[t]);
    free(J.touched[t]);
  }
  free(J.seen);
  free(J.in_list);
  free(J.visited);
  free(J.touched);
  return 0;
}

/* ------------------------------------------------------------------ */
/* reachability alpha*(G) (Definition 2.1)                             */
/* ------------------------------------------------------------------ */
/* alpha*(G) = min over ordered pairs (p, q), q != p, (p, q) not an edge, of
   max over p' in N_out(p) of D(p, q) / D(p', q); D(p', q) = 0 makes q reachable
   at every alpha (ratio +inf); a node with no out-neighbour gives ratio 0. */

typedef struct {
  const double *D2; /* n x n squared distances, or NULL */
  const double *Dm; /* n x n distances (general metric), or NULL */
  int64_t n;
  const int64_t *row_ptr;
  const int32_t *col;
  double *per_node;
  /* with neither matrix: distances from the vectors, one pair at a time */
  const void *X;
  int dtype, d;
  const int64_t *nodes; /* item i is node nodes[i] (NULL: node i) */
} reach_job;

static double rj_dist(const reach_job *J, int64_t a, int64_t b) {
  if (J->Dm) return J->Dm[a * J->n + b];
  if (J->D2) return sqrt(J->D2[a * J->n + b]);
  return sqrt(d2_pts(J->X, J->dtype, J->d, a, b));
}

static void reach_item(void *arg, int64_t i, int tid) {
  (void)tid;
  reach_job *J = (reach_job *)arg;
  const int64_t p = J->nodes ? J->nodes[i] : i;
  double worst = INFINITY;
  int64_t a = J->row_ptr[p], b = J->row_ptr[p + 1];
  for (int64_t q = 0; q < J->n; q++) {
    if (q == p) continue;
    int edge = 0;
    for (int64_t e = a; e < b; e++)
      if (J->col[e] == q) { edge = 1; break; }
    if (edge) continue;
    double best = 0.0;
    double dpq = rj_dist(J, p, q);
    for (int64_t e = a; e < b; e++) {
      double dd = rj_dist(J, J->col[e], q);
      double r = dd == 0.0 ? INFINITY : dpq / dd;
      if (r > best) best = r;
    }
    if (best < worst) worst = best;
  }
  J->per_node[i] = worst;
}

static double reach_run(reach_job *J, int nthreads) {
  J->per_node = (double *)malloc(sizeof(double) * (size_t)(J->n > 0 ? J->n : 1));
  parallel_for(J->n, resolve_threads(nthreads), reach_item, J);
  double w = INFINITY;
  for (int64_t p = 0; p < J->n; p++)
    if (J->per_node[p] < w) w = J->per_node[p];
  free(J->per_node);
  return w;
}

double orc_reachability(const void *X, int dtype, int64_t n, int d, const int64_t *row_ptr,
                        const int32_t *col, int nthreads) {
  double *D2 = (double *)malloc(sizeof(double) * (size_t)(n * n > 0 ? n * n : 1));
  for (int64_t a = 0; a < n; a++)
    for (int64_t b = 0; b < n; b++) D2[a * n + b] = d2_pts(X, dtype, d, a, b);
  reach_job J = {D2, NULL, n, row_ptr, col, NULL, NULL, 0, 0, NULL};
  double r = reach_run(&J, nthreads);
  free(D2);
  return r;
}

double orc_reachability_dmat(const double *D, int64_t n, const int64_t *row_ptr,
                             const int32_t *col) {
  reach_job J = {NULL, D, n, row_ptr, col, NULL, NULL, 0, 0, NULL};
  return reach_run(&J, 1);
}

/* Per-node terms of alpha*(G) at the nodes asked for (NULL: every node),
   distances computed pair by pair (no n x n matrix, so any n):
   out[i] = min over q != p, (p, q) not an edge, of max over p' in N_out(p)
   of D(p, q) / D(p', q), p = nodes[i]. */
int orc_reachability_nodes(const void *X, int dtype, int64_t n, int d, const int64_t *row_ptr,
                           const int32_t *col, const int64_t *nodes, int64_t n_nodes, int nthreads,
                           double *out) {
  reach_job J = {NULL, NULL, n, row_ptr, col, out, X, dtype, d, nodes};
  parallel_for(n_nodes, resolve_threads(nthreads), reach_item, &J);
  return 0;
}

/* canonical squared distances for a list of (a, b) base-point pairs */
int orc_d2_pairs(const void *X, int dtype, int d, const int64_t *a, const int64_t *b,
                 int64_t npairs, double *out) {
  for (int64_t i = 0; i < npairs; i++) out[i] = d2_pts(X, dtype, d, a[i], b[i]);
  return 0;
}

/* canonical squared distances from free vectors Q[i] to base points ids[i*k + j] */
int orc_d2_query(const void *X, int dtype, int d, const void *Q, int64_t nq,
                 const int32_t *ids, int k, double *out) {
  size_t esz = dtype == ORC_U8 ? 1 : 4;
  for (int64_t i = 0; i < nq; i++)
    for (int j = 0; j < k; j++) {
      int32_t v = ids[i * k + j];
      out[i * k + j] = v < 0 ? INFINITY
                             : d2_vec(X, dtype, d, (const char *)Q + (size_t)i * d * esz, v);
    }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Vamana, the "fast preprocessing" construction (§2.1; §4.1 builds   */
/* the base indices with it at alpha1 = 1.2, R, L_build = 75), run in */
/* batches.                                                           */
/* ------------------------------------------------------------------ */
/*
 * The paper treats Vamana as a black box and prints no listing of it.  This
 * is its reading of the construction, with the batch schedule fixed so that
 * the result is defined independently of any parallel execution:
 *
 *   The graph starts empty.  Points are inserted in the order perm[], in
 *   batches of 1, 2, 4, ... points, each at most max_batch.  For every point
 *   p of a batch, against the graph as it stood when the batch began:
 *     V_p   = the visited set of GreedySearch(s, x_p, 1, L) (Algorithm 2), in
 *             expansion order, its first vcap members (vcap bounds memory);
 *     N'(p) = RobustPrune(p, V_p, alpha, R) (Algorithm 1, sorted; its first
 *             step takes the union with the current N_out(p) and drops p).
 *   Then every N_out(p) <- N'(p).  Then the back edges: for every j named in
 *   some N'(p), P_j = the batch points naming j, ascending by id, its first
 *   512 members (VAMANA_MAX_SENDERS: this bounds every candidate list a
 *   hub point gets); the merged list is N_out(j) followed by the members of
 *   P_j not already in it; if it
 *   holds at most R points it becomes N_out(j), otherwise
 *   N_out(j) <- RobustPrune(j, merged, alpha, R).
 * A pass inserts every point once; pass i uses alpha = A[i] / 1000 (the
 * original construction runs alpha = 1 and then alpha1).  s is the start
 * vertex.  The graph is held as nbr[p * R + 0 .. deg[p]).
 */

typedef struct {
  const void *X;
  int dtype, d;
  int64_t n;
  const int32_t *nbr, *deg; /* the graph at the batch's start */
  int32_t R, L, vcap;
  int64_t start;
  int32_t A;
  const int32_t *batch;
  int32_t *new_nbr, *new_deg; /* per batch point: R slots */
  int64_t *visited_over;      /* searches whose visited set was cut to vcap */
  char **inL, **vis, **seen;
  int64_t **touched;
  int32_t **scratch;
} vamana_job;

/* GreedySearch(s, x_p, 1, L) on (nbr, deg), recording the expanded points in
   order; returns how many were expanded, writing the first vcap into out. */
static int64_t vamana_visit(const vamana_job *J, int64_t p, int tid, int32_t *out) {
  size_t esz = J->dtype == ORC_U8 ? 1 : 4;
  const void *q = (const char *)J->X + (size_t)p * (size_t)J->d * esz;
  char *inL = J->inL[tid], *vis = J->vis[tid], *seen = J->seen[tid];
  int64_t *touched = J->touched[tid]; /* every point marked during this search, once */
  int64_t ntouched = 0, ls = 0, expansions = 0;
  entry *Lst = (entry *)malloc(sizeof(entry) * (size_t)(J->L + J->R + 1));
  Lst[ls].dist = d2_vec(J->X, J->dtype, J->d, q, J->start);
  Lst[ls].id = (int32_t)J->start;
  ls++;
  inL[J->start] = 1;
  seen[J->start] = 1;
  touched[ntouched++] = J->start;
  for (;;) {
    int64_t best = -1;
    for (int64_t j = 0; j < ls; j++) {
      if (vis[Lst[j].id]) continue;
      if (best < 0 || entry_cmp(&Lst[j], &Lst[best]) < 0) best = j;
    }
    if (best < 0) break;
    int32_t ps = Lst[best].id;
    if (expansions < J->vcap) out[expansions] = ps;
    expansions++;
    vis[ps] = 1;
    for (int32_t e = 0; e < J->deg[ps]; e++) {
      int32_t v = J->nbr[(int64_t)ps * J->R + e];
      if (inL[v]) continue;
      inL[v] = 1;
      if (!seen[v]) { seen[v] = 1; touched[ntouched++] = v; }
      Lst[ls].dist = d2_vec(J->X, J->dtype, J->d, q, v);
      Lst[ls].id = v;
      ls++;
    }
    if (ls > J->L) {
      qsort(Lst, (size_t)ls, sizeof(entry), entry_cmp);
      for (int64_t j = J->L; j < ls; j++) inL[Lst[j].id] = 0;
      ls = J->L;
    }
  }
  for (int64_t j = 0; j < ntouched; j++) {
    inL[touched[j]] = 0;
    vis[touched[j]] = 0;
    seen[touched[j]] = 0;
  }
  free(Lst);
  return expansions;
}

static void vamana_item(void *arg, int64_t i, int tid) {
  vamana_job *J = (vamana_job *)arg;
  int64_t p = J->batch[i];
  int32_t *cand = J->scratch[tid];
  int64_t nv = vamana_visit(J, p, tid, cand);
  if (nv > J->vcap) {
    __atomic_fetch_add(J->visited_over, 1, __ATOMIC_RELAXED);
    nv = J->vcap;
  }
  /* V_p, then the current N_out(p); Algorithm 1 takes the union and drops p */
  for (int32_t e = 0; e < J->deg[p]; e++) cand[nv++] = J->nbr[p * J->R + e];
  prune_env E;
  memset(&E, 0, sizeof E);
  E.X = J->X; E.dtype = J->dtype; E.d = J->d; E.A = J->A; E.p = p;
  J->new_deg[i] = (int32_t)robust_prune_env(&E, cand, nv, J->R, ORC_SORTED, J->new_nbr + i * J->R);
}

typedef struct {
  int32_t j, p;
} back_edge;

static int back_edge_cmp(const void *a, const void *b) {
  const back_edge *x = (const back_edge *)a, *y = (const back_edge *)b;
  if (x->j != y->j) return (x->j > y->j) - (x->j < y->j);
  return (x->p > y->p) - (x->p < y->p);
}

#define VAMANA_MAX_SENDERS 512

/* Batch sizes: 1, 2, 4, ... capped at max_batch; the last batch takes the rest. */
static int64_t vamana_batch_size(int64_t k, int64_t max_batch) {
  int64_t b = 1;
  for (int64_t i = 0; i < k && b < max_batch; i++) b *= 2;
  return b < max_batch ? b : max_batch;
}

int orc_vamana(const void *X, int dtype, int64_t n, int d, const int32_t *perm, int npass,
               const int32_t *A, int32_t R, int32_t L, int32_t vcap, int64_t max_batch, int64_t start,
               int nthreads, int32_t *nbr /* n * R */, int32_t *deg /* n */, int64_t *visited_over) {
  if (n < 1 || R < 1 || L < 1 || vcap < 1 || max_batch < 1 || start < 0 || start >= n) return -1;
  int T = resolve_threads(nthreads);
  vamana_job J;
  memset(&J, 0, sizeof J);
  J.X = X; J.dtype = dtype; J.d = d; J.n = n; J.R = R; J.L = L; J.vcap = vcap; J.start = start;
  J.nbr = nbr; J.deg = deg;
  int64_t over = 0;
  J.visited_over = &over;
  memset(deg, 0, sizeof(int32_t) * (size_t)n);
  int32_t *new_nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)max_batch * (size_t)R);
  int32_t *new_deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)max_batch);
  back_edge *be = (back_edge *)malloc(sizeof(back_edge) * (size_t)max_batch * (size_t)R);
  int32_t *merged = (int32_t *)malloc(sizeof(int32_t) * (size_t)(R + max_batch));
  int32_t *kept = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
  J.new_nbr = new_nbr; J.new_deg = new_deg;
  J.inL = (char **)malloc(sizeof(char *) * (size_t)T);
  J.vis = (char **)malloc(sizeof(char *) * (size_t)T);
  J.seen = (char **)malloc(sizeof(char *) * (size_t)T);
  J.touched = (int64_t **)malloc(sizeof(int64_t *) * (size_t)T);
  J.scratch = (int32_t **)malloc(sizeof(int32_t *) * (size_t)T);
  for (int t = 0; t < T; t++) {
    J.inL[t] = (char *)calloc((size_t)n, 1);
    J.vis[t] = (char *)calloc((size_t)n, 1);
    J.seen[t] = (char *)calloc((size_t)n, 1);
    J.touched[t] = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    J.scratch[t] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(vcap + R));
  }
  for (int pass = 0; pass < npass; pass++) {
    J.A = A[pass];
    int64_t b0 = 0;
    for (int64_t k = 0; b0 < n; k++) {
      int64_t bsz = vamana_batch_size(k, max_batch);
      if (bsz > n - b0) bsz = n - b0;
      J.batch = perm + b0;
      parallel_for(bsz, T, vamana_item, &J);
      int64_t nbe = 0;
      for (int64_t i = 0; i < bsz; i++) {
        int64_t p = perm[b0 + i];
        memcpy(nbr + p * R, new_nbr + i * R, sizeof(int32_t) * (size_t)new_deg[i]);
        deg[p] = new_deg[i];
        for (int32_t e = 0; e < new_deg[i]; e++) {
          be[nbe].j = new_nbr[i * R + e];
          be[nbe].p = (int32_t)p;
          nbe++;
        }
      }
      qsort(be, (size_t)nbe, sizeof(back_edge), back_edge_cmp);
      for (int64_t g0 = 0; g0 < nbe;) {
        int64_t g1 = g0;
        while (g1 < nbe && be[g1].j == be[g0].j) g1++;
        int64_t j = be[g0].j, m = 0;
        for (int32_t e = 0; e < deg[j]; e++) merged[m++] = nbr[j * R + e];
        int64_t have = m;
        /* at most VAMANA_MAX_SENDERS back edges per batch: the smallest sender ids */
        int64_t gl = g1 - g0 > VAMANA_MAX_SENDERS ? g0 + VAMANA_MAX_SENDERS : g1;
        for (int64_t g = g0; g < gl; g++) {
          int dup = 0;
          for (int64_t e = 0; e < have; e++)
            if (merged[e] == be[g].p) { dup = 1; break; }
          if (!dup) merged[m++] = be[g].p;
        }
        if (m <= R) {
          memcpy(nbr + j * R, merged, sizeof(int32_t) * (size_t)m);
          deg[j] = (int32_t)m;
        } else {
          prune_env E;
          memset(&E, 0, sizeof E);
          E.X = X; E.dtype = dtype; E.d = d; E.A = A[pass]; E.p = j;
          int64_t c = robust_prune_env(&E, merged, m, R, ORC_SORTED, kept);
          memcpy(nbr + j * R, kept, sizeof(int32_t) * (size_t)c);
          deg[j] = (int32_t)c;
        }
        g0 = g1;
      }
      b0 += bsz;
    }
  }
  for (int t = 0; t < T; t++) {
    free(J.inL[t]);
    free(J.vis[t]);
    free(J.seen[t]);
    free(J.touched[t]);
    free(J.scratch[t]);
  }
  free(J.inL); free(J.vis); free(J.seen); free(J.touched); free(J.scratch);
  free(new_nbr); free(new_deg); free(be); free(merged); free(kept);
  if (visited_over) *visited_over = over;
  return 0;
}
