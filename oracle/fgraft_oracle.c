/*
 * fgraft_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow CPU restatement of the FGraft builder of "Batched Feedback and
 * the Random-Access Wall in Search-Based Graph Construction" (Section 3,
 * "Batched feedback", and Proposition 1), written from the paper's text.  It
 * exists so that the tests, the smoke check and the CPU-baseline leg of the
 * benchmark can check the CUDA library against an independent program.  It
 * shares no code, header, table or constant generator with the CUDA path, and
 * the product library never links or calls it.
 *
 * Every step is the algorithm as the paper states it, in the paper's order,
 * with sets held as sorted arrays, qsort for ordering and byte arrays for
 * visited sets.  Points where the paper is silent follow the readings listed
 * beside each function (they are the same readings the CUDA path implements,
 * written down independently).
 *
 * Compile with -ffp-contract=off: the canonical distance is defined operation
 * by operation (fmaf where an FMA is meant, separate rounding elsewhere).
 *
 * Metric codes: 0 = squared L2 on float32, 1 = angular on unit float32
 * vectors (1 - <x,y>), 2 = squared L2 on uint8 (exact integer arithmetic).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FGO_L2_F32 0
#define FGO_ANGULAR_F32 1
#define FGO_L2_U8 2

typedef struct {
  const void* X;   /* n rows, row stride ld elements */
  int64_t n;
  int32_t d;
  int64_t ld;
  int32_t metric;
} fgo_data;

typedef struct {
  uint64_t sat_evals;
  uint64_t harvest_evals;
  uint64_t prune_evals;
  uint64_t final_prune_evals;
  uint64_t expansions;
} fgo_counters;

typedef struct {
  float d;
  int32_t id;
  int32_t expanded;
} ent;

static int ent_cmp(const void* a, const void* b) {
  const ent* x = (const ent*)a;
  const ent* y = (const ent*)b;
  if (x->d < y->d) return -1;
  if (x->d > y->d) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

static int i32_cmp(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static const void* row_ptr(const fgo_data* D, int64_t i) {
  if (D->metric == FGO_L2_U8) return (const uint8_t*)D->X + i * D->ld;
  return (const float*)D->X + i * D->ld;
}

/* ------------------------------------------------------------------------ *
 * Canonical distance.
 *
 * The paper uses Euclidean distance on float32 vectors, angular data being
 * L2-normalised so that all systems solve a Euclidean problem (Section 2,
 * "Systems").  A bit-exact comparison needs one summation order; this is the
 * fixed order (the reading the whole build uses):
 *   32 virtual lanes; lane l owns elements j = 128k + 4l + c (k = 0,1,..;
 *   c = 0..3) in that order, each accumulating acc = fmaf(t, t, acc) with
 *   t = x_j - y_j rounded to float first (acc = fmaf(x_j, y_j, acc) for the
 *   angular inner product), starting from +0.0f; then the lane partials are
 *   combined pairwise: p[l] += p[l+16], then +8, +4, +2, +1.
 * Angular: delta = 1.0f - dot.  uint8: exact sum of squared differences.
 * ------------------------------------------------------------------------ */
static float canon_f32(const float* x, const float* y, int d, int angular) {
  float p[32];
  for (int l = 0; l < 32; ++l) {
    float acc = 0.0f;
    for (int k = 0; 128 * k < d; ++k) {
      for (int c = 0; c < 4; ++c) {
        int j = 128 * k + 4 * l + c;
        if (j >= d) continue;
        if (angular) {
          acc = fmaf(x[j], y[j], acc);
        } else {
          float t = x[j] - y[j];
          acc = fmaf(t, t, acc);
        }
      }
    }
    p[l] = acc;
  }
  for (int s = 16; s >= 1; s >>= 1)
    for (int l = 0; l < s; ++l) p[l] = p[l] + p[l + s];
  if (angular) return 1.0f - p[0];
  return p[0];
}

static float canon_u8(const uint8_t* x, const uint8_t* y, int d) {
  int32_t s = 0;
  for (int j = 0; j < d; ++j) {
    int32_t t = (int32_t)x[j] - (int32_t)y[j];
    s += t * t;
  }
  return (float)s; /* exact: s < 2^24 for d <= 256 */
}

static float dist_ptr(const fgo_data* D, const void* x, const void* y) {
  if (D->metric == FGO_L2_U8) return canon_u8((const uint8_t*)x, (const uint8_t*)y, D->d);
  return canon_f32((const float*)x, (const float*)y, D->d, D->metric == FGO_ANGULAR_F32);
}

static float dist_ij(const fgo_data* D, int64_t i, int64_t j) {
  return dist_ptr(D, row_ptr(D, i), row_ptr(D, j));
}

float fgo_dist(const fgo_data* D, int64_t i, int64_t j) { return dist_ij(D, i, j); }

/* distance from a free vector q (same element type and layout as a row of X) */
float fgo_dist_vec(const fgo_data* D, const void* q, int64_t j) {
  return dist_ptr(D, q, row_ptr(D, j));
}

/* The same quantity in double precision (reference for error bounds). */
double fgo_dist_f64(const fgo_data* D, int64_t i, int64_t j) {
  double s = 0.0;
  if (D->metric == FGO_L2_U8) {
    const uint8_t* x = (const uint8_t*)row_ptr(D, i);
    const uint8_t* y = (const uint8_t*)row_ptr(D, j);
    for (int k = 0; k < D->d; ++k) {
      double t = (double)x[k] - (double)y[k];
      s += t * t;
    }
    return s;
  }
  const float* x = (const float*)row_ptr(D, i);
  const float* y = (const float*)row_ptr(D, j);
  if (D->metric == FGO_ANGULAR_F32) {
    for (int k = 0; k < D->d; ++k) s += (double)x[k] * (double)y[k];
    return 1.0 - s;
  }
  for (int k = 0; k < D->d; ++k) {
    double t = (double)x[k] - (double)y[k];
    s += t * t;
  }
  return s;
}

/* ------------------------------------------------------------------------ *
 * Keyed roots.  The paper fixes only that randomness is keyed (Proposition 1)
 * and that the beam enters at the tree roots (Section 3).  Reading: root t is
 * splitmix64(seed ^ (G * (t+1)) + j) mod n for the smallest j >= 0 that gives
 * a root distinct from roots 0..t-1; G = 0x9E3779B97F4A7C15 and splitmix64(z)
 * is the first output of the SplitMix64 generator (Steele, Lea and Flood,
 * OOPSLA 2014) started at state z.
 * ------------------------------------------------------------------------ */
uint64_t fgo_splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

int fgo_roots(uint64_t seed, int32_t T, int64_t n, int32_t* roots) {
  if (T < 1 || n < T) return 1;
  for (int t = 0; t < T; ++t) {
    uint64_t base = seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(t + 1));
    for (uint64_t j = 0;; ++j) {
      int32_t r = (int32_t)(fgo_splitmix64(base + j) % (uint64_t)n);
      int dup = 0;
      for (int s = 0; s < t; ++s) dup |= (roots[s] == r);
      if (!dup) {
        roots[t] = r;
        break;
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ *
 * Spatial approximation tree (Navarro 2002, cited in Section 1 for the
 * scaffold).  For a node a holding the point set P (a excluded):
 *   sort P by (delta(x,a), id);
 *   scan it: x becomes a child of a iff delta(x,a) < delta(x,b) for every
 *   child b already chosen (strict, so a tie keeps x out);
 *   every other y goes to the child b minimising (delta(y,b), id_b);
 *   recurse into each child with the points assigned to it.
 * Work counted per node (a reading; the paper only says that every evaluation
 * is counted): m + k(k-1)/2 + (m-k)k, m = |P|, k = number of children.
 * parent[root] = -1.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t a;
  int64_t start, len;
} sat_node;

int fgo_sat_tree(const fgo_data* D, int32_t root, int32_t* parent, uint64_t* evals_out) {
  const int64_t n = D->n;
  int32_t* W = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 1 ? n - 1 : 1));
  int32_t* W2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 1 ? n - 1 : 1));
  ent* L = (ent*)malloc(sizeof(ent) * (size_t)(n > 1 ? n : 1));
  int32_t* members = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 1 ? n : 1));
  int32_t* owner = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 1 ? n : 1));
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 1 ? n : 1));
  sat_node* stack = (sat_node*)malloc(sizeof(sat_node) * (size_t)(n > 1 ? n : 1));
  if (!W || !W2 || !L || !members || !owner || !cnt || !stack) return 2;
  uint64_t evals = 0;
  for (int64_t i = 0; i < n; ++i) parent[i] = -1;
  int64_t w = 0;
  for (int64_t i = 0; i < n; ++i)
    if (i != root) W[w++] = (int32_t)i;
  int64_t sp = 0;
  stack[sp++] = (sat_node){root, 0, n - 1};
  while (sp > 0) {
    sat_node nd = stack[--sp];
    const int64_t m = nd.len;
    if (m == 0) continue;
    const void* xa = row_ptr(D, nd.a);
    for (int64_t i = 0; i < m; ++i) {
      int32_t x = W[nd.start + i];
      L[i].d = dist_ptr(D, row_ptr(D, x), xa);
      L[i].id = x;
      L[i].expanded = 0;
    }
    qsort(L, (size_t)m, sizeof(ent), ent_cmp);
    int64_t k = 0;
    for (int64_t i = 0; i < m; ++i) {
      int joins = 1;
      for (int64_t bi = 0; bi < k && joins; ++bi) {
        float dxb = dist_ij(D, L[i].id, members[bi]);
        if (!(L[i].d < dxb)) joins = 0;
      }
      if (joins) {
        members[k++] = L[i].id;
        L[i].expanded = 1; /* marks membership */
      }
    }
    /* assignment of non-members to their closest child */
    for (int64_t bi = 0; bi < k; ++bi) cnt[bi] = 0;
    for (int64_t i = 0; i < m; ++i) {
      if (L[i].expanded) {
        owner[i] = -1;
        continue;
      }
      int64_t best = 0;
      float bestd = dist_ij(D, L[i].id, members[0]);
      for (int64_t bi = 1; bi < k; ++bi) {
        float dd = dist_ij(D, L[i].id, members[bi]);
        if (dd < bestd || (dd == bestd && members[bi] < members[best])) {
          best = bi;
          bestd = dd;
        }
      }
      owner[i] = (int32_t)best;
      cnt[best]++;
    }
    evals += (uint64_t)m + (uint64_t)(k * (k - 1) / 2) + (uint64_t)((m - k) * k);
    /* lay out: [b_0, set(b_0)..., b_1, set(b_1)..., ...] */
    int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    int64_t acc = 0;
    for (int64_t bi = 0; bi < k; ++bi) {
      pos[bi] = acc + 1;
      W2[nd.start + acc] = members[bi];
      acc += 1 + cnt[bi];
    }
    for (int64_t i = 0; i < m; ++i)
      if (owner[i] >= 0) W2[nd.start + pos[owner[i]]++] = L[i].id;
    memcpy(W + nd.start, W2 + nd.start, sizeof(int32_t) * (size_t)m);
    acc = 0;
    for (int64_t bi = 0; bi < k; ++bi) {
      parent[members[bi]] = nd.a;
      stack[sp++] = (sat_node){members[bi], nd.start + acc + 1, cnt[bi]};
      acc += 1 + cnt[bi];
    }
    free(pos);
  }
  free(W);
  free(W2);
  free(L);
  free(members);
  free(owner);
  free(cnt);
  free(stack);
  if (evals_out) *evals_out = evals;
  return 0;
}

/* T trees that differ only by their keyed root (Section 1; Section 3). */
int fgo_sat_forest(const fgo_data* D, int32_t T, uint64_t seed, int32_t* roots,
                   int32_t* parents /* T*n */, uint64_t* sat_evals) {
  if (fgo_roots(seed, T, D->n, roots)) return 1;
  uint64_t* ev = (uint64_t*)calloc((size_t)T, sizeof(uint64_t));
  int err = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : err)
  for (int t = 0; t < T; ++t) err |= fgo_sat_tree(D, roots[t], parents + (int64_t)t * D->n, &ev[t]);
  uint64_t s = 0;
  for (int t = 0; t < T; ++t) s += ev[t];
  free(ev);
  if (sat_evals) *sat_evals = s;
  return err;
}

/* ------------------------------------------------------------------------ *
 * Scaffold S_0: the union of the T trees' edges, symmetrised (Section 3).
 * Rows are sorted by id and free of duplicates.  Two calls: the first with
 * ids == NULL returns the number of entries in *nnz.
 * ------------------------------------------------------------------------ */
int fgo_scaffold(int64_t n, int32_t T, const int32_t* parents, int64_t* off, int32_t* ids,
                 int64_t* nnz) {
  int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  for (int t = 0; t < T; ++t)
    for (int64_t x = 0; x < n; ++x) {
      int32_t p = parents[(int64_t)t * n + x];
      if (p >= 0) {
        deg[x]++;
        deg[p]++;
      }
    }
  int64_t* o = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  o[0] = 0;
  for (int64_t x = 0; x < n; ++x) o[x + 1] = o[x] + deg[x];
  int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(o[n] > 0 ? o[n] : 1));
  int64_t* fill = (int64_t*)calloc((size_t)n, sizeof(int64_t));
  for (int t = 0; t < T; ++t)
    for (int64_t x = 0; x < n; ++x) {
      int32_t p = parents[(int64_t)t * n + x];
      if (p >= 0) {
        tmp[o[x] + fill[x]++] = p;
        tmp[o[p] + fill[p]++] = (int32_t)x;
      }
    }
  int64_t total = 0;
  for (int64_t x = 0; x < n; ++x) {
    int32_t* r = tmp + o[x];
    int64_t len = o[x + 1] - o[x];
    qsort(r, (size_t)len, sizeof(int32_t), i32_cmp);
    int64_t u = 0;
    for (int64_t i = 0; i < len; ++i)
      if (i == 0 || r[i] != r[i - 1]) r[u++] = r[i];
    if (off) off[x] = total;
    if (ids) memcpy(ids + total, r, sizeof(int32_t) * (size_t)u);
    total += u;
  }
  if (off) off[n] = total;
  if (nnz) *nnz = total;
  free(deg);
  free(o);
  free(tmp);
  free(fill);
  return 0;
}

/* ------------------------------------------------------------------------ *
 * Scaffold degree cap (Section 6, an ablation the paper reports as negative):
 * every row of S_0 longer than K keeps its K nearest entries by
 * (delta(u, v), v); rows stay sorted by id.  Two calls as for fgo_scaffold.
 * ------------------------------------------------------------------------ */
int fgo_scaffold_cap(const fgo_data* D, const int64_t* off, const int32_t* ids, int32_t K,
                     int64_t* out_off, int32_t* out_ids, int64_t* nnz) {
  int64_t total = 0, maxlen = 0;
  for (int64_t u = 0; u < D->n; ++u)
    if (off[u + 1] - off[u] > maxlen) maxlen = off[u + 1] - off[u];
  ent* e = (ent*)malloc(sizeof(ent) * (size_t)(maxlen > 0 ? maxlen : 1));
  int32_t* keep = (int32_t*)malloc(sizeof(int32_t) * (size_t)(maxlen > 0 ? maxlen : 1));
  for (int64_t u = 0; u < D->n; ++u) {
    const int64_t len = off[u + 1] - off[u];
    int64_t m = len;
    if (len > K) {
      for (int64_t i = 0; i < len; ++i) {
        e[i].id = ids[off[u] + i];
        e[i].d = dist_ptr(D, row_ptr(D, u), row_ptr(D, e[i].id));
        e[i].expanded = 0;
      }
      qsort(e, (size_t)len, sizeof(ent), ent_cmp);
      m = K;
      for (int64_t i = 0; i < m; ++i) keep[i] = e[i].id;
      qsort(keep, (size_t)m, sizeof(int32_t), i32_cmp);
    } else {
      for (int64_t i = 0; i < m; ++i) keep[i] = ids[off[u] + i];
    }
    if (out_off) out_off[u] = total;
    if (out_ids) memcpy(out_ids + total, keep, sizeof(int32_t) * (size_t)m);
    total += m;
  }
  if (out_off) out_off[D->n] = total;
  if (nnz) *nnz = total;
  free(e);
  free(keep);
  return 0;
}

/* ------------------------------------------------------------------------ *
 * Beam search (Section 3: "beam search of width ef_h from the tree roots").
 * visited = {}, pool = {}; each root not yet visited is evaluated, marked and
 * put in the pool; then, while the pool holds an unexpanded entry, the one
 * smallest in (delta, id) is expanded: it is appended to E, every neighbour
 * not yet visited is evaluated and marked, and the pool becomes the ef
 * smallest (delta, id) of the pool and the new entries, expanded marks kept.
 * The query point itself gets no special treatment here.  Every evaluation
 * counts, the roots included.
 * Scratch (per thread): visited[n] zeroed, vlist[n], pool[ef + maxdeg].
 * Returns the number of expansions; E_ids/E_d (capacity n) get the expanded
 * vertices in expansion order; pool_out (capacity ef) the final pool.
 * ------------------------------------------------------------------------ */
typedef struct {
  uint8_t* visited;
  int32_t* vlist;
  ent* pool;
  int64_t pool_cap;
} beam_scratch;

static int64_t beam_run(const fgo_data* D, const int64_t* off, const int32_t* ids,
                        const int32_t* roots, int T, const void* q, int ef, beam_scratch* S,
                        int32_t* E_ids, float* E_d, int64_t* n_eval, int64_t* pool_len) {
  int64_t nv = 0, np = 0, ne = 0;
  for (int t = 0; t < T; ++t) {
    int32_t r = roots[t];
    if (S->visited[r]) continue;
    S->visited[r] = 1;
    S->vlist[nv++] = r;
    S->pool[np].d = dist_ptr(D, q, row_ptr(D, r));
    S->pool[np].id = r;
    S->pool[np].expanded = 0;
    np++;
  }
  qsort(S->pool, (size_t)np, sizeof(ent), ent_cmp);
  if (np > ef) np = ef;
  for (;;) {
    int64_t ci = -1;
    for (int64_t i = 0; i < np; ++i)
      if (!S->pool[i].expanded) {
        ci = i;
        break;
      }
    if (ci < 0) break;
    S->pool[ci].expanded = 1;
    int32_t c = S->pool[ci].id;
    E_ids[ne] = c;
    E_d[ne] = S->pool[ci].d;
    ne++;
    int64_t add = np;
    for (int64_t e = off[c]; e < off[c + 1]; ++e) {
      int32_t v = ids[e];
      if (S->visited[v]) continue;
      S->visited[v] = 1;
      S->vlist[nv++] = v;
      S->pool[add].d = dist_ptr(D, q, row_ptr(D, v));
      S->pool[add].id = v;
      S->pool[add].expanded = 0;
      add++;
    }
    qsort(S->pool, (size_t)add, sizeof(ent), ent_cmp);
    np = add < ef ? add : ef;
  }
  for (int64_t i = 0; i < nv; ++i) S->visited[S->vlist[i]] = 0;
  *n_eval = nv;
  *pool_len = np;
  return ne;
}

static int64_t csr_maxdeg(int64_t n, const int64_t* off) {
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i)
    if (off[i + 1] - off[i] > m) m = off[i + 1] - off[i];
  return m;
}

/* One beam search over a CSR graph (exposed for the tests). */
int fgo_beam(const fgo_data* D, const int64_t* off, const int32_t* ids, const int32_t* roots,
             int32_t T, const void* q, int32_t ef, int32_t* E_ids, float* E_d, int64_t* n_exp,
             int32_t* pool_ids, float* pool_d, int64_t* pool_len, int64_t* n_eval) {
  beam_scratch S;
  int64_t maxdeg = csr_maxdeg(D->n, off);
  S.visited = (uint8_t*)calloc((size_t)D->n, 1);
  S.vlist = (int32_t*)malloc(sizeof(int32_t) * (size_t)D->n);
  S.pool_cap = ef + maxdeg + T;
  S.pool = (ent*)malloc(sizeof(ent) * (size_t)S.pool_cap);
  int64_t pl = 0;
  *n_exp = beam_run(D, off, ids, roots, T, q, ef, &S, E_ids, E_d, n_eval, &pl);
  for (int64_t i = 0; i < pl; ++i) {
    pool_ids[i] = S.pool[i].id;
    pool_d[i] = S.pool[i].d;
  }
  *pool_len = pl;
  free(S.visited);
  free(S.vlist);
  free(S.pool);
  return 0;
}

/* The visited set V of one beam search, in visiting order (Section 5.5 and
 * Table 6 measure how much the V of queries searched together overlap). */
int fgo_visited(const fgo_data* D, const int64_t* off, const int32_t* ids, const int32_t* roots,
                int32_t T, const void* q, int32_t ef, int32_t* out_ids, int64_t* out_n) {
  beam_scratch S;
  int64_t maxdeg = csr_maxdeg(D->n, off);
  S.visited = (uint8_t*)calloc((size_t)D->n, 1);
  S.vlist = (int32_t*)malloc(sizeof(int32_t) * (size_t)D->n);
  S.pool_cap = ef + maxdeg + T;
  S.pool = (ent*)malloc(sizeof(ent) * (size_t)S.pool_cap);
  int32_t* E_ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)D->n);
  float* E_d = (float*)malloc(sizeof(float) * (size_t)D->n);
  int64_t nev = 0, pl = 0;
  beam_run(D, off, ids, roots, T, q, ef, &S, E_ids, E_d, &nev, &pl);
  for (int64_t i = 0; i < nev; ++i) out_ids[i] = S.vlist[i];
  *out_n = nev;
  free(S.visited);
  free(S.vlist);
  free(S.pool);
  free(E_ids);
  free(E_d);
  return 0;
}

/* ------------------------------------------------------------------------ *
 * Occlusion prune (Section 3, after FANNG and DiskANN's RobustPrune).
 * Input: candidates of point p with their delta(p, .), p already removed.
 * They are sorted by (delta, id); the first alive one c* is kept and every
 * alive c after it with fl(alpha2 * delta(c*, c)) <= delta(p, c) is removed,
 * alpha2 = fl(alpha * alpha) (alpha acts on the unsquared distance); this
 * repeats until R are kept or none is alive.  No refill.  The removal pass is
 * not run after the R-th keep.  Work counted: one evaluation per alive
 * candidate examined in a removal pass.
 * ------------------------------------------------------------------------ */
static int32_t prune_sorted(const fgo_data* D, const ent* C, int64_t m, float alpha, int32_t R,
                            int32_t* out, uint8_t* alive, uint64_t* evals) {
  const float a2 = alpha * alpha;
  int32_t kept = 0;
  uint64_t ev = 0;
  for (int64_t i = 0; i < m; ++i) alive[i] = 1;
  for (int64_t i = 0; i < m && kept < R; ++i) {
    if (!alive[i]) continue;
    out[kept++] = C[i].id;
    alive[i] = 0;
    if (kept == R) break;
    for (int64_t j = i + 1; j < m; ++j) {
      if (!alive[j]) continue;
      ev++;
      float dd = dist_ij(D, C[i].id, C[j].id);
      float lhs = a2 * dd;
      if (lhs <= C[j].d) alive[j] = 0;
    }
  }
  *evals += ev;
  return kept;
}

/* Prune one explicit candidate list of point p (exposed for the tests).
 * Candidates equal to p and repeated ids are dropped first. */
int32_t fgo_prune_list(const fgo_data* D, int32_t p, const int32_t* cand, int64_t m, float alpha,
                       int32_t R, int32_t* out, uint64_t* evals) {
  ent* C = (ent*)malloc(sizeof(ent) * (size_t)(m > 0 ? m : 1));
  uint8_t* alive = (uint8_t*)malloc((size_t)(m > 0 ? m : 1));
  int64_t k = 0;
  for (int64_t i = 0; i < m; ++i) {
    if (cand[i] == p) continue;
    C[k].id = cand[i];
    C[k].d = dist_ij(D, p, cand[i]);
    C[k].expanded = 0;
    k++;
  }
  qsort(C, (size_t)k, sizeof(ent), ent_cmp);
  int64_t u = 0;
  for (int64_t i = 0; i < k; ++i)
    if (i == 0 || C[i].id != C[u - 1].id) C[u++] = C[i];
  uint64_t ev = 0;
  int32_t r = prune_sorted(D, C, u, alpha, R, out, alive, &ev);
  if (evals) *evals = ev + (uint64_t)u;
  free(C);
  free(alive);
  return r;
}

/* ------------------------------------------------------------------------ *
 * FGraft (Section 3).  Points are split into B blocks, block(p) = p mod B
 * (B <= 1: one block, the frozen Graft harvest).  For b = 0..B-1 every point
 * p of block b beam-searches S_b with x_p as the query (width ef_h, entry at
 * the T roots), the expanded set minus p is occlusion-pruned into A[p]
 * (at most R ids, in keep order), and then
 *     S_{b+1} = S_b  U  {(p,u), (u,p) : u in A[p], p in block b}.
 * S_b is held literally: one sorted, duplicate-free neighbour array per
 * vertex, starting from the scaffold.
 * A: n*R ids (-1 padded); cnt: n.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t* v;
  int64_t len, cap;
} vec32;

static void vec_push(vec32* a, int32_t x) {
  if (a->len == a->cap) {
    a->cap = a->cap ? 2 * a->cap : 8;
    a->v = (int32_t*)realloc(a->v, sizeof(int32_t) * (size_t)a->cap);
  }
  a->v[a->len++] = x;
}

static void vec_sort_unique(vec32* a) {
  qsort(a->v, (size_t)a->len, sizeof(int32_t), i32_cmp);
  int64_t u = 0;
  for (int64_t i = 0; i < a->len; ++i)
    if (i == 0 || a->v[i] != a->v[u - 1]) a->v[u++] = a->v[i];
  a->len = u;
}

static void adj_to_csr(int64_t n, const vec32* adj, int64_t* off, int32_t** ids) {
  off[0] = 0;
  for (int64_t u = 0; u < n; ++u) off[u + 1] = off[u] + adj[u].len;
  *ids = (int32_t*)realloc(*ids, sizeof(int32_t) * (size_t)(off[n] > 0 ? off[n] : 1));
  for (int64_t u = 0; u < n; ++u) memcpy(*ids + off[u], adj[u].v, sizeof(int32_t) * (size_t)adj[u].len);
}

int fgo_fgraft(const fgo_data* D, int32_t T, const int32_t* roots, const int64_t* s_off,
               const int32_t* s_ids, int32_t R, int32_t ef_h, int32_t B, float alpha,
               int32_t nthreads, int32_t* A, int32_t* cnt, fgo_counters* ctr,
               uint64_t* per_block_evals /* optional, nblocks entries */) {
  const int64_t n = D->n;
  const int32_t nb = B <= 1 ? 1 : B;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  int nth = omp_get_max_threads();
#else
  (void)nthreads;
  int nth = 1;
#endif
  vec32* adj = (vec32*)calloc((size_t)n, sizeof(vec32));
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = s_off[u]; e < s_off[u + 1]; ++e) vec_push(&adj[u], s_ids[e]);
  for (int64_t i = 0; i < n * (int64_t)R; ++i) A[i] = -1;
  for (int64_t i = 0; i < n; ++i) cnt[i] = 0;
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  int32_t* ids = NULL;
  uint64_t* ev_h = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
  uint64_t* ev_p = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
  uint64_t* ex = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
  for (int32_t b = 0; b < nb; ++b) {
    adj_to_csr(n, adj, off, &ids);
    int64_t maxdeg = csr_maxdeg(n, off);
#pragma omp parallel num_threads(nth)
    {
      beam_scratch S;
      S.visited = (uint8_t*)calloc((size_t)n, 1);
      S.vlist = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
      S.pool_cap = ef_h + maxdeg + T;
      S.pool = (ent*)malloc(sizeof(ent) * (size_t)S.pool_cap);
      int32_t* E_ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
      float* E_d = (float*)malloc(sizeof(float) * (size_t)n);
      ent* C = (ent*)malloc(sizeof(ent) * (size_t)n);
      uint8_t* alive = (uint8_t*)malloc((size_t)n);
#pragma omp for schedule(dynamic, 16)
      for (int64_t p = b; p < n; p += nb) {
        int64_t nev = 0, pl = 0;
        int64_t ne = beam_run(D, off, ids, roots, T, row_ptr(D, p), ef_h, &S, E_ids, E_d, &nev, &pl);
        int64_t m = 0;
        for (int64_t i = 0; i < ne; ++i) {
          if (E_ids[i] == (int32_t)p) continue;
          C[m].id = E_ids[i];
          C[m].d = E_d[i];
          C[m].expanded = 0;
          m++;
        }
        qsort(C, (size_t)m, sizeof(ent), ent_cmp);
        uint64_t pe = 0;
        cnt[p] = prune_sorted(D, C, m, alpha, R, A + p * R, alive, &pe);
        ev_h[p] = (uint64_t)nev;
        ev_p[p] = pe;
        ex[p] = (uint64_t)ne;
      }
      free(S.visited);
      free(S.vlist);
      free(S.pool);
      free(E_ids);
      free(E_d);
      free(C);
      free(alive);
    }
    uint64_t blk = 0;
    for (int64_t p = b; p < n; p += nb) blk += ev_h[p];
    if (per_block_evals) per_block_evals[b] = blk;
    /* union update, after every row of block b is final */
    for (int64_t p = b; p < n; p += nb)
      for (int32_t i = 0; i < cnt[p]; ++i) {
        int32_t u = A[p * R + i];
        vec_push(&adj[p], u);
        vec_push(&adj[u], (int32_t)p);
      }
    for (int64_t u = 0; u < n; ++u) vec_sort_unique(&adj[u]);
  }
  if (ctr) {
    for (int64_t p = 0; p < n; ++p) {
      ctr->harvest_evals += ev_h[p];
      ctr->prune_evals += ev_p[p];
      ctr->expansions += ex[p];
    }
  }
  for (int64_t u = 0; u < n; ++u) free(adj[u].v);
  free(adj);
  free(off);
  free(ids);
  free(ev_h);
  free(ev_p);
  free(ex);
  return 0;
}

/* S_b as a CSR (scaffold plus the rows of blocks < b, both directions);
 * two calls, the first with ids == NULL for the size.  Exposed for tests. */
int fgo_substrate(int64_t n, const int64_t* s_off, const int32_t* s_ids, const int32_t* A,
                  const int32_t* cnt, int32_t R, int32_t B, int32_t b, int64_t* off, int32_t* ids,
                  int64_t* nnz) {
  const int32_t nb = B <= 1 ? 1 : B;
  vec32* adj = (vec32*)calloc((size_t)n, sizeof(vec32));
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = s_off[u]; e < s_off[u + 1]; ++e) vec_push(&adj[u], s_ids[e]);
  for (int64_t p = 0; p < n; ++p) {
    if ((p % nb) >= b) continue;
    for (int32_t i = 0; i < cnt[p]; ++i) {
      int32_t u = A[p * R + i];
      vec_push(&adj[p], u);
      vec_push(&adj[u], (int32_t)p);
    }
  }
  int64_t total = 0;
  for (int64_t u = 0; u < n; ++u) {
    vec_sort_unique(&adj[u]);
    if (off) off[u] = total;
    if (ids) memcpy(ids + total, adj[u].v, sizeof(int32_t) * (size_t)adj[u].len);
    total += adj[u].len;
    free(adj[u].v);
  }
  if (off) off[n] = total;
  if (nnz) *nnz = total;
  free(adj);
  return 0;
}

/* ------------------------------------------------------------------------ *
 * Final graph (Section 3: harvested rows symmetrised and re-pruned, plus the
 * tree-0 spine).  Reading: C(u) = A[u] U {p : u in A[p]}; when |C(u)| > R the
 * row is the occlusion prune of C(u) (sorted by (delta(u,.), id)) to R,
 * otherwise C(u); then the tree-0 parent and children of u are added; the row
 * is sorted by (delta(u,v), id).  Work counted: one evaluation per distinct
 * vertex of C(u) U spine(u) plus the removal passes.
 * Two calls: the first with ids == NULL gives the size.
 * ------------------------------------------------------------------------ */
int fgo_final(const fgo_data* D, const int32_t* A, const int32_t* cnt, int32_t R, float alpha,
              const int32_t* parent0, int64_t* off, int32_t* ids, int64_t* nnz,
              uint64_t* evals_out) {
  const int64_t n = D->n;
  vec32* cand = (vec32*)calloc((size_t)n, sizeof(vec32));
  vec32* spine = (vec32*)calloc((size_t)n, sizeof(vec32));
  for (int64_t p = 0; p < n; ++p)
    for (int32_t i = 0; i < cnt[p]; ++i) {
      int32_t u = A[p * R + i];
      vec_push(&cand[p], u);
      vec_push(&cand[u], (int32_t)p);
    }
  for (int64_t x = 0; x < n; ++x)
    if (parent0[x] >= 0) {
      vec_push(&spine[x], parent0[x]);
      vec_push(&spine[parent0[x]], (int32_t)x);
    }
  uint64_t ev = 0;
  int64_t total = 0;
  for (int64_t u = 0; u < n; ++u) {
    vec_sort_unique(&cand[u]);
    vec_sort_unique(&spine[u]);
    int64_t m = cand[u].len;
    ent* C = (ent*)malloc(sizeof(ent) * (size_t)(m + spine[u].len + 1));
    for (int64_t i = 0; i < m; ++i) {
      C[i].id = cand[u].v[i];
      C[i].d = dist_ij(D, u, C[i].id);
      C[i].expanded = 0;
    }
    ev += (uint64_t)m;
    qsort(C, (size_t)m, sizeof(ent), ent_cmp);
    int64_t rl = m;
    if (m > R) {
      int32_t* keep = (int32_t*)malloc(sizeof(int32_t) * (size_t)R);
      uint8_t* alive = (uint8_t*)malloc((size_t)m);
      int32_t k = prune_sorted(D, C, m, alpha, R, keep, alive, &ev);
      /* kept entries keep their delta; rebuild the row from them */
      ent* K = (ent*)malloc(sizeof(ent) * (size_t)(k > 0 ? k : 1));
      for (int32_t i = 0; i < k; ++i) {
        for (int64_t j = 0; j < m; ++j)
          if (C[j].id == keep[i]) {
            K[i] = C[j];
            break;
          }
      }
      memcpy(C, K, sizeof(ent) * (size_t)k);
      rl = k;
      free(K);
      free(keep);
      free(alive);
    }
    /* spine union: a spine vertex already a candidate has its delta known */
    for (int64_t s = 0; s < spine[u].len; ++s) {
      int32_t v = spine[u].v[s];
      int in_row = 0, in_cand = 0;
      for (int64_t j = 0; j < rl; ++j) in_row |= (C[j].id == v);
      for (int64_t j = 0; j < m; ++j) in_cand |= (cand[u].v[j] == v);
      if (!in_cand) ev++;
      if (in_row) continue;
      C[rl].id = v;
      C[rl].d = dist_ij(D, u, v);
      C[rl].expanded = 0;
      rl++;
    }
    qsort(C, (size_t)rl, sizeof(ent), ent_cmp);
    if (off) off[u] = total;
    if (ids)
      for (int64_t j = 0; j < rl; ++j) ids[total + j] = C[j].id;
    total += rl;
    free(C);
  }
  if (off) off[n] = total;
  if (nnz) *nnz = total;
  if (evals_out) *evals_out = ev;
  for (int64_t u = 0; u < n; ++u) {
    free(cand[u].v);
    free(spine[u].v);
  }
  free(cand);
  free(spine);
  return 0;
}

/* ------------------------------------------------------------------------ *
 * Query search over a CSR graph: the same beam as the harvest with width
 * ef_s, entering at the T roots; the answer is the first k pool entries
 * (padded with -1 / +inf when fewer were reached).  Q rows have stride ldq.
 * ------------------------------------------------------------------------ */
int fgo_search(const fgo_data* D, const int64_t* off, const int32_t* ids, const int32_t* roots,
               int32_t T, const void* Q, int64_t nq, int64_t ldq, int32_t k, int32_t ef_s,
               int32_t* out_ids, float* out_d, uint32_t* out_evals, int32_t nthreads) {
  const int64_t n = D->n;
  int64_t maxdeg = csr_maxdeg(n, off);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    beam_scratch S;
    S.visited = (uint8_t*)calloc((size_t)n, 1);
    S.vlist = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    S.pool_cap = ef_s + maxdeg + T;
    S.pool = (ent*)malloc(sizeof(ent) * (size_t)S.pool_cap);
    int32_t* E_ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    float* E_d = (float*)malloc(sizeof(float) * (size_t)n);
#pragma omp for schedule(dynamic, 16)
    for (int64_t qi = 0; qi < nq; ++qi) {
      const void* q = D->metric == FGO_L2_U8 ? (const void*)((const uint8_t*)Q + qi * ldq)
                                              : (const void*)((const float*)Q + qi * ldq);
      int64_t nev = 0, pl = 0;
      beam_run(D, off, ids, roots, T, q, ef_s, &S, E_ids, E_d, &nev, &pl);
      for (int32_t i = 0; i < k; ++i) {
        out_ids[qi * k + i] = i < pl ? S.pool[i].id : -1;
        out_d[qi * k + i] = i < pl ? S.pool[i].d : INFINITY;
      }
      if (out_evals) out_evals[qi] = (uint32_t)nev;
    }
    free(S.visited);
    free(S.vlist);
    free(S.pool);
    free(E_ids);
    free(E_d);
  }
  return 0;
}

/* Exact top-k of each query over all n points by (delta, id): the
 * brute-force answer key of Section 2. */
int fgo_bruteforce(const fgo_data* D, const void* Q, int64_t nq, int64_t ldq, int32_t k,
                   int32_t* out_ids, float* out_d, int32_t nthreads) {
  const int64_t n = D->n;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    ent* L = (ent*)malloc(sizeof(ent) * (size_t)n);
#pragma omp for schedule(dynamic, 4)
    for (int64_t qi = 0; qi < nq; ++qi) {
      const void* q = D->metric == FGO_L2_U8 ? (const void*)((const uint8_t*)Q + qi * ldq)
                                              : (const void*)((const float*)Q + qi * ldq);
      for (int64_t j = 0; j < n; ++j) {
        L[j].d = dist_ptr(D, q, row_ptr(D, j));
        L[j].id = (int32_t)j;
        L[j].expanded = 0;
      }
      qsort(L, (size_t)n, sizeof(ent), ent_cmp);
      for (int32_t i = 0; i < k; ++i) {
        out_ids[qi * k + i] = i < n ? L[i].id : -1;
        out_d[qi * k + i] = i < n ? L[i].d : INFINITY;
      }
    }
    free(L);
  }
  return 0;
}

/* ------------------------------------------------------------------------ *
 * Dense block (Section 5.3: a pair set fixed before evaluation): for each block of
 * bs ids (-1 = padding), every ordered pair i != j of valid members, the
 * canonical delta, and per row the k smallest (delta, id).  Rows of padding
 * and missing neighbours are filled with -1 / +inf.  use_f64 != 0 ranks by
 * the double-precision distance instead (reference for error reports).
 * ------------------------------------------------------------------------ */
int fgo_dense_block(const fgo_data* D, const int32_t* block_ids, int64_t nb, int32_t bs,
                    int32_t k, int32_t use_f64, int32_t* out_ids, float* out_d, double* out_d64,
                    int32_t nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    ent* L = (ent*)malloc(sizeof(ent) * (size_t)bs);
    double* L64 = (double*)malloc(sizeof(double) * (size_t)bs);
    int32_t* L64i = (int32_t*)malloc(sizeof(int32_t) * (size_t)bs);
#pragma omp for collapse(2) schedule(dynamic, 8)
    for (int64_t blk = 0; blk < nb; ++blk)
      for (int32_t i = 0; i < bs; ++i) {
        const int32_t* ids = block_ids + blk * bs;
        int64_t o = (blk * bs + i) * (int64_t)k;
        int32_t xi = ids[i];
        int64_t m = 0;
        if (xi >= 0) {
          for (int32_t j = 0; j < bs; ++j) {
            int32_t xj = ids[j];
            if (j == i || xj < 0) continue;
            if (use_f64) {
              L64[m] = fgo_dist_f64(D, xi, xj);
              L64i[m] = xj;
            } else {
              L[m].d = dist_ij(D, xi, xj);
              L[m].id = xj;
              L[m].expanded = 0;
            }
            m++;
          }
        }
        if (use_f64) {
          /* selection of the k smallest (d64, id), plain repeated minimum */
          for (int32_t s = 0; s < k; ++s) {
            int64_t best = -1;
            for (int64_t j = 0; j < m; ++j) {
              if (L64i[j] < 0) continue;
              if (best < 0 || L64[j] < L64[best] || (L64[j] == L64[best] && L64i[j] < L64i[best]))
                best = j;
            }
            out_ids[o + s] = best >= 0 ? L64i[best] : -1;
            if (out_d64) out_d64[o + s] = best >= 0 ? L64[best] : INFINITY;
            if (out_d) out_d[o + s] = best >= 0 ? (float)L64[best] : INFINITY;
            if (best >= 0) L64i[best] = -1;
          }
        } else {
          qsort(L, (size_t)m, sizeof(ent), ent_cmp);
          for (int32_t s = 0; s < k; ++s) {
            out_ids[o + s] = s < m ? L[s].id : -1;
            if (out_d) out_d[o + s] = s < m ? L[s].d : INFINITY;
          }
        }
      }
    free(L);
    free(L64);
    free(L64i);
  }
  return 0;
}
