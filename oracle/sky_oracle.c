/*
 * Plain CPU oracle for the partitioned skyline method of Ciaccia & Martinenghi,
 * "Optimization Strategies for Parallel Computation of Skylines" (arXiv 2411.14968).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The GPU library never links,
 * includes or calls it, and this file includes nothing from the GPU library.
 *
 * Everything here is deliberately slow and direct: loops written from the
 * paper's definitions, no blocking, no fusion.  They run single-threaded unless
 * orc_set_threads asks for more: then Algorithm 2's two parallel loops (the
 * local skyline of every partition, and NoSeq's per-tuple checks) are spread
 * over OpenMP threads, as the paper spreads them over cores; results and test
 * counts are the same for any thread count.  Floating point is the
 * input's own FP32 (the method compares the caller's FP32 values), compiled
 * with -ffp-contract=off and without fast-math so every sum is a correctly
 * rounded FP32 addition in the stated order.
 *
 * Readings of places where the paper is silent or garbled (each also listed in
 * the design notes):
 *  - score f(t) = FP32 sum of the attributes, added left to right (§2 monotone
 *    scoring function; a sum is the paper's example of one); a tuple holding
 *    both +inf and -inf, whose sum is undefined, scores +inf;
 *  - SFS sort key = (f, x_1, ..., x_d, index): a total order that is a
 *    topological sort of dominance even when f ties (Algorithm 1, §2);
 *  - Grid cell index = sum_i clamp(floor(fl(x_i * m_i)), 0, m_i - 1) * prod_{j<i} m_j
 *    (§3.2 equation; clamping covers x = 1.0 and values outside [0,1]);
 *  - Angular index computed without transcendentals (§3.3, Eq. index-angular):
 *    k_i = #{k in 1..m_i-1 : S_i >= fl(x_i^2) * T_{i,k}},
 *    S_i = FP32 suffix sum x_d^2 + ... + x_{i+1}^2 accumulated from the right,
 *    T_{i,k} = (float)(tan(k*pi/(2*m_i))^2) evaluated in double;
 *  - Random: the i-th output of SplitMix64(seed) (Steele, Lea & Flood 2014) is
 *    point i's random key; rank by (key, i); pid = floor(rank * p / N) (§3.1);
 *  - Sliced: rank by (x_dim, f, index); pid = floor(start * p / N) where start
 *    is the rank of the first point having the same (x_dim, f) (§3.4; the
 *    paper's (N-1) denominator would leave the last tuple alone in partition p);
 *  - Sorted representatives: the first k points of each partition in (f, index)
 *    order; dominated representatives are removed before filtering (§4.1);
 *  - Region representatives (§4.1, volume of the dominance region): the k
 *    points of each partition with the largest V(t) = prod_i (1 - c_i) in
 *    double, factors left to right, where c_i is the attribute (divided by
 *    the column maximum when normalising) clamped to [0, 1] -- the volume of
 *    the part of the dominance region inside the unit cube; ties by index;
 *  - NoSeq potential dominators (§4.2): Random/Angular u \ u_i; Grid the u_j
 *    whose cell is componentwise <= cell i (weak grid dominance read as <=);
 *    Sliced the u_j with j < i.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* scheme / option codes used by the oracle's entry points */
enum { ORC_RANDOM = 0, ORC_GRID = 1, ORC_ANGULAR = 2, ORC_SLICED = 3, ORC_NONE = 4 };
enum { ORC_REP_NONE = 0, ORC_REP_SORTED = 1, ORC_REP_REGION = 2 };
enum { ORC_MERGE_SEQUENTIAL = 0, ORC_MERGE_NOSEQ = 1 };
/* per-point stage codes: where the point left the pipeline */
enum {
  ORC_ST_SKY = 1,        /* in Sky(r)                                   */
  ORC_ST_GRID = 2,       /* in a cell removed by Grid Filtering (§3.2)  */
  ORC_ST_REP = 3,        /* dominated by a representative (§4.1)        */
  ORC_ST_LOCAL = 4,      /* dominated inside its partition (Alg. 2)     */
  ORC_ST_MERGE = 5       /* in u but not in Sky(r) (Alg. 2 / §4.2)      */
};

/* ---------------------------------------------------------------- §2, Def. 1 */

/* t dominates s: t[A] <= s[A] for every A, and t[A'] < s[A'] for some A'. */
static int dominates(const float *t, const float *s, int d) {
  int strictly_better = 0;
  for (int a = 0; a < d; ++a) {
    if (!(t[a] <= s[a])) return 0;
    if (t[a] < s[a]) strictly_better = 1;
  }
  return strictly_better;
}

int orc_dominates(const float *t, const float *s, int d) { return dominates(t, s, d); }

/* Sky(r) straight from Def. 1: t is kept iff no s in r dominates it. O(N^2). */
void orc_skyline_brute(const float *pts, int64_t n, int d, uint8_t *in_sky) {
  for (int64_t i = 0; i < n; ++i) {
    int kept = 1;
    for (int64_t j = 0; j < n && kept; ++j)
      if (j != i && dominates(pts + j * d, pts + i * d, d)) kept = 0;
    in_sky[i] = (uint8_t)kept;
  }
}

/* Relative skyline Sky_c(r) (§4.2 definition): keep t in r iff no s in c dominates t. */
void orc_relative_skyline(const float *r, int64_t nr, const float *c, int64_t nc, int d,
                          uint8_t *kept) {
  for (int64_t i = 0; i < nr; ++i) {
    int k = 1;
    for (int64_t j = 0; j < nc && k; ++j)
      if (dominates(c + j * d, r + i * d, d)) k = 0;
    kept[i] = (uint8_t)k;
  }
}

/* --------------------------------------------------- rank space (from Def. 1) */

/* Def. 1 looks at each attribute of two tuples only through <= and <, so
   replacing every value of column a by its dense rank in that column (the
   number of distinct values of the column below it) keeps every dominance
   relation.  ranks[i*d + a] = that rank (-0.0 and +0.0 are one value);
   distinct[a] = the column's number of distinct values. */
static int cmp_float(const void *a, const void *b) {
  const float x = *(const float *)a, y = *(const float *)b;
  return (x < y) ? -1 : (x > y);
}

void orc_dense_ranks(const float *pts, int64_t n, int d, uint32_t *ranks, uint32_t *distinct) {
  float *col = (float *)malloc((size_t)(n > 0 ? n : 1) * sizeof(float));
  for (int a = 0; a < d; ++a) {
    for (int64_t i = 0; i < n; ++i) col[i] = pts[i * d + a] + 0.0f;
    qsort(col, (size_t)n, sizeof(float), cmp_float);
    int64_t m = 0; /* the distinct values, ascending, in col[0..m) */
    for (int64_t i = 0; i < n; ++i)
      if (m == 0 || col[i] != col[m - 1]) col[m++] = col[i];
    distinct[a] = (uint32_t)m;
    for (int64_t i = 0; i < n; ++i) {
      const float v = pts[i * d + a] + 0.0f;
      int64_t lo = 0, hi = m; /* first position holding a value >= v */
      while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < v) lo = mid + 1; else hi = mid;
      }
      ranks[i * d + a] = (uint32_t)lo;
    }
  }
  free(col);
}

/* ------------------------------------------------- §2 monotone scoring function */

static float score_of(const float *t, int d) {
  float f = t[0];
  for (int a = 1; a < d; ++a) f = f + t[a];
  /* a tuple holding both +inf and -inf has no sum (inf - inf); it can only
     dominate tuples that hold +inf in the same attribute, whose sum is +inf
     or undefined too, so +inf keeps the score monotone under dominance */
  return f != f ? INFINITY : f;
}

void orc_scores(const float *pts, int64_t n, int d, float *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = score_of(pts + i * d, d);
}

/* ------------------------------------------------------------ threads */

/* Threads of Algorithm 2's parallel loops (1: the plain loops).  Only the
   CPU timing of the method uses more than one. */
static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

/* Threads available to the parallel loops (1 when built without OpenMP). */
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------ Algorithm 1 (SFS) */

typedef struct { float f; int64_t id; } scored_t;

static _Thread_local const float *g_pts; /* sort context of the calling thread */
static _Thread_local int g_d;

/* (f, x_1..x_d, id) ascending: a linear extension of dominance (if s dominates
   t then f(s) <= f(t) and, on equal f, s precedes t lexicographically). */
static int cmp_sfs(const void *a, const void *b) {
  const scored_t *x = (const scored_t *)a, *y = (const scored_t *)b;
  if (x->f < y->f) return -1;
  if (x->f > y->f) return 1;
  const float *px = g_pts + x->id * g_d, *py = g_pts + y->id * g_d;
  for (int k = 0; k < g_d; ++k) {
    if (px[k] < py[k]) return -1;
    if (px[k] > py[k]) return 1;
  }
  return (x->id < y->id) ? -1 : (x->id > y->id);
}

/* SFS over the subset ids[0..m) of pts: sort by f, scan, keep a window of the
   tuples no window tuple dominates.  in_sky[id] is set to 1 for window tuples
   and 0 for the other ids of the subset.  *tests counts window comparisons.
   Returns |window|. */
int64_t orc_sfs(const float *pts, int d, const int64_t *ids, int64_t m, uint8_t *in_sky,
                uint64_t *tests) {
  if (m <= 0) return 0;
  scored_t *ord = (scored_t *)malloc((size_t)m * sizeof(scored_t));
  int64_t *w = (int64_t *)malloc((size_t)m * sizeof(int64_t));
  for (int64_t i = 0; i < m; ++i) {
    ord[i].id = ids[i];
    ord[i].f = score_of(pts + ids[i] * d, d);
  }
  g_pts = pts;
  g_d = d;
  qsort(ord, (size_t)m, sizeof(scored_t), cmp_sfs);
  int64_t wn = 0;
  uint64_t cnt = 0;
  for (int64_t i = 0; i < m; ++i) {
    const float *t = pts + ord[i].id * d;
    int dominated = 0;
    for (int64_t j = 0; j < wn; ++j) {
      ++cnt;
      if (dominates(pts + w[j] * d, t, d)) { dominated = 1; break; }
    }
    in_sky[ord[i].id] = (uint8_t)!dominated;
    if (!dominated) w[wn++] = ord[i].id;
  }
  if (tests) *tests += cnt;
  free(ord);
  free(w);
  return wn;
}

/* Whole-set SFS convenience: in_sky[i] for i in [0, n). */
int64_t orc_sfs_all(const float *pts, int64_t n, int d, uint8_t *in_sky, uint64_t *tests) {
  int64_t *ids = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) ids[i] = i;
  int64_t k = orc_sfs(pts, d, ids, n, in_sky, tests);
  free(ids);
  return k;
}

/* ------------------------------------------------------- partition assignment */

/* Per-column key scale for Grid/Angular on data outside [0,1]: the column
   maximum when it is positive and finite, else 1. */
void orc_key_scale(const float *pts, int64_t n, int d, float *scale) {
  for (int a = 0; a < d; ++a) {
    float mx = -INFINITY;
    for (int64_t i = 0; i < n; ++i)
      if (pts[i * d + a] > mx) mx = pts[i * d + a];
    scale[a] = (mx > 0.0f && isfinite(mx)) ? mx : 1.0f;
  }
}

static float key_coord(const float *t, int a, const float *scale) {
  return scale ? t[a] / scale[a] : t[a];
}

/* §3.2: p(t) = sum_i floor(t[A_i] * m_i) * prod_{j<i} m_j, each digit clamped to
   [0, m_i - 1]. */
void orc_assign_grid(const float *pts, int64_t n, int d, const uint32_t *m,
                     const float *scale, uint32_t *pid) {
  for (int64_t i = 0; i < n; ++i) {
    const float *t = pts + i * d;
    uint64_t id = 0, weight = 1;
    for (int a = 0; a < d; ++a) {
      float v = key_coord(t, a, scale) * (float)m[a];
      float fl = floorf(v);
      uint32_t c;
      if (!(fl > 0.0f)) c = 0;
      else if (fl >= (float)(m[a] - 1)) c = m[a] - 1;
      else c = (uint32_t)fl;
      id += (uint64_t)c * weight;
      weight *= m[a];
    }
    pid[i] = (uint32_t)id;
  }
}

/* Threshold table of the Angular reading: T[k-1] = (float)(tan(k*pi/(2m))^2), k = 1..m-1. */
static void angular_table(uint32_t m, float *T) {
  const double pi = 3.14159265358979323846;
  for (uint32_t k = 1; k < m; ++k) {
    double tk = tan((double)k * pi / (2.0 * (double)m));
    T[k - 1] = (float)(tk * tk);
  }
}

/* §3.3, Eq. (index-angular): p(t) = sum_i floor(2 phi_i m_i / pi) * prod_{j<i} m_j
   with tan(phi_i) = sqrt(sum_{j>i} x_j^2) / x_i, evaluated as the count of
   angular thresholds phi_i reaches (exact in real arithmetic, clamped to m_i - 1). */
void orc_assign_angular(const float *pts, int64_t n, int d, const uint32_t *m,
                        const float *scale, uint32_t *pid) {
  size_t off[8], tot = 0;
  for (int a = 0; a + 1 < d; ++a) { off[a] = tot; tot += m[a]; }
  float *T = (float *)malloc(sizeof(float) * (tot + 1));
  for (int a = 0; a + 1 < d; ++a) angular_table(m[a], T + off[a]);
  for (int64_t i = 0; i < n; ++i) {
    const float *t = pts + i * d;
    float x[8], S[8];
    for (int a = 0; a < d; ++a) x[a] = key_coord(t, a, scale);
    /* S[a] = x_{a+1}^2 + S[a+1], accumulated from the last coordinate */
    float acc = 0.0f;
    for (int a = d - 1; a >= 1; --a) {
      float sq = x[a] * x[a];
      acc = (a == d - 1) ? sq : sq + acc;
      S[a - 1] = acc;
    }
    uint64_t id = 0, weight = 1;
    for (int a = 0; a + 1 < d; ++a) {
      float xx = x[a] * x[a];
      uint32_t k = 0;
      for (uint32_t j = 1; j < m[a]; ++j)
        if (S[a] >= xx * T[off[a] + (j - 1)]) ++k;
      id += (uint64_t)k * weight;
      weight *= m[a];
    }
    pid[i] = (uint32_t)id;
  }
  free(T);
}

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the i-th output (i from 0) of
   the generator whose state starts at `seed`. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct { uint64_t key; int64_t id; } rkey_t;

static int cmp_rkey(const void *a, const void *b) {
  const rkey_t *x = (const rkey_t *)a, *y = (const rkey_t *)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->id < y->id) ? -1 : (x->id > y->id);
}

/* §3.1: random, equi-numerous partitions. */
void orc_assign_random(int64_t n, uint32_t p, uint64_t seed, uint32_t *pid) {
  if (n <= 0) return;
  rkey_t *ord = (rkey_t *)malloc((size_t)n * sizeof(rkey_t));
  for (int64_t i = 0; i < n; ++i) {
    ord[i].key = orc_splitmix64(seed, (uint64_t)i);
    ord[i].id = i;
  }
  qsort(ord, (size_t)n, sizeof(rkey_t), cmp_rkey);
  for (int64_t r = 0; r < n; ++r)
    pid[ord[r].id] = (uint32_t)(((unsigned __int128)r * p) / (uint64_t)n);
  free(ord);
}

typedef struct { float x, f; int64_t id; } skey_t;

static int cmp_skey(const void *a, const void *b) {
  const skey_t *u = (const skey_t *)a, *v = (const skey_t *)b;
  if (u->x < v->x) return -1;
  if (u->x > v->x) return 1;
  if (u->f < v->f) return -1;
  if (u->f > v->f) return 1;
  return (u->id < v->id) ? -1 : (u->id > v->id);
}

/* §3.4: sort on one dimension (tie-break f, then index) and cut into p slices of
   equal size; a run of equal (x_dim, f) keys is never split. */
void orc_assign_sliced(const float *pts, int64_t n, int d, int dim, uint32_t p, uint32_t *pid) {
  if (n <= 0) return;
  skey_t *ord = (skey_t *)malloc((size_t)n * sizeof(skey_t));
  for (int64_t i = 0; i < n; ++i) {
    ord[i].x = pts[i * d + dim];
    ord[i].f = score_of(pts + i * d, d);
    ord[i].id = i;
  }
  qsort(ord, (size_t)n, sizeof(skey_t), cmp_skey);
  int64_t start = 0;
  for (int64_t r = 0; r < n; ++r) {
    if (r > 0 && !(ord[r].x == ord[r - 1].x && ord[r].f == ord[r - 1].f)) start = r;
    pid[ord[r].id] = (uint32_t)(((unsigned __int128)start * p) / (uint64_t)n);
  }
  free(ord);
}

/* ------------------------------------------------------- §3.2 Grid Filtering */

static void cell_coords(uint32_t cell, int d, const uint32_t *m, uint32_t *c) {
  for (int a = 0; a < d; ++a) {
    c[a] = cell % m[a];
    cell /= m[a];
  }
}

/* dropped[h] = 1 iff some non-empty cell i grid-dominates h, i.e. c_i[j] < c_h[j]
   for every dimension j. */
void orc_grid_filter(const uint32_t *pid, int64_t n, int d, const uint32_t *m,
                     uint8_t *dropped) {
  uint64_t P = 1;
  for (int a = 0; a < d; ++a) P *= m[a];
  uint8_t *occ = (uint8_t *)calloc((size_t)P, 1);
  for (int64_t i = 0; i < n; ++i) occ[pid[i]] = 1;
  uint32_t ch[8], ci[8];
  for (uint64_t h = 0; h < P; ++h) {
    dropped[h] = 0;
    cell_coords((uint32_t)h, d, m, ch);
    for (uint64_t i = 0; i < P && !dropped[h]; ++i) {
      if (!occ[i]) continue;
      cell_coords((uint32_t)i, d, m, ci);
      int all_less = 1;
      for (int a = 0; a < d; ++a)
        if (!(ci[a] < ch[a])) { all_less = 0; break; }
      if (all_less) dropped[h] = 1;
    }
  }
  free(occ);
}

/* ------------------------------------------------------------ Algorithm 2 */

typedef struct { float f; int64_t id; } fid_t;
typedef struct { double v; int64_t id; } vid_t;

/* Descending volume, then ascending index. */
static int cmp_vid(const void *a, const void *b) {
  const vid_t *x = (const vid_t *)a, *y = (const vid_t *)b;
  if (x->v > y->v) return -1;
  if (x->v < y->v) return 1;
  return (x->id < y->id) ? -1 : (x->id > y->id);
}

/* §4.1: hyper-volume of the dominance region of t within [0,1]^d. */
double orc_region_volume(const float *t, int d, const float *scale) {
  double v = 1.0;
  for (int a = 0; a < d; ++a) {
    double c = (double)key_coord(t, a, scale);
    if (c < 0.0) c = 0.0;
    if (c > 1.0) c = 1.0;
    v = v * (1.0 - c);
  }
  return v;
}

static int cmp_fid(const void *a, const void *b) {
  const fid_t *x = (const fid_t *)a, *y = (const fid_t *)b;
  if (x->f < y->f) return -1;
  if (x->f > y->f) return 1;
  return (x->id < y->id) ? -1 : (x->id > y->id);
}

/* Algorithm 2 with the optional optimisations of §3.2 (Grid Filtering),
   §4.1 (Sorted representatives) and §4.2 (NoSeq).  Outputs:
     pid[i]   partition of point i;
     stage[i] ORC_ST_* code saying where point i left the pipeline;
     tests[0] dominance tests of the local SFS runs, tests[1] of the merge.
   Returns |Sky(r)|.  slices: Grid m per dimension (d entries), Angular m per
   angle (d-1 entries).  p: partitions for Random/Sliced (clamped to [1, n]).
   The caller validates the input (no NaN, d in 1..8). */
int64_t orc_partitioned(const float *pts, int64_t n, int d, int scheme, uint32_t p,
                        const uint32_t *slices, int normalize, int slice_dim, uint64_t seed,
                        int grid_filter, int rep, uint32_t reps_per_partition, int merge,
                        uint32_t *pid, uint8_t *stage, uint64_t *tests) {
  if (tests) { tests[0] = 0; tests[1] = 0; }
  if (n <= 0) return 0;
  uint64_t P = 1;
  float scale[8];
  const float *sc = NULL;
  if (normalize && (scheme == ORC_GRID || scheme == ORC_ANGULAR || rep == ORC_REP_REGION)) {
    orc_key_scale(pts, n, d, scale);
    sc = scale;
  }
  /* the partition keys use the scale only for Grid and Angular */
  const float *key_sc = (scheme == ORC_GRID || scheme == ORC_ANGULAR) ? sc : NULL;
  /* Partition(r, p): Alg. 2 first phase */
  if (scheme == ORC_GRID) {
    for (int a = 0; a < d; ++a) P *= slices[a];
    orc_assign_grid(pts, n, d, slices, key_sc, pid);
  } else if (scheme == ORC_ANGULAR) {
    for (int a = 0; a + 1 < d; ++a) P *= slices[a];
    orc_assign_angular(pts, n, d, slices, key_sc, pid);
  } else if (scheme == ORC_RANDOM || scheme == ORC_SLICED) {
    P = p < 1 ? 1 : p;
    if (P > (uint64_t)n) P = (uint64_t)n;
    if (scheme == ORC_RANDOM) orc_assign_random(n, (uint32_t)P, seed, pid);
    else orc_assign_sliced(pts, n, d, slice_dim, (uint32_t)P, pid);
  } else {
    P = 1;
    for (int64_t i = 0; i < n; ++i) pid[i] = 0;
  }
  for (int64_t i = 0; i < n; ++i) stage[i] = 0;

  /* Grid Filtering (§3.2) */
  if (scheme == ORC_GRID && grid_filter) {
    uint8_t *dropped = (uint8_t *)malloc((size_t)P);
    orc_grid_filter(pid, n, d, slices, dropped);
    for (int64_t i = 0; i < n; ++i)
      if (dropped[pid[i]]) stage[i] = ORC_ST_GRID;
    free(dropped);
  }

  /* members of each partition, in index order */
  int64_t *cnt = (int64_t *)calloc((size_t)P + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i)
    if (!stage[i]) cnt[pid[i] + 1]++;
  for (uint64_t q = 0; q < P; ++q) cnt[q + 1] += cnt[q];
  int64_t *mem = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *fill = (int64_t *)malloc((size_t)(P + 1) * sizeof(int64_t));
  memcpy(fill, cnt, (size_t)(P + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i)
    if (!stage[i]) mem[fill[pid[i]]++] = i;

  /* Representatives (§4.1): Sorted = first k tuples of every partition in
     (f, index) order; Region = the k tuples of largest dominance-region
     volume.  Dominated representatives are discarded, then every tuple a
     remaining representative dominates is deleted. */
  if (rep == ORC_REP_SORTED || rep == ORC_REP_REGION) {
    uint32_t k = reps_per_partition < 1 ? 1 : reps_per_partition;
    int64_t *reps = (int64_t *)malloc((size_t)(P * k + 1) * sizeof(int64_t));
    int64_t nrep = 0;
    for (uint64_t q = 0; q < P; ++q) {
      int64_t len = cnt[q + 1] - cnt[q];
      if (len == 0) continue;
      if (rep == ORC_REP_SORTED) {
        fid_t *o = (fid_t *)malloc((size_t)len * sizeof(fid_t));
        for (int64_t j = 0; j < len; ++j) {
          o[j].id = mem[cnt[q] + j];
          o[j].f = score_of(pts + o[j].id * d, d);
        }
        qsort(o, (size_t)len, sizeof(fid_t), cmp_fid);
        for (int64_t j = 0; j < len && j < (int64_t)k; ++j) reps[nrep++] = o[j].id;
        free(o);
      } else {
        vid_t *o = (vid_t *)malloc((size_t)len * sizeof(vid_t));
        for (int64_t j = 0; j < len; ++j) {
          o[j].id = mem[cnt[q] + j];
          o[j].v = orc_region_volume(pts + o[j].id * d, d, sc);
        }
        qsort(o, (size_t)len, sizeof(vid_t), cmp_vid);
        for (int64_t j = 0; j < len && j < (int64_t)k; ++j) reps[nrep++] = o[j].id;
        free(o);
      }
    }
    uint8_t *rep_kept = (uint8_t *)malloc((size_t)(nrep + 1));
    for (int64_t a = 0; a < nrep; ++a) {
      rep_kept[a] = 1;
      for (int64_t b = 0; b < nrep; ++b)
        if (b != a && dominates(pts + reps[b] * d, pts + reps[a] * d, d)) { rep_kept[a] = 0; break; }
    }
    for (int64_t i = 0; i < n; ++i) {
      if (stage[i]) continue;
      for (int64_t a = 0; a < nrep; ++a)
        if (rep_kept[a] && dominates(pts + reps[a] * d, pts + i * d, d)) { stage[i] = ORC_ST_REP; break; }
    }
    free(rep_kept);
    free(reps);
  }

  /* ComputeLocalSet: u_i = SFS over what is left of r_i */
  uint8_t *flag = (uint8_t *)calloc((size_t)n, 1);
  int64_t *sub = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  uint64_t t_local = 0, t_merge = 0;
  /* the partitions are independent: each uses its own slice of sub */
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1) reduction(+ : t_local) if (g_threads > 1)
  for (int64_t q = 0; q < (int64_t)P; ++q) {
    int64_t *own = sub + cnt[q];
    int64_t m = 0;
    for (int64_t j = cnt[q]; j < cnt[q + 1]; ++j)
      if (!stage[mem[j]]) own[m++] = mem[j];
    orc_sfs(pts, d, own, m, flag, &t_local);
    for (int64_t j = 0; j < m; ++j)
      if (!flag[own[j]]) stage[own[j]] = ORC_ST_LOCAL;
  }

  /* final phase: Sky(u) (sequential) or the NoSeq identity of Prop. 2 */
  int64_t nu = 0;
  for (int64_t i = 0; i < n; ++i)
    if (!stage[i]) sub[nu++] = i;
  int64_t result = 0;
  if (merge == ORC_MERGE_SEQUENTIAL || P == 1) {
    memset(flag, 0, (size_t)n);
    orc_sfs(pts, d, sub, nu, flag, &t_merge);
    for (int64_t j = 0; j < nu; ++j) {
      int64_t i = sub[j];
      stage[i] = flag[i] ? ORC_ST_SKY : ORC_ST_MERGE;
      result += flag[i];
    }
  } else {
    uint8_t *kill = (uint8_t *)calloc((size_t)n, 1);
    /* every union tuple is checked independently */
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 64) reduction(+ : t_merge) if (g_threads > 1)
    for (int64_t a = 0; a < nu; ++a) {
      uint32_t ci[8], cj[8];
      int64_t t = sub[a];
      uint32_t pi = pid[t];
      if (scheme == ORC_GRID) cell_coords(pi, d, slices, ci);
      for (int64_t b = 0; b < nu; ++b) {
        int64_t s = sub[b];
        uint32_t pj = pid[s];
        if (pj == pi) continue; /* pd_i is a subset of u \ u_i */
        int in_pd;
        if (scheme == ORC_SLICED) {
          in_pd = pj < pi;
        } else if (scheme == ORC_GRID) {
          cell_coords(pj, d, slices, cj);
          in_pd = 1;
          for (int x = 0; x < d; ++x)
            if (!(cj[x] <= ci[x])) { in_pd = 0; break; }
        } else {
          in_pd = 1;
        }
        if (!in_pd) continue;
        ++t_merge;
        if (dominates(pts + s * d, pts + t * d, d)) { kill[t] = 1; break; }
      }
    }
    for (int64_t a = 0; a < nu; ++a) {
      int64_t t = sub[a];
      stage[t] = kill[t] ? ORC_ST_MERGE : ORC_ST_SKY;
      result += !kill[t];
    }
    free(kill);
  }
  if (tests) { tests[0] = t_local; tests[1] = t_merge; }
  free(sub);
  free(flag);
  free(fill);
  free(mem);
  free(cnt);
  return result;
}
