/*
 * Seeded synthetic graph generators and a CSR builder.
 *
 * This file produces the INPUTS shared by the CPU oracle and the GPU path:
 * simple undirected graphs as int64 row offsets + int32 sorted adjacency.
 * It holds none of the estimator's arithmetic (no intersections, no counts,
 * no edge sampler): only random graph models and a sort/dedupe CSR build.
 *
 * Random numbers come from a counter-based generator (Murmur3's 64-bit
 * finaliser applied to a Weyl sequence), so every draw is a pure function of
 * (seed, stream, index) and the output is identical for any thread count.
 *
 * Models:
 *   - Erdos-Renyi G(n, m): exactly m distinct pairs, uniform by rejection.
 *   - Chung-Lu: endpoints drawn i.i.d. proportional to a capped power-law
 *     weight vector (Vose alias table), self-loops and repeats dropped.
 *   - R-MAT: recursive quadrant choice with probabilities (a, b, c, d).
 *   - 2-D random geometric graph: points in the unit square, radius r.
 * Vertex labels can be randomly permuted after generation (Graph500 style).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ RNG */

static inline uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdULL;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ULL;
  k ^= k >> 33;
  return k;
}

static inline uint64_t rng_u64(uint64_t seed, uint64_t stream, uint64_t idx) {
  uint64_t key = fmix64(seed ^ (stream * 0xd1342543de82ef95ULL + 0x632be59bd9b4e019ULL));
  return fmix64(key + (idx + 1) * 0x9e3779b97f4a7c15ULL);
}

static inline double rng_unit(uint64_t seed, uint64_t stream, uint64_t idx) {
  return (double)(rng_u64(seed, stream, idx) >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------ CSR build */

typedef struct {
  int64_t n;
  int64_t nnz;
  int64_t* row_ptr;
  int32_t* col;
} synth_csr;

static int cmp_i32(const void* x, const void* y) {
  int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

static void sort_i32(int32_t* p, int64_t len) {
  if (len < 48) {
    for (int64_t i = 1; i < len; ++i) {
      int32_t x = p[i];
      int64_t j = i - 1;
      while (j >= 0 && p[j] > x) {
        p[j + 1] = p[j];
        --j;
      }
      p[j + 1] = x;
    }
  } else {
    qsort(p, (size_t)len, sizeof(int32_t), cmp_i32);
  }
}

/* Builds a simple undirected CSR from e unordered pairs (a[i], b[i]).
 * Self-loops and repeated pairs are dropped; both orientations are stored;
 * every adjacency list is sorted ascending. Returns NULL on allocation
 * failure. */
static synth_csr* build_csr(int64_t n, int64_t e, const int32_t* a, const int32_t* b) {
  synth_csr* g = (synth_csr*)calloc(1, sizeof(synth_csr));
  int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!g || !deg) return NULL;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < e; ++i) {
    if (a[i] == b[i]) continue;
    __atomic_fetch_add(&deg[a[i]], 1, __ATOMIC_RELAXED);
    __atomic_fetch_add(&deg[b[i]], 1, __ATOMIC_RELAXED);
  }
  int64_t* off = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!off) return NULL;
  off[0] = 0;
  for (int64_t v = 0; v < n; ++v) off[v + 1] = off[v] + deg[v];
  int64_t total = off[n];
  int32_t* tmp = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  if (!tmp) return NULL;
  memcpy(deg, off, (size_t)n * sizeof(int64_t)); /* deg now holds cursors */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < e; ++i) {
    int32_t x = a[i], y = b[i];
    if (x == y) continue;
    int64_t px = __atomic_fetch_add(&deg[x], 1, __ATOMIC_RELAXED);
    int64_t py = __atomic_fetch_add(&deg[y], 1, __ATOMIC_RELAXED);
    tmp[px] = y;
    tmp[py] = x;
  }
  /* sort + dedupe each row in place; deg[v] := distinct count */
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < n; ++v) {
    int32_t* p = tmp + off[v];
    int64_t len = off[v + 1] - off[v];
    sort_i32(p, len);
    int64_t w = 0;
    for (int64_t i = 0; i < len; ++i)
      if (w == 0 || p[i] != p[w - 1]) p[w++] = p[i];
    deg[v] = w;
  }
  g->n = n;
  g->row_ptr = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!g->row_ptr) return NULL;
  g->row_ptr[0] = 0;
  for (int64_t v = 0; v < n; ++v) g->row_ptr[v + 1] = g->row_ptr[v] + deg[v];
  g->nnz = g->row_ptr[n];
  g->col = (int32_t*)malloc((size_t)(g->nnz > 0 ? g->nnz : 1) * sizeof(int32_t));
  if (!g->col) return NULL;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < n; ++v)
    memcpy(g->col + g->row_ptr[v], tmp + off[v], (size_t)deg[v] * sizeof(int32_t));
  free(tmp);
  free(off);
  free(deg);
  return g;
}

/* Fisher-Yates permutation of [0, n) from the counter RNG (stream 7). */
static int32_t* random_perm(int64_t n, uint64_t seed) {
  int32_t* p = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!p) return NULL;
  for (int64_t i = 0; i < n; ++i) p[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    uint64_t r = rng_u64(seed, 7, (uint64_t)i);
    int64_t j = (int64_t)(r % (uint64_t)(i + 1));
    int32_t t = p[i];
    p[i] = p[j];
    p[j] = t;
  }
  return p;
}

static void apply_perm(int64_t e, int32_t* a, int32_t* b, const int32_t* perm) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < e; ++i) {
    a[i] = perm[a[i]];
    b[i] = perm[b[i]];
  }
}

static synth_csr* finish(int64_t n, int64_t e, int32_t* a, int32_t* b, int permute, uint64_t seed) {
  if (permute) {
    int32_t* perm = random_perm(n, seed);
    if (!perm) return NULL;
    apply_perm(e, a, b, perm);
    free(perm);
  }
  synth_csr* g = build_csr(n, e, a, b);
  free(a);
  free(b);
  return g;
}

/* ------------------------------------------------------------ models */

/* R-MAT: e draws on 2^scale vertices; quadrant probabilities a, b, c and
 * d = 1 - a - b - c at every level, no noise. */
synth_csr* synth_rmat(int scale, int64_t e, double pa, double pb, double pc, uint64_t seed,
                      int permute) {
  int64_t n = (int64_t)1 << scale;
  int32_t* a = (int32_t*)malloc((size_t)e * sizeof(int32_t));
  int32_t* b = (int32_t*)malloc((size_t)e * sizeof(int32_t));
  if (!a || !b) return NULL;
  double ab = pa + pb, abc = pa + pb + pc;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < e; ++i) {
    uint32_t src = 0, dst = 0;
    for (int lvl = 0; lvl < scale; ++lvl) {
      double r = rng_unit(seed, 1, (uint64_t)i * 64 + (uint64_t)lvl);
      uint32_t bit = 1u << (scale - 1 - lvl);
      if (r < pa) {
      } else if (r < ab) {
        dst |= bit;
      } else if (r < abc) {
        src |= bit;
      } else {
        src |= bit;
        dst |= bit;
      }
    }
    a[i] = (int32_t)src;
    b[i] = (int32_t)dst;
  }
  return finish(n, e, a, b, permute, seed);
}

/* Chung-Lu: weight w_i = min(cap, c * (i+1)^(-1/(gamma-1))) with c chosen so
 * that sum(w) = total_weight; `draws` endpoint pairs drawn i.i.d.
 * proportional to w (Vose alias table). */
synth_csr* synth_chung_lu(int64_t n, int64_t draws, double gamma, double cap, double total_weight,
                          uint64_t seed, int permute) {
  double alpha = 1.0 / (gamma - 1.0);
  double* w = (double*)malloc((size_t)n * sizeof(double));
  if (!w) return NULL;
  double lo = 0.0, hi = total_weight;
  for (int it = 0; it < 200; ++it) {
    double c = 0.5 * (lo + hi), s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double x = c * pow((double)(i + 1), -alpha);
      s += x < cap ? x : cap;
    }
    if (s < total_weight) lo = c; else hi = c;
  }
  double c = 0.5 * (lo + hi), s = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double x = c * pow((double)(i + 1), -alpha);
    w[i] = x < cap ? x : cap;
    s += w[i];
  }
  /* Vose alias table */
  double* prob = (double*)malloc((size_t)n * sizeof(double));
  int32_t* alias = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* small = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* large = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  if (!prob || !alias || !small || !large) return NULL;
  int64_t ns = 0, nl = 0;
  for (int64_t i = 0; i < n; ++i) {
    prob[i] = w[i] * (double)n / s;
    if (prob[i] < 1.0) small[ns++] = (int32_t)i; else large[nl++] = (int32_t)i;
  }
  while (ns > 0 && nl > 0) {
    int32_t l = small[--ns], g = large[--nl];
    alias[l] = g;
    prob[g] = (prob[g] + prob[l]) - 1.0;
    if (prob[g] < 1.0) small[ns++] = g; else large[nl++] = g;
  }
  while (nl > 0) prob[large[--nl]] = 1.0;
  while (ns > 0) prob[small[--ns]] = 1.0;
  free(small);
  free(large);
  free(w);
  int32_t* a = (int32_t*)malloc((size_t)draws * sizeof(int32_t));
  int32_t* b = (int32_t*)malloc((size_t)draws * sizeof(int32_t));
  if (!a || !b) return NULL;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < draws; ++i) {
    int32_t ends[2];
    for (int k = 0; k < 2; ++k) {
      uint64_t r = rng_u64(seed, 2, (uint64_t)i * 2 + (uint64_t)k);
      int64_t col = (int64_t)((r >> 32) % (uint64_t)n);
      double f = (double)(r & 0xffffffffULL) * (1.0 / 4294967296.0);
      ends[k] = f < prob[col] ? (int32_t)col : alias[col];
    }
    a[i] = ends[0];
    b[i] = ends[1];
  }
  free(prob);
  free(alias);
  return finish(n, draws, a, b, permute, seed);
}

/* Erdos-Renyi G(n, m): exactly m distinct unordered pairs, drawn uniformly by
 * rejection (open-addressing set of pair keys). Requires m <= n(n-1)/2. */
synth_csr* synth_er(int64_t n, int64_t m, uint64_t seed, int permute) {
  if (n < 2 || m > n * (n - 1) / 2) return NULL;
  int64_t cap = 1;
  while (cap < 2 * m + 16) cap <<= 1;
  uint64_t* set = (uint64_t*)malloc((size_t)cap * sizeof(uint64_t));
  int32_t* a = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  int32_t* b = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  if (!set || !a || !b) return NULL;
  memset(set, 0xff, (size_t)cap * sizeof(uint64_t));
  int64_t have = 0;
  for (uint64_t i = 0; have < m; ++i) {
    uint64_t r = rng_u64(seed, 3, i);
    int64_t x = (int64_t)((r >> 32) % (uint64_t)n), y = (int64_t)((r & 0xffffffffULL) % (uint64_t)n);
    if (x == y) continue;
    if (x > y) { int64_t t = x; x = y; y = t; }
    uint64_t key = ((uint64_t)x << 32) | (uint64_t)y;
    uint64_t h = fmix64(key) & (uint64_t)(cap - 1);
    int dup = 0;
    while (set[h] != ~0ULL) {
      if (set[h] == key) { dup = 1; break; }
      h = (h + 1) & (uint64_t)(cap - 1);
    }
    if (dup) continue;
    set[h] = key;
    a[have] = (int32_t)x;
    b[have] = (int32_t)y;
    ++have;
  }
  free(set);
  return finish(n, m, a, b, permute, seed);
}

/* 2-D random geometric graph: n points uniform in the unit square, an edge
 * between every pair at Euclidean distance < r (cell grid of side r). */
synth_csr* synth_rgg(int64_t n, double r, uint64_t seed, int permute) {
  double* px = (double*)malloc((size_t)n * sizeof(double));
  double* py = (double*)malloc((size_t)n * sizeof(double));
  if (!px || !py) return NULL;
  for (int64_t i = 0; i < n; ++i) {
    px[i] = rng_unit(seed, 4, (uint64_t)i * 2);
    py[i] = rng_unit(seed, 4, (uint64_t)i * 2 + 1);
  }
  int64_t g = (int64_t)floor(1.0 / r);
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  int64_t cells = g * g;
  int64_t* head = (int64_t*)calloc((size_t)cells + 1, sizeof(int64_t));
  int64_t* idx = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  int64_t* cell_of = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!head || !idx || !cell_of) return NULL;
  for (int64_t i = 0; i < n; ++i) {
    int64_t cx = (int64_t)(px[i] * (double)g), cy = (int64_t)(py[i] * (double)g);
    if (cx >= g) cx = g - 1;
    if (cy >= g) cy = g - 1;
    cell_of[i] = cy * g + cx;
    head[cell_of[i] + 1]++;
  }
  for (int64_t c = 0; c < cells; ++c) head[c + 1] += head[c];
  int64_t* cur = (int64_t*)malloc((size_t)cells * sizeof(int64_t));
  if (!cur) return NULL;
  memcpy(cur, head, (size_t)cells * sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) idx[cur[cell_of[i]]++] = i;
  free(cur);
  int64_t capE = 1024, e = 0;
  int32_t* a = (int32_t*)malloc((size_t)capE * sizeof(int32_t));
  int32_t* b = (int32_t*)malloc((size_t)capE * sizeof(int32_t));
  if (!a || !b) return NULL;
  double r2 = r * r;
  for (int64_t i = 0; i < n; ++i) {
    int64_t cx = cell_of[i] % g, cy = cell_of[i] / g;
    for (int64_t dy = -1; dy <= 1; ++dy)
      for (int64_t dx = -1; dx <= 1; ++dx) {
        int64_t x = cx + dx, y = cy + dy;
        if (x < 0 || y < 0 || x >= g || y >= g) continue;
        int64_t c = y * g + x;
        for (int64_t p = head[c]; p < head[c + 1]; ++p) {
          int64_t j = idx[p];
          if (j <= i) continue;
          double ddx = px[i] - px[j], ddy = py[i] - py[j];
          if (ddx * ddx + ddy * ddy >= r2) continue;
          if (e == capE) {
            capE *= 2;
            a = (int32_t*)realloc(a, (size_t)capE * sizeof(int32_t));
            b = (int32_t*)realloc(b, (size_t)capE * sizeof(int32_t));
            if (!a || !b) return NULL;
          }
          a[e] = (int32_t)i;
          b[e] = (int32_t)j;
          ++e;
        }
      }
  }
  free(px);
  free(py);
  free(head);
  free(idx);
  free(cell_of);
  return finish(n, e, a, b, permute, seed);
}

/* Arbitrary pair list (e.g. from Python) to CSR, no permutation. */
synth_csr* synth_from_pairs(int64_t n, int64_t e, const int32_t* a, const int32_t* b) {
  return build_csr(n, e, a, b);
}

/* ------------------------------------------------------------ access */

int64_t synth_csr_n(const synth_csr* g) { return g->n; }
int64_t synth_csr_nnz(const synth_csr* g) { return g->nnz; }

void synth_csr_copy(const synth_csr* g, int64_t* row_ptr, int32_t* col) {
  memcpy(row_ptr, g->row_ptr, ((size_t)g->n + 1) * sizeof(int64_t));
  memcpy(col, g->col, (size_t)g->nnz * sizeof(int32_t));
}

void synth_csr_free(synth_csr* g) {
  if (!g) return;
  free(g->row_ptr);
  free(g->col);
  free(g);
}

int synth_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
