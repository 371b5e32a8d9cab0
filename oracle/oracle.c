/*
 * CPU ORACLE -- test infrastructure only.
 *
 * A plain, slow, single-threaded restatement of the paper's edge-centric
 * local counting ("Estimation of Graphlet Statistics", Rossi, Zhou, Ahmed):
 * Algorithm 2 (per-edge triangle / 2-star split with a marker table Phi),
 * Algorithm 3 (4-cliques through the edge) and Algorithm 4 (4-cycles through
 * the edge, read as testing membership of S_v), plus the uniform edge sampler
 * of Algorithm 1 (Bernoulli per edge, SplitMix64 counter hash) and the exact
 * integer sums the estimators consume. Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg may call it; the library never does. It
 * shares no code with the GPU path.
 *
 * Graph: simple undirected, int64 row offsets + int32 sorted adjacency, both
 * orientations stored (the paper's "ordered" neighbour sets, Sec. 2.1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

/* ----------------------------------------------------------------------
 * Per-edge local counts (Algorithm 2 with Algorithms 3 and 4).
 *
 * For each sampled edge e = (v, u) the marker table Phi labels vertices:
 *   L1: neighbours of v other than u (later: S_v)
 *   L3: triangle-closing vertices T_e = N(u) cap N(v)
 *   L2: 2-star vertices of u, S_u = N(u) \ {v} \ N(v)
 * Labels carry an epoch per edge so Phi never needs clearing (the paper's
 * "unique lambda per neighbourhood" trick). u is the endpoint of smaller
 * degree (ties: smaller id), as in the complexity discussion of Sec. 2.5;
 * the counts do not depend on this choice.
 *
 * Outputs per edge j (all int64):
 *   t[j] = |T_e|, a[j] = |S_u|, b[j] = |S_v|,
 *   k[j] = 4-cliques containing e   = unordered adjacent pairs inside T_e,
 *   q[j] = induced 4-cycles with e  = pairs (w in S_u, r in S_v), w ~ r.
 * Returns 0, or -1 if a pair is not an edge of the graph / out of range.
 * ---------------------------------------------------------------------- */
static int local_counts(int64_t n, const int64_t* row_ptr, const int32_t* col, int64_t num_pairs,
                        const int32_t* pairs, int want_four, int literal_alg4, int64_t* t_out,
                        int64_t* a_out, int64_t* b_out, int64_t* k_out, int64_t* q_out) {
  int64_t* phi = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int32_t* tri = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t* star_u = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!phi || !tri || !star_u) return -2;
  int rc = 0;
  for (int64_t j = 0; j < num_pairs; ++j) {
    int64_t x = pairs[2 * j], y = pairs[2 * j + 1];
    if (x < 0 || y < 0 || x >= n || y >= n || x == y) { rc = -1; break; }
    int64_t dx = row_ptr[x + 1] - row_ptr[x], dy = row_ptr[y + 1] - row_ptr[y];
    int64_t u, v;
    if (dx < dy || (dx == dy && x < y)) { u = x; v = y; } else { u = y; v = x; }
    const int64_t L1 = 4 * (j + 1) + 1, L2 = 4 * (j + 1) + 2, L3 = 4 * (j + 1) + 3;
    /* mark N(v) \ {u} with lambda_1 */
    int adjacent = 0;
    for (int64_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
      int64_t w = col[p];
      if (w == u) { adjacent = 1; continue; }
      phi[w] = L1;
    }
    if (!adjacent) { rc = -1; break; }
    /* scan N(u) \ {v}: triangle (lambda_3) or 2-star of u (lambda_2) */
    int64_t nt = 0, na = 0;
    for (int64_t p = row_ptr[u]; p < row_ptr[u + 1]; ++p) {
      int64_t w = col[p];
      if (w == v) continue;
      if (phi[w] == L1) {
        tri[nt++] = (int32_t)w;
        phi[w] = L3;
      } else {
        star_u[na++] = (int32_t)w;
        phi[w] = L2;
      }
    }
    int64_t du = row_ptr[u + 1] - row_ptr[u], dv = row_ptr[v + 1] - row_ptr[v];
    t_out[j] = nt;
    a_out[j] = na; /* = du - 1 - nt */
    b_out[j] = dv - 1 - nt;
    (void)du;
    int64_t kk = 0, qq = 0;
    if (want_four) {
      /* Algorithm 3: for each w in T, count neighbours still labelled
       * lambda_3, then clear w's label so each adjacent pair counts once. */
      for (int64_t i = 0; i < nt; ++i) {
        int64_t w = tri[i];
        for (int64_t p = row_ptr[w]; p < row_ptr[w + 1]; ++p)
          if (phi[col[p]] == L3) ++kk;
        phi[w] = 0;
      }
      /* Algorithm 4 (reading: r must be in S_v, i.e. still lambda_1; the
       * literal test against lambda_2 is kept only so the tests can show
       * that it disagrees with brute-force enumeration). */
      const int64_t want = literal_alg4 ? L2 : L1;
      for (int64_t i = 0; i < na; ++i) {
        int64_t w = star_u[i];
        for (int64_t p = row_ptr[w]; p < row_ptr[w + 1]; ++p)
          if (phi[col[p]] == want) ++qq;
      }
    }
    k_out[j] = kk;
    q_out[j] = qq;
  }
  free(phi);
  free(tri);
  free(star_u);
  return rc;
}

int oracle_local_counts(int64_t n, const int64_t* row_ptr, const int32_t* col, int64_t num_pairs,
                        const int32_t* pairs, int want_four, int64_t* t_out, int64_t* a_out,
                        int64_t* b_out, int64_t* k_out, int64_t* q_out) {
  return local_counts(n, row_ptr, col, num_pairs, pairs, want_four, 0, t_out, a_out, b_out, k_out,
                      q_out);
}

/* Algorithm 4 exactly as printed (tests Phi(r) = lambda_2): a planted
 * mistake for the tests, never used to produce expected values. */
int oracle_local_counts_literal_alg4(int64_t n, const int64_t* row_ptr, const int32_t* col,
                                     int64_t num_pairs, const int32_t* pairs, int64_t* t_out,
                                     int64_t* a_out, int64_t* b_out, int64_t* k_out,
                                     int64_t* q_out) {
  return local_counts(n, row_ptr, col, num_pairs, pairs, 1, 1, t_out, a_out, b_out, k_out, q_out);
}

/* ----------------------------------------------------------------------
 * Per-edge numerators N_i and their exact sums.
 *
 * With sigma = M/K the estimators of Sec. 2.3 (X_3..X_12, weights W) are
 * linear in per-edge terms: X_i = sigma * sum_e N_i(e) / D_i, where
 *   N3 = t                                  D3 = 3
 *   N4 = a + b                              D4 = 2
 *   N7 = k                                  D7 = 6
 *   N8 = C(t,2) - k                         D8 = 1
 *   N9 = t(a+b) - 4 N8                      D9 = 2
 *   N10 = q                                 D10 = 4
 *   N11 = 2[C(a,2)+C(b,2)] - t(a+b) + 4 N8  D11 = 6
 *   N12 = a b - q                           D12 = 1
 * (X9 = (sigma C9 - 4 X8)/2 and X11 = (sigma C11 - X9)/3 expanded per edge.)
 * sums[i] receives sum N_i as a signed 128-bit integer (lo, hi words) and
 * sq[i] receives sum N_i^2 as an unsigned 128-bit integer, i indexing
 * (3,4,7,8,9,10,11,12) as 0..7.
 * ---------------------------------------------------------------------- */
void oracle_numerators(int64_t num, const int64_t* t, const int64_t* a, const int64_t* b,
                       const int64_t* k, const int64_t* q, int64_t* n_out /* [num][8] or NULL */,
                       uint64_t* sums /* [8][2] */, uint64_t* sq /* [8][2] */) {
  i128 s[8];
  u128 s2[8];
  for (int i = 0; i < 8; ++i) { s[i] = 0; s2[i] = 0; }
  for (int64_t j = 0; j < num; ++j) {
    i128 tt = t[j], aa = a[j], bb = b[j], kk = k[j], qq = q[j];
    i128 n8 = tt * (tt - 1) / 2 - kk;
    i128 N[8];
    N[0] = tt;
    N[1] = aa + bb;
    N[2] = kk;
    N[3] = n8;
    N[4] = tt * (aa + bb) - 4 * n8;
    N[5] = qq;
    N[6] = 2 * (aa * (aa - 1) / 2 + bb * (bb - 1) / 2) - tt * (aa + bb) + 4 * n8;
    N[7] = aa * bb - qq;
    for (int i = 0; i < 8; ++i) {
      s[i] += N[i];
      i128 m = N[i] < 0 ? -N[i] : N[i];
      s2[i] += (u128)m * (u128)m;
      if (n_out) n_out[j * 8 + i] = (int64_t)N[i];
    }
  }
  for (int i = 0; i < 8; ++i) {
    u128 us = (u128)s[i];
    sums[2 * i] = (uint64_t)us;
    sums[2 * i + 1] = (uint64_t)(us >> 64);
    sq[2 * i] = (uint64_t)s2[i];
    sq[2 * i + 1] = (uint64_t)(s2[i] >> 64);
  }
}

/* ----------------------------------------------------------------------
 * Uniform edge sampling (Algorithm 1 with a Bernoulli distribution F).
 *
 * The paper leaves the random source open; this oracle fixes it:
 *   sm(x)  = SplitMix64 output for state x (Steele, Lea, Flood 2014):
 *            z = x + 0x9e3779b97f4a7c15;
 *            z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9;
 *            z = (z ^ (z >> 27)) * 0x94d049bb133111eb;
 *            return z ^ (z >> 31);
 *   edge i (the i-th pair u < v in row-major CSR order) is kept iff
 *            (sm(seed ^ sm(i)) >> 11) < threshold,
 *   threshold = floor(p * 2^53) computed by the caller in double precision.
 * Kept edges are written as (u, v) pairs in increasing i. Returns the
 * number kept (all are counted even beyond max_pairs; only max_pairs are
 * written).
 * ---------------------------------------------------------------------- */
uint64_t oracle_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

int64_t oracle_sample(int64_t n, const int64_t* row_ptr, const int32_t* col, uint64_t threshold,
                      uint64_t seed, int32_t* out_pairs, int64_t max_pairs) {
  int64_t kept = 0;
  uint64_t i = 0;
  for (int64_t u = 0; u < n; ++u) {
    for (int64_t p = row_ptr[u]; p < row_ptr[u + 1]; ++p) {
      int64_t v = col[p];
      if (v <= u) continue;
      uint64_t h = oracle_splitmix64(seed ^ oracle_splitmix64(i));
      if ((h >> 11) < threshold) {
        if (kept < max_pairs) {
          out_pairs[2 * kept] = (int32_t)u;
          out_pairs[2 * kept + 1] = (int32_t)v;
        }
        ++kept;
      }
      ++i;
    }
  }
  return kept;
}

/* ----------------------------------------------------------------------
 * Algorithm 7 (micro-level estimation) for each sampled edge.
 *
 * The marker table Phi carries the labels of Algorithm 7:
 *   L1  neighbours of v other than u (S_v, and T until relabelled)
 *   L2  S_u = neighbours of u that are not neighbours of v (not v itself)
 *   L3  T_e = common neighbours of u and v, not yet processed
 *   L4  T_e members already processed by the 4-clique loop
 *   0   an S_u or S_v member already processed (its pairs are counted)
 * Each loop visits its set in increasing vertex id (the sorted neighbour
 * lists), so an unordered pair inside a set is counted once, from its
 * smaller member -- the effect of the paper's resets.
 *
 * Neighbour selection for a vertex w of degree d_w: c_w = ceil(d_w p_e)
 * probes, read as a circular window of c_w consecutive entries of N(w)
 * starting at offset o_w = floor(h d_w / 2^64), h = sm(sm(seed ^ sm(key))
 * ^ w), key = (min(u,v) << 32) | max(u,v), sm = SplitMix64. Every
 * neighbour lies in the window with probability c_w / d_w, so weighting each
 * hit by d_w / c_w (as the algorithm does) is unbiased; p_e = 1 probes every
 * neighbour once and the statistics are exact.
 *
 * Output row j (x3 .. x17, 15 doubles) with t = |T_e|, a = |S_u|,
 * b = |S_v|, R = n - 2 - t - a - b:
 *   x3 = t, x4 = a + b, x5 = R, x6 = C(n,3) - x3 - x4 - x5,
 *   x7 = 4-clique hits (pairs inside T),  x8 = C(t,2) - x7,
 *   x9 = tailed-triangle hits (pairs inside S_u, pairs inside S_v),
 *   x10 = 4-cycle hits (S_u to S_v),
 *   x11 = C(a,2) + C(b,2) - x9,  x12 = a b - x10,
 *   x13 = t R,  x14 = (a + b) R,  x15 = m - (t + d_u + d_v + 1) - omega,
 *   x16 = C(R,2),  x17 = C(n,4) - (x7 + ... + x16),
 * and omega_out[j] = omega (hits from S_u or S_v into T). Weighted hit sums
 * are formed with Neumaier's compensated summation. Returns 0, or -1 if a
 * pair is not an edge.
 * ---------------------------------------------------------------------- */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum* a, double x) {
  double t = a->s + x;
  if ((a->s >= 0 ? a->s : -a->s) >= (x >= 0 ? x : -x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}

static double nsum_value(const nsum* a) { return a->s + a->c; }

static int64_t micro_probes(int64_t d, double pe) {
  double c = ceil((double)d * pe);
  return (int64_t)c;
}

static int64_t micro_offset(uint64_t seed, int64_t x, int64_t y, int64_t w, int64_t d) {
  uint64_t key = ((uint64_t)(x < y ? x : y) << 32) | (uint64_t)(x < y ? y : x);
  uint64_t h = oracle_splitmix64(oracle_splitmix64(seed ^ oracle_splitmix64(key)) ^ (uint64_t)w);
  return (int64_t)(((u128)h * (u128)(uint64_t)d) >> 64);
}

int oracle_micro(int64_t n, int64_t m, const int64_t* row_ptr, const int32_t* col,
                 int64_t num_pairs, const int32_t* pairs, double pe, uint64_t seed,
                 double* x_out, double* omega_out) {
  int64_t* phi = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int32_t* T = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t* Su = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  int32_t* Sv = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!phi || !T || !Su || !Sv) return -2;
  const i128 N = n;
  const i128 cn3 = N * (N - 1) * (N - 2) / 6;
  const i128 cn4 = N * (N - 1) / 2 * (N - 2) * (N - 3) / 12;
  int rc = 0;
  for (int64_t j = 0; j < num_pairs; ++j) {
    int64_t x = pairs[2 * j], y = pairs[2 * j + 1];
    if (x < 0 || y < 0 || x >= n || y >= n || x == y) { rc = -1; break; }
    int64_t dx = row_ptr[x + 1] - row_ptr[x], dy = row_ptr[y + 1] - row_ptr[y];
    int64_t u, v;
    if (dx < dy || (dx == dy && x < y)) { u = x; v = y; } else { u = y; v = x; }
    const int64_t E = 5 * (j + 1);
    const int64_t L1 = E + 1, L2 = E + 2, L3 = E + 3, L4 = E + 4;
    /* mark N(v) \ {u} with L1 */
    int adjacent = 0;
    for (int64_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
      if (col[p] == u) { adjacent = 1; continue; }
      phi[col[p]] = L1;
    }
    if (!adjacent) { rc = -1; break; }
    /* N(u) \ {v}: a triangle (L3) or a 2-star of u (L2) */
    int64_t t = 0, a = 0, b = 0;
    for (int64_t p = row_ptr[u]; p < row_ptr[u + 1]; ++p) {
      int64_t w = col[p];
      if (w == v) continue;
      if (phi[w] == L1) { T[t++] = (int32_t)w; phi[w] = L3; }
      else { Su[a++] = (int32_t)w; phi[w] = L2; }
    }
    for (int64_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p)
      if (col[p] != u && phi[col[p]] == L1) Sv[b++] = col[p];
    const int64_t du = row_ptr[u + 1] - row_ptr[u], dv = row_ptr[v + 1] - row_ptr[v];
    const int64_t R = n - 2 - t - a - b;
    nsum s7 = {0, 0}, s9 = {0, 0}, s10 = {0, 0}, sw = {0, 0};
    /* 4-cliques: probes of N(w) for w in T that land on unprocessed T */
    for (int64_t i = 0; i < t; ++i) {
      const int64_t w = T[i], bw = row_ptr[w], dw = row_ptr[w + 1] - bw;
      const int64_t c = micro_probes(dw, pe), o = micro_offset(seed, x, y, w, dw);
      int64_t h7 = 0;
      for (int64_t q = 0; q < c; ++q)
        if (phi[col[bw + (o + q) % dw]] == L3) ++h7;
      if (h7) nsum_add(&s7, ((double)h7 * (double)dw) / (double)c);
      phi[w] = L4;
    }
    /* S_u: 4-cycles (S_v, L1), tailed triangles (unprocessed S_u, L2) and
     * omega (T, L4) */
    for (int64_t i = 0; i < a; ++i) {
      const int64_t w = Su[i], bw = row_ptr[w], dw = row_ptr[w + 1] - bw;
      const int64_t c = micro_probes(dw, pe), o = micro_offset(seed, x, y, w, dw);
      int64_t h10 = 0, h9 = 0, hw = 0;
      for (int64_t q = 0; q < c; ++q) {
        const int64_t lab = phi[col[bw + (o + q) % dw]];
        if (lab == L1) ++h10;
        if (lab == L2) ++h9;
        if (lab == L4) ++hw;
      }
      if (h10) nsum_add(&s10, ((double)h10 * (double)dw) / (double)c);
      if (h9) nsum_add(&s9, ((double)h9 * (double)dw) / (double)c);
      if (hw) nsum_add(&sw, ((double)hw * (double)dw) / (double)c);
      phi[w] = 0;
    }
    /* S_v: tailed triangles (unprocessed S_v, L1) and omega (T, L4) */
    for (int64_t i = 0; i < b; ++i) {
      const int64_t w = Sv[i], bw = row_ptr[w], dw = row_ptr[w + 1] - bw;
      const int64_t c = micro_probes(dw, pe), o = micro_offset(seed, x, y, w, dw);
      int64_t h9 = 0, hw = 0;
      for (int64_t q = 0; q < c; ++q) {
        const int64_t lab = phi[col[bw + (o + q) % dw]];
        if (lab == L1) ++h9;
        if (lab == L4) ++hw;
      }
      if (h9) nsum_add(&s9, ((double)h9 * (double)dw) / (double)c);
      if (hw) nsum_add(&sw, ((double)hw * (double)dw) / (double)c);
      phi[w] = 0;
    }
    /* clear the remaining labels of this edge (T members) */
    for (int64_t i = 0; i < t; ++i) phi[T[i]] = 0;
    const double x7 = nsum_value(&s7), x9 = nsum_value(&s9), x10 = nsum_value(&s10);
    const double om = nsum_value(&sw);
    double* r = x_out + 15 * j;
    r[0] = (double)t;
    r[1] = (double)(a + b);
    r[2] = (double)R;
    r[3] = (double)(cn3 - t - (a + b) - R);
    r[4] = x7;
    r[5] = (double)(t * (t - 1) / 2) - x7;
    r[6] = x9;
    r[7] = x10;
    r[8] = (double)(a * (a - 1) / 2 + b * (b - 1) / 2) - x9;
    r[9] = (double)(a * b) - x10;
    r[10] = (double)((i128)t * R);
    r[11] = (double)((i128)(a + b) * R);
    r[12] = (double)(m - (t + du + dv + 1)) - om;
    r[13] = (double)((i128)R * (R - 1) / 2);
    double s = 0.0;
    for (int i = 4; i <= 13; ++i) s += r[i];
    r[14] = (double)cn4 - s;
    if (omega_out) omega_out[j] = om;
  }
  free(phi);
  free(T);
  free(Su);
  free(Sv);
  return rc;
}

/* ----------------------------------------------------------------------
 * k-core numbers (the weights of the k-core sampling distribution of
 * Sec. 3.1 / Sec. 7): core[v] = the largest k such that v belongs to a
 * subgraph whose every vertex has degree >= k. Bucket peeling of Batagelj
 * and Zaversnik (2003): vertices in buckets by current degree; repeatedly
 * remove a vertex of least current degree, its core number is that degree
 * (never below the previous one), and move each later neighbour one bucket
 * down.
 * ---------------------------------------------------------------------- */
void oracle_core_numbers(int64_t n, const int64_t* row_ptr, const int32_t* col, int32_t* core) {
  if (n <= 0) return;
  int64_t maxd = 0;
  int64_t* deg = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  for (int64_t v = 0; v < n; ++v) {
    deg[v] = row_ptr[v + 1] - row_ptr[v];
    if (deg[v] > maxd) maxd = deg[v];
  }
  int64_t* bin = (int64_t*)calloc((size_t)(maxd + 2), sizeof(int64_t));
  int64_t* pos = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  int64_t* vert = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  for (int64_t v = 0; v < n; ++v) bin[deg[v]]++;
  int64_t start = 0;
  for (int64_t d = 0; d <= maxd; ++d) {
    int64_t num = bin[d];
    bin[d] = start;
    start += num;
  }
  for (int64_t v = 0; v < n; ++v) {
    pos[v] = bin[deg[v]];
    vert[pos[v]] = v;
    bin[deg[v]]++;
  }
  for (int64_t d = maxd; d >= 1; --d) bin[d] = bin[d - 1];
  bin[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t v = vert[i];
    core[v] = (int32_t)deg[v];
    for (int64_t p = row_ptr[v]; p < row_ptr[v + 1]; ++p) {
      int64_t x = col[p];
      if (deg[x] > deg[v]) {
        int64_t dx = deg[x], px = pos[x], pw = bin[dx], w = vert[pw];
        if (x != w) {  /* swap x with the first vertex of its bucket */
          pos[x] = pw;
          vert[px] = w;
          pos[w] = px;
          vert[pw] = x;
        }
        bin[dx]++;
        deg[x]--;
      }
    }
  }
  free(deg);
  free(bin);
  free(pos);
  free(vert);
}

/* ----------------------------------------------------------------------
 * Weighted edge sampling (Algorithm 1 with a non-uniform distribution F,
 * Sec. 3.1: "k-core numbers, degrees, or any attribute of interest").
 * Edge weight w_e = min(vw[u], vw[v]) (for core numbers: the edge's own
 * core number); W = sum of w_e over the edges; each canonical edge i is
 * kept independently with probability pi_e = min(1, s w_e), s = fraction
 * M / W, by the sampler key of oracle_sample:
 *   keep iff (sm(seed ^ sm(i)) >> 11) < floor(pi_e 2^53).
 * Writes the kept pairs (u < v, increasing i) and their weights; returns
 * the number kept (at most max_pairs written). *scale_out = s.
 * ---------------------------------------------------------------------- */
int64_t oracle_sample_weighted(int64_t n, const int64_t* row_ptr, const int32_t* col,
                               const int32_t* vw, double fraction, uint64_t seed,
                               int32_t* out_pairs, int32_t* out_w, int64_t max_pairs,
                               double* scale_out) {
  int64_t m = 0, W = 0;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t p = row_ptr[u]; p < row_ptr[u + 1]; ++p) {
      int64_t v = col[p];
      if (v <= u) continue;
      ++m;
      W += vw[u] < vw[v] ? vw[u] : vw[v];
    }
  const double s = W > 0 ? fraction * (double)m / (double)W : 0.0;
  *scale_out = s;
  int64_t kept = 0;
  uint64_t i = 0;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t p = row_ptr[u]; p < row_ptr[u + 1]; ++p) {
      int64_t v = col[p];
      if (v <= u) continue;
      const int32_t we = vw[u] < vw[v] ? vw[u] : vw[v];
      double pi = s * (double)we;
      if (pi > 1.0) pi = 1.0;
      const uint64_t threshold = (uint64_t)floor(pi * 9007199254740992.0);
      const uint64_t h = oracle_splitmix64(seed ^ oracle_splitmix64(i));
      if ((h >> 11) < threshold) {
        if (kept < max_pairs) {
          out_pairs[2 * kept] = (int32_t)u;
          out_pairs[2 * kept + 1] = (int32_t)v;
          out_w[kept] = we;
        }
        ++kept;
      }
      ++i;
    }
  return kept;
}
