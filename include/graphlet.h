/*
 * graphlet.h -- C ABI of libgraphlet, a GB300 (sm_103a) implementation of
 * the edge-centric graphlet estimator of Rossi, Zhou and Ahmed, "Estimation
 * of Graphlet Statistics".
 *
 * The library counts, around each sampled edge e = (u, v) of a simple
 * undirected graph, the connected 3- and 4-node graphlets that contain e
 * (Algorithm 2: triangles T_e and 2-stars S_u, S_v; Algorithm 3: 4-cliques;
 * Algorithm 4: 4-cycles), folds the per-edge counts into exact integer sums
 * and turns them into the unbiased estimates of Sec. 2.3 with a variance and
 * 95% bounds (Sec. 6.2).
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA global-memory pointers on the current device;
 *     host pointers are ordinary CPU memory. Each argument says which.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Work is enqueued on it; calls that return host results
 *     synchronise that stream before returning.
 *   - The caller owns every pointer it passes; the library never frees or
 *     retains caller memory beyond the call, except the CSR arrays given to
 *     gs_graph_create, which must stay valid until gs_graph_destroy.
 *   - Every call returns a gs_status. On failure gs_last_error() returns a
 *     message for the calling thread; outputs are then unspecified.
 *   - Graph ids are int32; row offsets int64; edge counts int64.
 *   - Graphlets are named by the paper's index G_i (Table 1). Connected ones
 *     handled here: G3 triangle, G4 2-star, G7 4-clique, G8 chordal-cycle,
 *     G9 tailed-triangle, G10 4-cycle, G11 3-star, G12 4-path. Arrays of 8
 *     per-graphlet values use the order (3, 4, 7, 8, 9, 10, 11, 12).
 */
#ifndef GRAPHLET_H
#define GRAPHLET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gs_status;
enum {
  GS_OK = 0,
  GS_EINVAL = 1,       /* bad argument (null pointer, negative size, bad mask, ...) */
  GS_ENOTSORTED = 2,   /* an adjacency list is not strictly increasing */
  GS_ESELFLOOP = 3,    /* a vertex lists itself */
  GS_EDUP = 4,         /* an adjacency list repeats a neighbour */
  GS_EASYM = 5,        /* u lists v but v does not list u */
  GS_EEDGE = 6,        /* a sampled pair is out of range or not an edge */
  GS_EDUPSAMPLE = 7,   /* an explicit sample lists the same edge twice */
  GS_EOVERFLOW = 8,    /* a value does not fit its output type */
  GS_ENOMEM = 9,       /* device allocation failed */
  GS_EBUDGET = 10,     /* request exceeds a configured memory budget */
  GS_ETIMEOUT = 11,    /* a bounded device-side wait expired */
  GS_ECUDA = 12,       /* a CUDA runtime call failed (message has details) */
  GS_ECAPACITY = 13,   /* an output buffer is too small (size is reported) */
  GS_ECANCELLED = 14   /* a queued request was dropped by gs_server_destroy */
};

/* Graphlet mask: bit i set = graphlet G_i requested. */
#define GS_G3 (1u << 3)
#define GS_G4 (1u << 4)
#define GS_G7 (1u << 7)
#define GS_G8 (1u << 8)
#define GS_G9 (1u << 9)
#define GS_G10 (1u << 10)
#define GS_G11 (1u << 11)
#define GS_G12 (1u << 12)
#define GS_THREE_NODE (GS_G3 | GS_G4)
#define GS_CONNECTED (GS_G3 | GS_G4 | GS_G7 | GS_G8 | GS_G9 | GS_G10 | GS_G11 | GS_G12)

/* gs_graph_create flags */
#define GS_VALIDATE 1u  /* check sorted / simple / symmetric CSR on the device */

/* Per-graphlet result flags */
#define GS_F_COMPUTED 1u        /* graphlet was in the mask */
#define GS_F_EXACT 2u           /* every edge sampled: exact[] is valid, V = 0 */
#define GS_F_VAR_UNDEFINED 4u   /* fewer than 2 sampled edges: V, lb, ub are NaN */
#define GS_F_OVERFLOW 8u        /* exact count does not fit uint64 */
#define GS_F_VAR_OVERFLOW 16u   /* a sum of squares exceeded 128 bits: V, lb, ub are NaN */

/* Exact integer sums over the sampled edges J (Sec. 2.3, Alg. 2 accumulators).
 * For each graphlet i the per-edge numerator N_i(e) is the integer with
 * X_i = (M / K) * sum_e N_i(e) / D_i, D = (3, 2, 6, 1, 2, 4, 6, 1):
 *   N3 = t, N4 = a + b, N7 = k, N8 = C(t,2) - k, N9 = t(a+b) - 4 N8,
 *   N10 = q, N11 = 2[C(a,2) + C(b,2)] - t(a+b) + 4 N8, N12 = a b - q,
 * with t = |T_e|, a = |S_u|, b = |S_v|, k = 4-cliques through e,
 * q = 4-cycles through e. sum[i] is a signed 128-bit integer stored as
 * (low word, high word); sumsq[i] = sum N_i^2 as an unsigned 128-bit value. */
typedef struct {
  int64_t k;            /* number of sampled edges |J| */
  int64_t m;            /* number of edges of the graph |E| */
  uint32_t mask;        /* graphlets computed */
  uint32_t reserved;
  uint64_t sum[8][2];
  uint64_t sumsq[8][2];
} gs_sums;

/* Estimates per graphlet, in the order (3, 4, 7, 8, 9, 10, 11, 12). */
typedef struct {
  double x[8];          /* X_i, Sec. 2.3 estimators with sigma = M / K */
  double var[8];        /* estimated Var[X_i] (see gs_estimate) */
  double lb[8];         /* X_i - z sqrt(var) (Sec. 6.2) */
  double ub[8];         /* X_i + z sqrt(var) */
  uint64_t exact[8];    /* sum N_i / D_i when K = M (flag GS_F_EXACT) */
  uint32_t flags[8];    /* GS_F_* */
} gs_result;

typedef struct gs_graph gs_graph;
typedef struct gs_workspace gs_workspace;

/* Thread-local message describing the last failure of this thread. */
const char* gs_last_error(void);

/* Library version string. */
const char* gs_version(void);

/* Registers a simple undirected graph given as CSR (Sec. 2.1: ordered
 * neighbour sets). d_row_ptr: device int64[n+1], d_col: device int32[nnz],
 * nnz = 2|E|, every list strictly increasing, both orientations present, no
 * self-loops. The arrays are borrowed (not copied) and must outlive the
 * handle. With GS_VALIDATE the structure is checked on the device and
 * GS_ENOTSORTED / GS_ESELFLOOP / GS_EDUP / GS_EASYM / GS_EINVAL returned.
 * Builds the per-graph index (upper-edge offsets for the sampler, adjacency
 * bitmaps of the highest-degree vertices, an adjacency bit matrix among the
 * top 32767 of them with, per vertex, the matrix slots of its matrix
 * neighbours and its neighbours above it outside the matrix, a co-degree
 * table |N(a) cap N(b)| among the top vertices, plus a mid x big co-degree
 * table, adjacency bucket directories and degree-oriented adjacency lists
 * for the exact 3-node pass, see gs_graph_index_info) in library-owned
 * device memory;
 * hub_budget_bytes bounds that index (0 = default 96 GiB, a third of the
 * GPU, for one large resident graph; pass less when several graphs share
 * the device): bitmaps and matrix up to 1/8 each, directories up to 1/16,
 * the 16-bit co-degree table most of the rest (at most 65535 vertices), the
 * mid x big table and a table slot per adjacency entry whatever remains.
 * The budget is an upper bound: a small graph's index stays small.
 * Synchronises `stream`. */
gs_status gs_graph_create(const int64_t* d_row_ptr, const int32_t* d_col, int64_t n, int64_t nnz,
                          uint32_t flags, uint64_t hub_budget_bytes, void* stream,
                          gs_graph** out);

/* Frees the library-owned per-graph index. The CSR arrays are not freed. */
gs_status gs_graph_destroy(gs_graph* g);

/* Host outputs: vertex count, undirected edge count, maximum degree, number
 * of hub vertices with adjacency bitmaps and with co-degree table rows. Any
 * output pointer may be NULL. */
gs_status gs_graph_info(const gs_graph* g, int64_t* n, int64_t* m, int64_t* max_degree,
                        int64_t* bitmap_hubs, int64_t* table_hubs);

/* Host outputs describing the rest of the per-graph index: the number of
 * vertices in the hub-pair bit matrix, the shape of the mid x big
 * co-degree table (16-bit |N(a) cap N(b)| for "mid" vertices a, the
 * highest-degree vertices below the co-degree table's threshold, against
 * "big" vertices b, the top table vertices; 0 rows when it was not built),
 * and the number of vertices whose adjacency list has a bucket directory
 * (offsets of the neighbours by the high bits of their ids, so that a
 * membership test reads one directory entry and a few neighbours instead of
 * halving the whole list). Any output pointer may be NULL. */
gs_status gs_graph_index_info(const gs_graph* g, int64_t* matrix_hubs, int64_t* mid_rows,
                              int64_t* big_hubs, int64_t* dir_vertices);

/* Library-owned scratch for gs_sample / gs_count. One workspace serves one
 * stream at a time; it grows on demand (cudaMalloc, after synchronising the
 * stream it was last used on) and is released by gs_workspace_destroy. */
gs_status gs_workspace_create(gs_workspace** out);
gs_status gs_workspace_destroy(gs_workspace* ws);
/* Host output: bytes currently held by the workspace. */
gs_status gs_workspace_bytes(const gs_workspace* ws, uint64_t* bytes);

/* Uniform edge sampling (Algorithm 1 with a Bernoulli distribution):
 * canonical edge i (the i-th pair u < v in row-major CSR order) is kept iff
 * (sm(seed ^ sm(i)) >> 11) < floor(fraction * 2^53), sm = SplitMix64 output
 * function. Kept edges are written in increasing i to d_pairs (device
 * int32[2*max_k], (u, v) with u < v). *k_out (host) receives the number
 * kept; GS_ECAPACITY if it exceeds max_k (then nothing useful is written).
 * fraction must lie in [0, 1]. Synchronises `stream`. */
gs_status gs_sample(const gs_graph* g, gs_workspace* ws, double fraction, uint64_t seed,
                    int32_t* d_pairs, int64_t max_k, int64_t* k_out, void* stream);

/* Local counting over a sampled edge set J (Algorithms 2-4) and exact
 * folding of the per-edge numerators into *h_sums (host).
 * d_pairs: device int32[2*k], each pair an edge in either orientation, no
 * edge twice (GS_EDUPSAMPLE); NULL with k = |E| means J = all edges. k = 0
 * is an empty sample (d_pairs not read; all sums zero).
 * mask: graphlets wanted (GS_* bits); 4-clique work runs only if G7, G8,
 * G9 or G11 is set, 4-cycle work only if G10 or G12 is set.
 * d_per_edge: optional device int64[3*k]; receives (t, k, q) per pair in
 * input order (k, q are 0 when their pass did not run).
 * Synchronises `stream`. */
gs_status gs_count(const gs_graph* g, gs_workspace* ws, const int32_t* d_pairs, int64_t k,
                   uint32_t mask, int64_t* d_per_edge, gs_sums* h_sums, void* stream);

/* Estimates from exact sums (host only, no GPU work):
 *   X_i   = (M / K) * sum N_i / D_i                  (Sec. 2.3, sigma = |E|/|J|)
 *   var_i = M (M - K) (K sumsq_i - sum_i^2) / (K^2 (K - 1) D_i^2)
 *           -- the without-replacement design variance of the expansion
 *           estimator; the paper states bounds from Var[X] (Sec. 6.2) but
 *           prints no formula for it, this is the library's choice.
 *   lb_i, ub_i = X_i -/+ z sqrt(var_i), z = 1.96 for 95% (Sec. 6.2).
 * K = M gives var = 0 and exact counts. */
gs_status gs_estimate(const gs_sums* s, double z, gs_result* out);

/* Work statistics and device timings of the last gs_count on a workspace.
 * model_bytes is the streaming cost model of the method: per sampled edge
 *   B(e) = 24 + 4 (d_u + d_v)                         (pair, offsets, Alg. 2)
 *        + [4-clique pass]  sum_{w in T_e} (8 + 4 d_w)            (Alg. 3)
 *        + [4-cycle pass]   min over the two sides of
 *                           sum_{w in S_side} (8 + 4 d_w)        (Alg. 4)
 * i.e. the bytes of every adjacency list Algorithms 2-4 scan. The kernels
 * read fewer bytes than that (searches, hub bitmaps, co-degree table). */
typedef struct {
  int64_t k;              /* sampled edges counted */
  int64_t tri_tests;      /* membership tests of the triangle pass (sum d_u) */
  int64_t quad_tests;     /* membership tests of the 4-node pass (plus the
                             128-bit matrix-row groups of the dense edges) */
  int64_t t_sum;          /* sum over J of |T_e| */
  int64_t tasks;          /* 4-node work units (task_probes tests each, default 512) */
  uint64_t model_bytes;   /* sum over J of B(e) */
  uint64_t model_tri_bytes;  /* the 24 + 4 (d_u + d_v) part (triangle pass) */
  uint64_t model_quad_bytes; /* the 4-clique + 4-cycle part (4-node pass) */
  int64_t launches;       /* kernels launched by that call */
  int64_t launches_total; /* kernels launched through this workspace so far */
  int32_t timed;          /* 1 if the ms_* fields below are valid */
  float ms_prep, ms_tri, ms_compact, ms_cost, ms_quad, ms_fold; /* device ms per phase */
  int64_t dense_edges;    /* sampled edges whose pairs of hub-matrix members in T
                             were counted word-parallel (matrix row AND T mask) */
  int64_t dense_groups;   /* 128-bit matrix-row groups ANDed for those edges
                             (groups where T's mask is non-zero; included in
                             quad_tests) */
  int64_t micro_probes;   /* gs_micro only: neighbour probes, sum of ceil(d_w p_e) */
} gs_stats;

/* Turns per-phase CUDA-event timing of gs_count on (1) or off (0). Events are
 * recorded on the call's stream around each phase. */
gs_status gs_workspace_set_timing(gs_workspace* ws, int enable);

/* Launch choices for gs_count on this workspace (the batched path's
 * autotuner searches the same knobs): resident CTAs per SM of the triangle
 * pass (1..8) and of the 4-node pass (1..8), membership tests per 4-node
 * work unit (32..2^20), and use_hubs = 0 to ignore the per-graph index
 * (bitmaps, co-degree tables, hub-pair matrix, bucket directories).
 * Without a call the defaults are 8, 8, 512, 1. Results do not depend on
 * them. */
gs_status gs_workspace_set_tuning(gs_workspace* ws, int tri_blocks_per_sm, int quad_blocks_per_sm,
                                  int64_t task_probes, int use_hubs);

/* Dense clique mode on this workspace (Sec. 2.6 counts the 4-cliques of an
 * edge from the pairs among T = N(u) cap N(v)): an edge whose T holds many
 * of the graph's highest-degree vertices counts the pairs among those
 * vertices by AND + popcount over rows of the hub-pair bit matrix. `slots`
 * is how many matrix slots (vertices in decreasing degree order) take part;
 * it is rounded down to a multiple of 128 and capped at the matrix size,
 * and 0 turns dense mode off. Vertices of the matrix beyond `slots` still
 * answer single membership tests from it. Default: all (32767). Results do not
 * depend on it; GS_EINVAL for a NULL workspace or slots < 0. Kept across
 * gs_workspace_set_tuning. */
gs_status gs_workspace_set_dense_slots(gs_workspace* ws, int64_t slots);

/* Host output: statistics of the last gs_count that used `ws`. */
gs_status gs_count_stats(const gs_workspace* ws, gs_stats* out);

/* Sample size for a target error (Sec. 6.2: K = (z sqrt(Var[X]) / margin)^2),
 * from a pilot sample's exact sums (host only): with the per-edge sample
 * variance S^2 = (k sumsq - sum^2) / (k (k - 1) D^2) of y = N / D, the
 * pilot estimate X and the margin h = rel_err |X| (the paper's margin read
 * as a relative error of the estimate),
 *   n0 = (z m S / h)^2,  K = ceil(n0 / (1 + n0 / m))
 * (the finite-population correction of sampling without replacement),
 * clamped to [1, m]. k_out (host int64[8], graphlet order of gs_sums):
 * -1 outside the mask or when the pilot has fewer than 2 edges; the pilot
 * size when its per-edge values do not vary; m when X = 0 but they do.
 * Evaluated in FP64. */
gs_status gs_sample_size(const gs_sums* s, double z, double rel_err, int64_t* k_out);

/* Algorithm 8 (adaptive estimation): grows the sampled edge set until the
 * estimates stop moving. Iteration t adds K_t = ceil(phi_t (m - |J|)) edges
 * drawn uniformly without replacement from those not yet sampled -- the
 * next K_t edges in the order of gs_sample's sampler keys, so J is always
 * the |J| smallest keys (gs_sample_fixed(|J|, seed)) -- counts only those
 * (mask as in gs_count), merges their exact sums into the running ones and
 * re-estimates; phi_{t+1} = phi_t / 2. The loss is the maximum relative
 * change max_i |X_i^(t) - X_i^(t-1)| / |X_i^(t-1)| over the 4-node
 * graphlets of the mask (the objective of Sec. 4 takes its maximum over
 * G^(4); a mask with none uses its 3-node graphlets); an unchanged estimate
 * counts 0 (also 0 -> 0), a change away from 0 counts as infinite. The
 * first iteration has loss 1. The loop stops when the loss is at most
 * beta (0 <= beta < 1; the first iteration always runs) or after t_max
 * iterations. phi <= 0 selects phi_1 = 1 / sqrt(m).
 * Outputs (host): the running sums, their estimates (z as gs_estimate),
 * the iterations run and the final sampled fraction |J| / m. The result
 * equals gs_count over gs_sample_fixed(|J|, seed).
 * Synchronises `stream`. */
gs_status gs_count_adaptive(const gs_graph* g, gs_workspace* ws, double beta, int32_t t_max,
                            double phi, uint64_t seed, uint32_t mask, double z,
                            gs_sums* sums_out, gs_result* out, int32_t* iters_out,
                            double* fraction_out, void* stream);

/* ---- disconnected graphlets (G5, G6, G13-G17) --------------------------
 * Sec. 2.3's estimators of the disconnected 3- and 4-node graphlets, read
 * with corrected terms (the printed block swaps C13 with C14 and C15 with
 * C16 and its weights do not match): with R_e = n - 2 - t - a - b (vertices
 * adjacent to neither end of e) and C16_e = m - d_u - d_v + 1 (edges
 * touching neither end), X5 = sigma sum R, X13 = (sigma sum tR - X9) / 3,
 * X14 = sigma sum (a+b)R / 2 - X12, X15 = sigma sum C16 / 2 - 3 X7 - 2 X8 -
 * X9 - 2 X10 - X12, X16 = sigma sum C(R,2) - 2 X15, X6 = C(n,3) - X3 - X4 -
 * X5, X17 = C(n,4) - (X7 + ... + X16); sigma = m / k. Each is a linear
 * expansion estimator (plus a constant for X6, X17) of one per-edge integer
 * numerator, which these calls fold exactly:
 *   N5 = R                         D = 1
 *   N6 = 2t + 3(a+b) + 6R          D = 6    X6 = C(n,3) - sigma sum N6 / 6
 *   N13 = 2tR - N9                 D = 6
 *   N14 = (a+b)R - 2 N12           D = 2
 *   N15 = C16 - N7 - 4N8 - N9 - N10 - 2 N12             D = 2
 *   N16 = C(R,2) - N15             D = 1
 *   N17 = 2N7 + 12N8 + 6N9 + 3N10 + 2N11 + 12N12 + 2N13 + 6N14 + 6N15 + 12N16
 *                                  D = 12   X17 = C(n,4) - sigma sum N17 / 12
 * (N7..N12 as in gs_estimate). The paper has no variance for these either;
 * gs_estimate's SRSWOR reading is applied to each numerator. */
typedef struct {
  int64_t k, m, n;      /* sampled edges, graph edges, graph vertices */
  uint32_t overflow;    /* bit i: sum of squares i exceeded 128 bits (variance NaN) */
  uint32_t reserved;
  uint64_t sum[7][2];   /* order (5, 6, 13, 14, 15, 16, 17), 128-bit two's complement */
  uint64_t sumsq[7][2]; /* sum N_i^2, 128-bit unsigned */
} gs_sums_disc;

typedef struct {
  double x[7], var[7], lb[7], ub[7];  /* order (5, 6, 13, 14, 15, 16, 17) */
  uint64_t exact[7];    /* exact counts when k = m (flag GS_F_EXACT) */
  uint32_t flags[7];    /* GS_F_* */
} gs_result_disc;

/* Folds the disconnected numerators of the sampled edges d_pairs (device
 * int32[2k], the list given to gs_count, any orientation) from the per-edge
 * (t, k, q) that gs_count wrote to d_per_edge (device int64[3k]) for the
 * same list with a mask holding every connected 4-node graphlet
 * (GS_CONNECTED). For all edges, pass the list gs_sample writes at
 * fraction 1. Results in *h_out (host). Uses the workspace's scratch;
 * synchronises `stream`. */
gs_status gs_count_disconnected(const gs_graph* g, gs_workspace* ws, const int32_t* d_pairs,
                                int64_t k, const int64_t* d_per_edge, gs_sums_disc* h_out,
                                void* stream);

/* Per-edge numerators (micro-level output): row e of d_out (device
 * int64[8k]) receives (N3, N4, N7, N8, N9, N10, N11, N12) of sampled edge e
 * (the numerators of gs_estimate; t, a+b, k, C(t,2) - k, q and ab - q are
 * also Algorithm 7's exact per-edge statistics x3, x4, x7, x8, x10, x12),
 * from the per-edge (t, k, q) that gs_count wrote for the same list with
 * mask GS_CONNECTED (N9 and N11 can be negative). The rows sum to
 * gs_count's sums. Synchronises `stream`. */
gs_status gs_per_edge_numerators(const gs_graph* g, gs_workspace* ws, const int32_t* d_pairs,
                                 int64_t k, const int64_t* d_per_edge, int64_t* d_out,
                                 void* stream);

/* Micro-level estimation (Algorithm 7): for every sampled edge e = (u, v)
 * (d_pairs: device int32[2k], each pair an edge in either orientation, no
 * edge twice) the per-edge statistics x3 .. x17 of the paper's micro-level
 * problem, written as row e of d_x (device double[15k]). u is the endpoint
 * of smaller degree (ties: smaller id); T = N(u) cap N(v), S_u, S_v the
 * rest of N(u) \ {v}, N(v) \ {u}; t, a, b their sizes, R = n - 2 - t - a - b.
 * Every w in T, S_u and S_v probes c_w = ceil(d_w p_e) consecutive entries
 * of N(w), a circular window from offset floor(h d_w / 2^64), h =
 * sm(sm(seed ^ sm(key)) ^ w), key = (min(u,v) << 32) | max(u,v) (sm =
 * SplitMix64), each probe landing in the tested set adding d_w / c_w
 * (every neighbour is in the window with probability c_w / d_w, so the
 * weighted counts are unbiased; 0 < p_e <= 1, p_e = 1 probes every
 * neighbour once and gives exact counts):
 *   x7  = probes from T into T above the prober      (4-cliques with e)
 *   x9  = probes from S_u into S_u above the prober and from S_v into S_v
 *         above the prober            (tailed triangles with e as tail)
 *   x10 = probes from S_u into S_v                   (4-cycles with e)
 *   omega = probes from S_u or S_v into T   (diamonds with e on the rim)
 * and, as printed in Algorithm 7 (x5 with the sign of R, x11 over S_u and
 * S_v): x3 = t, x4 = a + b, x5 = R, x6 = C(n,3) - x3 - x4 - x5,
 * x8 = C(t,2) - x7, x11 = C(a,2) + C(b,2) - x9, x12 = ab - x10, x13 = tR,
 * x14 = (a+b)R, x15 = m - (t + d_u + d_v + 1) - omega, x16 = C(R,2),
 * x17 = C(n,4) - (x7 + ... + x16) (x6, x17 rounded to FP64).
 * Weighted probe sums are accumulated exactly in fixed point (2^-64) and
 * rounded once. h_max / h_argmax (host double[15] / int64[15], either may
 * be NULL) receive the largest value of each statistic over the sample and
 * the first edge that has it: Sec. 7's extremal statistic Z_j = max_e x_j(e).
 * gs_count_stats then reports micro_probes. Synchronises `stream`. */
gs_status gs_micro(const gs_graph* g, gs_workspace* ws, const int32_t* d_pairs, int64_t k,
                   double p_e, uint64_t seed, double* d_x, double* h_max, int64_t* h_argmax,
                   void* stream);

/* Uniform sample of exactly k distinct edges (Algorithm 1 with a sample
 * size, without replacement; Algorithm 8 draws its iterations this way):
 * the k canonical edges with the smallest (key, i), key = gs_sample's
 * 53-bit sampler key (sm(seed ^ sm(i)) >> 11), found by a radix select on
 * the device. Every k-subset is equally likely, the samples of one seed
 * are nested in k, and they are nested with gs_sample's Bernoulli samples
 * of the same seed. Writes d_pairs (device int32[2k], (u, v), u < v,
 * increasing i); 0 <= k <= m. Synchronises `stream`. */
gs_status gs_sample_fixed(const gs_graph* g, gs_workspace* ws, int64_t k, uint64_t seed,
                          int32_t* d_pairs, void* stream);

/* The edges ranked [k_lo, k_hi) by gs_sample's sampler key (ties by
 * canonical index), written in increasing canonical index to d_pairs
 * (device int32[2 (k_hi - k_lo)]): the edges gs_sample_fixed(k_hi) adds to
 * gs_sample_fixed(k_lo), so a sample can be grown without replacement by
 * any number of edges. 0 <= k_lo <= k_hi <= m. Synchronises `stream`. */
gs_status gs_sample_ranks(const gs_graph* g, gs_workspace* ws, int64_t k_lo, int64_t k_hi,
                          uint64_t seed, int32_t* d_pairs, void* stream);

/* ---- weighted sampling (Sec. 3.1's weighted distribution F) ------------
 * k-core numbers: d_core (device int32[n]) receives the largest k such that
 * v lies in a subgraph whose every vertex has degree >= k (the weights of
 * the k-core distribution that Sec. 7 uses for the extremal problem);
 * *h_max_core (host, may be NULL) the largest. Parallel peeling; uses the
 * workspace; synchronises `stream`. */
gs_status gs_core_numbers(const gs_graph* g, gs_workspace* ws, int32_t* d_core,
                          int32_t* h_max_core, void* stream);

/* Weighted edge sampling (Algorithm 1 with a non-uniform F): with vertex
 * weights d_vertex_w (device int32[n], >= 0; e.g. gs_core_numbers' output or
 * the degrees) every edge e = (u, v) has weight w_e = min(w_u, w_v) and is
 * kept independently with probability pi_e = min(1, s w_e),
 * s = fraction m / sum_e w_e (so about fraction m edges are kept when no
 * pi_e reaches 1), by the key of gs_sample: canonical edge i is kept iff
 * (sm(seed ^ sm(i)) >> 11) < floor(pi_e 2^53). Equal weights give
 * gs_sample's uniform sample. Kept edges go to d_pairs (device int32[2 max_k],
 * (u, v), u < v, increasing i) and their w_e to d_pair_w (device
 * int32[max_k], may be NULL); *k_out and *scale_out = s (host).
 * GS_ECAPACITY if more than max_k are kept; GS_EINVAL for a negative weight
 * or no positive edge weight. Synchronises `stream`. */
gs_status gs_sample_weighted(const gs_graph* g, gs_workspace* ws, const int32_t* d_vertex_w,
                             double fraction, uint64_t seed, int32_t* d_pairs, int32_t* d_pair_w,
                             int64_t max_k, int64_t* k_out, double* scale_out, void* stream);

/* Estimates from a weighted sample (d_pairs, k as gs_count; d_vertex_w and
 * scale as given to / returned by gs_sample_weighted): the paper's inverse
 * sampling probability taken per edge, sigma_e = 1 / pi_e with
 * pi_e = min(1, scale w_e) (Horvitz-Thompson):
 *   x_i   = sum_e N_i(e) / (D_i pi_e)
 *   var_i = sum_e (1 - pi_e) N_i(e)^2 / (D_i^2 pi_e^2)   (independent
 *           inclusions; unbiased for Var[x_i])
 *   lb_i, ub_i = x_i -/+ z sqrt(var_i)
 * with N_i, D_i as in gs_sums. The per-edge numerators are summed exactly
 * per weight class on the device (every sampled edge needs 1 <= w_e < 2^22)
 * and the classes are combined in FP64 on the host in increasing weight.
 * When every edge is sampled with pi_e = 1 the counts are exact (flag
 * GS_F_EXACT, exact[] valid). Synchronises `stream`. */
gs_status gs_count_weighted(const gs_graph* g, gs_workspace* ws, const int32_t* d_pairs, int64_t k,
                            const int32_t* d_vertex_w, double scale, uint32_t mask, double z,
                            gs_result* out, void* stream);

/* Host FP64 estimates, variances and bounds of G5, G6, G13-G17 from the
 * folded sums (formulas above; var and bounds as in gs_estimate; exact
 * counts when k = m, with GS_F_OVERFLOW when a count does not fit uint64). */
gs_status gs_estimate_disconnected(const gs_sums_disc* s, double z, gs_result_disc* out);

/* gs_sums_merge for the disconnected sums (host only): acc += part; both
 * from the same graph (m, n), disjoint samples. */
gs_status gs_sums_disc_merge(gs_sums_disc* acc, const gs_sums_disc* part);

/* Exact merge of the sums of disjoint shards of one sample (host only):
 * acc += part. Splitting J across GPUs and merging their sums gives the
 * same result as counting J on one GPU (the only exchange the path needs;
 * the paper's distributed scheme sends one count vector per worker, Sec. 5).
 * Both must have the same graph edge count m and mask. */
gs_status gs_sums_merge(gs_sums* acc, const gs_sums* part);

/* Convenience: gs_sample (fraction < 1) or all edges (fraction == 1), then
 * gs_count and gs_estimate. *k_out (host, may be NULL) receives |J|. */
gs_status gs_count_estimate(const gs_graph* g, gs_workspace* ws, double fraction, uint64_t seed,
                            uint32_t mask, double z, gs_result* out, int64_t* k_out,
                            void* stream);

/* ------------------------------------------------------------------------
 * Batched exact counts over many small graphs.
 *
 * The batch is given as one packed CSR: d_vtx_off (device int64[G+1]) holds
 * each graph's first vertex, d_row_ptr (device int64[total_n+1]) the row
 * offsets into d_col over the whole pack, and d_col (device int32[total_nnz])
 * the sorted adjacency with ids LOCAL to each graph (0..n_g-1). The library
 * registers the disjoint union of the graphs (edges never cross graphs, so
 * every per-edge count of Algorithms 2-4 equals its value in its own graph),
 * sizes all buffers once, optionally times a grid of launch choices
 * (GS_BATCH_AUTOTUNE) and captures the whole counting sequence into one CUDA
 * graph. d_vtx_off and d_row_ptr are borrowed until gs_batch_destroy; d_col
 * is copied. flags: GS_VALIDATE and/or GS_BATCH_AUTOTUNE.
 * ------------------------------------------------------------------------ */
#define GS_BATCH_AUTOTUNE 2u
typedef struct gs_batch gs_batch;
typedef struct {
  int64_t num_graphs;
  int64_t edges;            /* total edges of the batch */
  int32_t tri_blocks_per_sm, quad_blocks_per_sm;
  int64_t task_probes;
  int32_t use_hubs;         /* launch choices in the captured graph */
  int32_t candidates;       /* autotuner candidates timed (0 = not tuned) */
  float best_ms, worst_ms;  /* autotuner: fastest and slowest candidate */
  int64_t graph_kernels;    /* kernel launches inside the captured graph */
  uint64_t workspace_bytes;
} gs_batch_stats;

gs_status gs_batch_create(const int64_t* d_vtx_off, const int64_t* d_row_ptr, const int32_t* d_col,
                          int64_t num_graphs, int64_t total_n, int64_t total_nnz, uint32_t mask,
                          uint32_t flags, uint64_t hub_budget_bytes, void* stream,
                          gs_batch** out);
/* Exact sums for every graph of the batch (K = M of each graph, so
 * gs_estimate gives exact counts): one CUDA-graph launch, then the
 * per-graph sums are copied to h_sums (host gs_sums[num_graphs]).
 * Synchronises `stream`. */
gs_status gs_batch_count(gs_batch* b, gs_sums* h_sums, void* stream);
gs_status gs_batch_info(const gs_batch* b, gs_batch_stats* out);
gs_status gs_batch_destroy(gs_batch* b);

/* ------------------------------------------------------------------------
 * Serving: estimation requests over resident graphs, batched continuously.
 *
 * gs_server_add_graph adds a graph (device CSR as for gs_graph_create,
 * borrowed until gs_server_destroy); gs_server_start registers every graph
 * (each with its own hub index) and starts `lanes` worker threads, each
 * with its own CUDA stream. A request names a graph, a graphlet mask, a
 * sample fraction (Algorithm 1, same sampler and seed semantics as
 * gs_sample on that graph), a seed and z. Workers take queued requests in
 * arrival order into a batch while the batch's estimated device memory fits
 * hbm_budget_bytes next to the batches other workers hold; a batch's
 * requests on one graph are sampled and counted in one pass with a separate
 * exact fold per request, so a request's result is identical to running it
 * alone. gs_server_wait blocks until a ticket's result is ready (or
 * timeout_s passes: GS_ETIMEOUT, the request stays queued). Latencies are
 * measured on the host from submit to completion.
 * ------------------------------------------------------------------------ */
typedef struct gs_server gs_server;
typedef struct {
  int32_t graph;        /* id from gs_server_add_graph */
  uint32_t mask;        /* GS_* graphlet bits */
  double fraction;      /* edge-sample fraction in [0, 1] */
  uint64_t seed;
  double z;             /* bound width, 1.96 for 95% */
} gs_request;
typedef struct {
  int64_t k;            /* sampled edges */
  int64_t batch_size;   /* requests counted in the same pass */
  double queue_s;       /* submit -> batch start */
  double latency_s;     /* submit -> result ready */
  int64_t est_bytes;    /* memory estimate used for admission */
} gs_request_stats;
typedef struct {
  int64_t graphs, batches, completed, pending;
  double mean_batch;
  uint64_t peak_reserved_bytes, budget_bytes;
  int32_t peak_in_flight;  /* most batches on the device at once */
} gs_server_stats;

gs_status gs_server_create(uint64_t hbm_budget_bytes, int32_t max_batch, int32_t lanes,
                           gs_server** out);
gs_status gs_server_add_graph(gs_server* s, const int64_t* d_row_ptr, const int32_t* d_col,
                              int64_t n, int64_t nnz, int32_t* graph_id);
gs_status gs_server_start(gs_server* s, uint32_t flags, uint64_t hub_budget_bytes, void* stream);
/* GS_EBUDGET if the request alone exceeds the budget. */
gs_status gs_server_submit(gs_server* s, const gs_request* r, uint64_t* ticket);
gs_status gs_server_wait(gs_server* s, uint64_t ticket, double timeout_s, gs_result* out,
                         gs_request_stats* stats);
gs_status gs_server_info(gs_server* s, gs_server_stats* out);
/* Cancels queued requests (GS_ECANCELLED), lets batches already on the
 * device finish, stops the workers and frees everything. No ticket may be
 * waited on after this call. */
gs_status gs_server_destroy(gs_server* s);

/* ------------------------------------------------------------------------
 * Counting without device allocation. (The paper has no counterpart: this
 * entry point exists for callers of the library, not for the method.)
 *
 * gs_count3_static computes the same triangle / 2-star sums as gs_count
 * with mask GS_G3 and/or GS_G4 (the mask must be a non-empty subset of
 * GS_THREE_NODE), but never calls cudaMalloc, cudaFree or any allocating
 * routine. It is meant for callers that cannot allocate device memory at
 * the time they count: hosts that give the GPU a fixed memory pool when
 * they start and forbid any growth afterwards (an allocation that fails in
 * the middle of a request is not acceptable there), and latency paths where
 * a cudaMalloc / cudaFree pair, which can wait for the whole device to go
 * idle, costs too much. The graph must still have been registered with
 * gs_graph_create beforehand.
 *
 * Its scratch is one file-scope device array of GS_STATIC_SCRATCH_BYTES
 * (48 MiB). Every GPU that loads the library's code holds it until the
 * process exits; with lazy module loading (the CUDA default) that can
 * happen only at the first call on that device. d_pairs: device
 * int32[2*k], k <= GS_STATIC_MAX_PAIRS (2^20), each pair an edge in either
 * orientation, no edge twice; larger k is rejected with GS_ECAPACITY before
 * anything is read (use gs_count). h_sums is host memory. The call
 * synchronises `stream`.
 *
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (once per device, with that device current). All
 * calls share the one array and it keeps the previous call's contents (the
 * call clears what must start at zero), so calls whose GPU work overlaps --
 * on different streams or host threads, for the same device -- race and
 * give wrong results: serialise them.
 * ------------------------------------------------------------------------ */
#define GS_STATIC_MAX_PAIRS (1 << 20)
#define GS_STATIC_SCRATCH_BYTES (48u << 20)
gs_status gs_count3_static(const gs_graph* g, const int32_t* d_pairs, int64_t k, uint32_t mask,
                           gs_sums* h_sums, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GRAPHLET_H */
