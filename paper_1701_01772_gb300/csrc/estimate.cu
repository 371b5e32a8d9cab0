// Host-side estimators (Sec. 2.3), variance and confidence bounds (Sec. 6.2),
// plus the fused sample -> count -> estimate convenience call.
#include <math.h>
#include <string.h>

#include "common.cuh"

namespace {

typedef unsigned __int128 u128;
typedef __int128 i128;

const int64_t kDenom[8] = {3, 2, 6, 1, 2, 4, 6, 1};
const uint32_t kBit[8] = {GS_G3, GS_G4, GS_G7, GS_G8, GS_G9, GS_G10, GS_G11, GS_G12};

// 256-bit unsigned integer as four 64-bit words, least significant first.
struct U256 {
  uint64_t w[4];
};

U256 mul_128x128(u128 a, u128 b) {
  uint64_t a0 = (uint64_t)a, a1 = (uint64_t)(a >> 64), b0 = (uint64_t)b, b1 = (uint64_t)(b >> 64);
  u128 p00 = (u128)a0 * b0, p01 = (u128)a0 * b1, p10 = (u128)a1 * b0, p11 = (u128)a1 * b1;
  U256 r;
  r.w[0] = (uint64_t)p00;
  u128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;
  r.w[1] = (uint64_t)mid;
  u128 hi = (mid >> 64) + (p01 >> 64) + (p10 >> 64) + (uint64_t)p11;
  r.w[2] = (uint64_t)hi;
  r.w[3] = (uint64_t)((hi >> 64) + (p11 >> 64));
  return r;
}

// a - b, requires a >= b.
U256 sub_256(const U256& a, const U256& b) {
  U256 r;
  uint64_t borrow = 0;
  for (int i = 0; i < 4; ++i) {
    u128 d = (u128)a.w[i] - b.w[i] - borrow;
    r.w[i] = (uint64_t)d;
    borrow = (uint64_t)(d >> 64) ? 1 : 0;
  }
  return r;
}

bool less_256(const U256& a, const U256& b) {
  for (int i = 3; i >= 0; --i)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i];
  return false;
}

double to_double_256(const U256& a) {
  double r = 0.0;
  for (int i = 3; i >= 0; --i) r = r * 18446744073709551616.0 + (double)a.w[i];
  return r;
}

i128 load_i128(const uint64_t v[2]) { return (i128)(((u128)v[1] << 64) | v[0]); }
u128 load_u128(const uint64_t v[2]) { return ((u128)v[1] << 64) | v[0]; }

// One estimator of the form X = c + sign * sigma * S / D (sigma = M / K; c and
// sign = -1 only for the complements X6, X17): estimate, SRSWOR variance of
// the linear part, bounds, and the exact count when K = M.
struct One {
  double x, var, lb, ub;
  uint64_t exact;
  uint32_t flags;
};

One estimate_one(i128 S, u128 S2, bool sq_wrapped, int64_t D, int64_t M, int64_t K, double z,
                 bool complement, u128 c) {
  One r{NAN, NAN, NAN, NAN, 0, GS_F_COMPUTED};
  double x = NAN;
  if (K >= 1) {
    // M S / (K D): one rounding of the exact product when it fits.
    const u128 absS = (u128)(S < 0 ? -S : S);
    if (absS < ((u128)1 << 90) && M < ((int64_t)1 << 36)) {
      x = (double)(S * (i128)M) / (double)(K * D);
    } else {
      x = ((double)M / (double)K) * ((double)S / (double)D);
    }
    if (complement) x = (double)c - x;
  }
  double var = NAN;
  if (K == M && K >= 1) {
    r.flags |= GS_F_EXACT;
    var = 0.0;
    if (S % D != 0) {
      r.flags |= GS_F_OVERFLOW;
    } else {
      const i128 q = S / D;
      const i128 cnt = complement ? (i128)c - q : q;
      if (cnt < 0 || (u128)cnt > (u128)UINT64_MAX)
        r.flags |= GS_F_OVERFLOW;
      else
        r.exact = (uint64_t)cnt;
    }
  } else if (K >= 2 && sq_wrapped) {
    r.flags |= GS_F_VAR_OVERFLOW;
  } else if (K >= 2) {
    // Q = K sum N^2 - (sum N)^2 >= 0 exactly, in 256 bits.
    const U256 a = mul_128x128(S2, (u128)K);
    const u128 absS = (u128)(S < 0 ? -S : S);
    const U256 b = mul_128x128(absS, absS);
    const double Q = less_256(a, b) ? 0.0 : to_double_256(sub_256(a, b));
    const double num = (double)M * (double)(M - K);
    const double den = (double)K * (double)K * (double)(K - 1) * (double)(D * D);
    var = num / den * Q;
  } else {
    r.flags |= GS_F_VAR_UNDEFINED;
  }
  r.x = x;
  r.var = var;
  if (!(r.flags & (GS_F_VAR_UNDEFINED | GS_F_VAR_OVERFLOW))) {
    const double half = z * sqrt(var);
    r.lb = x - half;
    r.ub = x + half;
  }
  return r;
}

}  // namespace

extern "C" gs_status gs_estimate(const gs_sums* s, double z, gs_result* out) {
  if (s == nullptr || out == nullptr || s->k < 0 || s->m < 0 || s->k > s->m || !(z >= 0.0)) {
    gs::set_error("gs_estimate: invalid arguments (need 0 <= k <= m, z >= 0)");
    return GS_EINVAL;
  }
  for (int i = 0; i < 8; ++i) {
    out->x[i] = out->var[i] = out->lb[i] = out->ub[i] = NAN;
    out->exact[i] = 0;
    out->flags[i] = 0;
    if (!(s->mask & kBit[i])) continue;
    const One r = estimate_one(load_i128(s->sum[i]), load_u128(s->sumsq[i]), false, kDenom[i],
                               s->m, s->k, z, false, 0);
    out->x[i] = r.x;
    out->var[i] = r.var;
    out->lb[i] = r.lb;
    out->ub[i] = r.ub;
    out->exact[i] = r.exact;
    out->flags[i] = r.flags;
  }
  return GS_OK;
}

extern "C" gs_status gs_estimate_disconnected(const gs_sums_disc* s, double z, gs_result_disc* out) {
  if (s == nullptr || out == nullptr || s->k < 0 || s->m < 0 || s->k > s->m || s->n < 0 ||
      !(z >= 0.0)) {
    gs::set_error("gs_estimate_disconnected: invalid arguments (need 0 <= k <= m, n >= 0, "
                  "z >= 0)");
    return GS_EINVAL;
  }
  static const int64_t D[7] = {1, 6, 6, 2, 2, 1, 12};  // order 5, 6, 13, 14, 15, 16, 17
  const u128 n = (u128)s->n;
  const u128 c3 = n < 3 ? 0 : n * (n - 1) * (n - 2) / 6;                  // C(n, 3)
  const u128 c4 = n < 4 ? 0 : n * (n - 1) * (n - 2) / 6 * (n - 3) / 4;    // C(n, 4)
  for (int i = 0; i < 7; ++i) {
    const bool complement = i == 1 || i == 6;
    const One r = estimate_one(load_i128(s->sum[i]), load_u128(s->sumsq[i]),
                               (s->overflow >> i) & 1u, D[i], s->m, s->k, z, complement,
                               i == 1 ? c3 : c4);
    out->x[i] = r.x;
    out->var[i] = r.var;
    out->lb[i] = r.lb;
    out->ub[i] = r.ub;
    out->exact[i] = r.exact;
    out->flags[i] = r.flags;
  }
  return GS_OK;
}

extern "C" gs_status gs_sums_merge(gs_sums* acc, const gs_sums* part) {
  if (acc == nullptr || part == nullptr || acc->m != part->m || acc->mask != part->mask ||
      part->k < 0 || acc->k < 0 || acc->k + part->k > acc->m) {
    gs::set_error("gs_sums_merge: sums must come from the same graph and mask, with disjoint "
                  "samples (k_acc + k_part <= m)");
    return GS_EINVAL;
  }
  acc->k += part->k;
  for (int i = 0; i < 8; ++i) {
    const u128 s = ((u128)acc->sum[i][1] << 64 | acc->sum[i][0]) +
                   ((u128)part->sum[i][1] << 64 | part->sum[i][0]);
    const u128 q = ((u128)acc->sumsq[i][1] << 64 | acc->sumsq[i][0]) +
                   ((u128)part->sumsq[i][1] << 64 | part->sumsq[i][0]);
    acc->sum[i][0] = (uint64_t)s;
    acc->sum[i][1] = (uint64_t)(s >> 64);
    acc->sumsq[i][0] = (uint64_t)q;
    acc->sumsq[i][1] = (uint64_t)(q >> 64);
  }
  return GS_OK;
}

extern "C" gs_status gs_count_estimate(const gs_graph* g, gs_workspace* ws, double fraction,
                                       uint64_t seed, uint32_t mask, double z, gs_result* out,
                                       int64_t* k_out, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (g == nullptr || ws == nullptr || out == nullptr || !(fraction >= 0.0 && fraction <= 1.0)) {
    gs::set_error("gs_count_estimate: invalid arguments");
    return GS_EINVAL;
  }
  gs_sums sums;
  int64_t K = 0;
  int64_t M = 0;
  gs_graph_info(g, nullptr, &M, nullptr, nullptr, nullptr);
  if (fraction == 1.0) {
    K = M;
    GS_TRY(gs_count(g, ws, nullptr, K, mask, nullptr, &sums, stream));
  } else {
    int32_t* pairs = nullptr;
    GS_TRY(gs::sample_impl(g, ws, fraction, seed, nullptr, 0, &K, &pairs, stream));
    GS_TRY(gs_count(g, ws, pairs, K, mask, nullptr, &sums, stream));
  }
  if (k_out) *k_out = K;
  return gs_estimate(&sums, z, out);
}

extern "C" gs_status gs_sample_size(const gs_sums* s, double z, double rel_err, int64_t* k_out) {
  if (s == nullptr || k_out == nullptr || !(z > 0.0) || !(rel_err > 0.0) || s->k < 0 ||
      s->k > s->m) {
    gs::set_error("gs_sample_size: invalid arguments (z > 0, rel_err > 0, 0 <= k <= m)");
    return GS_EINVAL;
  }
  const int64_t K = s->k, M = s->m;
  for (int i = 0; i < 8; ++i) {
    k_out[i] = -1;
    if (!(s->mask & kBit[i]) || K < 2) continue;
    const i128 S = load_i128(s->sum[i]);
    const u128 absS = (u128)(S < 0 ? -S : S);
    const U256 a = mul_128x128(load_u128(s->sumsq[i]), (u128)K);
    const U256 b = mul_128x128(absS, absS);
    const double Q = less_256(a, b) ? 0.0 : to_double_256(sub_256(a, b));
    const double D = (double)kDenom[i];
    // per-edge sample variance of y = N / D and the pilot estimate
    const double S2 = Q / ((double)K * (double)(K - 1) * D * D);
    const double X = (double)M * ((double)S / D) / (double)K;
    if (S2 == 0.0) {
      k_out[i] = K;
    } else if (X == 0.0) {
      k_out[i] = M;
    } else {
      const double h = rel_err * fabs(X);
      const double n0 = z * z * (double)M * (double)M * S2 / (h * h);
      const double need = n0 / (1.0 + n0 / (double)M);
      const double c = ceil(need);
      k_out[i] = c < 1.0 ? 1 : c >= (double)M ? M : (int64_t)c;
    }
  }
  return GS_OK;
}

extern "C" gs_status gs_count_adaptive(const gs_graph* g, gs_workspace* ws, double beta,
                                       int32_t t_max, double phi, uint64_t seed, uint32_t mask,
                                       double z, gs_sums* sums_out, gs_result* out,
                                       int32_t* iters_out, double* fraction_out, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (g == nullptr || ws == nullptr || sums_out == nullptr || out == nullptr ||
      !(beta >= 0.0 && beta < 1.0) || t_max < 1 || !(phi <= 1.0) || !(z >= 0.0)) {
    gs::set_error("gs_count_adaptive: invalid arguments (need 0 <= beta < 1, t_max >= 1, "
                  "phi <= 1, z >= 0)");
    return GS_EINVAL;
  }
  int64_t M = 0;
  gs_graph_info(g, nullptr, &M, nullptr, nullptr, nullptr);
  if (!(phi > 0.0)) phi = M > 0 ? 1.0 / sqrt((double)M) : 1.0;
  memset(sums_out, 0, sizeof(*sums_out));
  sums_out->m = M;
  sums_out->mask = mask;
  // The loss runs over the 4-node graphlets of the mask (the objective of
  // Sec. 4 takes its maximum over G^(4)); a mask without any falls back to
  // its 3-node graphlets.
  const uint32_t four = mask & (GS_G7 | GS_G8 | GS_G9 | GS_G10 | GS_G11 | GS_G12);
  const uint32_t loss_mask = four != 0 ? four : mask;
  static const uint32_t bit[8] = {GS_G3, GS_G4, GS_G7, GS_G8, GS_G9, GS_G10, GS_G11, GS_G12};
  double loss = 1.0;
  double prev[8];
  bool have_prev = false;
  int32_t t = 0;
  int64_t J = 0;  // edges sampled so far: the J smallest sampler keys
  while (loss > beta && t < t_max) {
    // K_t = ceil(phi (M - |J|)) new edges, uniformly without replacement:
    // the next K_t edges in sampler-key order
    const int64_t Kt = (int64_t)ceil(phi * (double)(M - J));
    const int64_t J_new = J + Kt < M ? J + Kt : M;
    const int64_t K = J_new - J;
    int32_t* pairs = nullptr;
    GS_TRY(gs::sample_ranks(g, ws, J, J_new, seed, nullptr, &pairs, stream));
    J = J_new;
    if (K > 0) {
      gs_sums part;
      GS_TRY(gs_count(g, ws, pairs, K, mask, nullptr, &part, stream));
      part.m = M;
      part.mask = mask;
      GS_TRY(gs_sums_merge(sums_out, &part));
    }
    GS_TRY(gs_estimate(sums_out, z, out));
    // relative change since the previous defined estimate: none counts 0
    // (also 0 -> 0), a change away from 0 counts as infinitely large
    double l = 0.0;
    for (int i = 0; i < 8; ++i) {
      if (!(loss_mask & bit[i])) continue;
      if (have_prev) {
        double r = 0.0;
        if (out->x[i] != prev[i]) {
          r = prev[i] == 0.0 ? INFINITY : fabs(out->x[i] - prev[i]) / fabs(prev[i]);
          if (isnan(r)) r = INFINITY;
        }
        if (r > l) l = r;
      }
    }
    loss = have_prev ? l : 1.0;
    if (sums_out->k > 0) {  // an empty sample has no estimate to compare with
      for (int i = 0; i < 8; ++i) prev[i] = out->x[i];
      have_prev = true;
    }
    phi *= 0.5;
    ++t;
  }
  if (iters_out) *iters_out = t;
  if (fraction_out) *fraction_out = M > 0 ? (double)J / (double)M : 0.0;
  return GS_OK;
}

extern "C" gs_status gs_sums_disc_merge(gs_sums_disc* acc, const gs_sums_disc* part) {
  if (acc == nullptr || part == nullptr || acc->m != part->m || acc->n != part->n ||
      part->k < 0 || acc->k < 0 || acc->k + part->k > acc->m) {
    gs::set_error("gs_sums_disc_merge: sums must come from the same graph, with disjoint "
                  "samples (k_acc + k_part <= m)");
    return GS_EINVAL;
  }
  acc->k += part->k;
  for (int i = 0; i < 7; ++i) {
    const u128 s = load_u128(acc->sum[i]) + load_u128(part->sum[i]);
    const u128 a = load_u128(acc->sumsq[i]), b = load_u128(part->sumsq[i]);
    const u128 q = a + b;
    if (q < a) acc->overflow |= 1u << i;
    acc->sum[i][0] = (uint64_t)s;
    acc->sum[i][1] = (uint64_t)(s >> 64);
    acc->sumsq[i][0] = (uint64_t)q;
    acc->sumsq[i][1] = (uint64_t)(q >> 64);
  }
  acc->overflow |= part->overflow;
  return GS_OK;
}
