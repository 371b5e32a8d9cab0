"""CPU oracle for the edge-centric graphlet estimator -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library never calls it, and it
shares no code with the GPU path.

What it computes (paper: Rossi, Zhou, Ahmed, "Estimation of Graphlet
Statistics"):

* ``local_counts``  -- Algorithm 2 per sampled edge (triangle set T_e, 2-star
  sets S_u, S_v via a marker table), Algorithm 3 (4-cliques through e) and
  Algorithm 4 read as counting pairs (w in S_u, r in S_v) with w ~ r
  (4-cycles through e).  Plain C in ``oracle.c``.
* ``sums``          -- exact per-edge numerators N_i (Sec. 2.3, Eqs. for
  X_3..X_12 with sigma = M/K) and their sums / sums of squares in 128-bit
  integers (C), returned as Python ints.
* ``estimate``      -- the estimators X_i = (M/K) sum N_i / D_i (Sec. 2.3), the
  variance V_i and the 95% bounds X -/+ 1.96 sqrt(V) (Sec. 6.2).  Exact
  rational arithmetic (``fractions.Fraction``) rounded once to fp64.
  The variance is this project's reading (the paper prints no formula): the
  design-based variance of the expansion estimator under simple random
  sampling without replacement, V = M (M-K) Q / (K^2 (K-1) D^2) with
  Q = K sum N^2 - (sum N)^2.  "parity unpinned" for V against the paper; it is
  pinned to a direct two-pass sample variance and to the spread across seeds.
* ``sample``        -- Algorithm 1 with uniform Bernoulli(p) selection of each
  edge, keyed by a SplitMix64 counter hash (project-defined random source).
* ``adaptive_estimate`` -- Algorithm 8 (adaptive estimation): grow the
  sample until the maximum relative change of the estimates is at most beta.
* ``micro``         -- Algorithm 7 (micro-level estimation): the per-edge
  vector x3..x17 with neighbour probes ceil(d_w p_e); exact at p_e = 1.
* ``core_numbers``, ``sample_weighted``, ``ht_estimate`` -- Algorithm 1 with
  a weighted distribution F (k-core numbers, degrees; Sec. 3.1) and the
  estimators with a per-edge inverse inclusion probability sigma_e = 1/pi_e
  (Horvitz-Thompson), exact rationals.
* ``disconnected_estimate`` -- Sec. 2.3's estimators of the disconnected
  graphlets G5, G6, G13-G17 with their terms corrected (the printed block
  swaps C13/C14 and C15/C16); exact rationals, variance read as above.
"""
from __future__ import annotations

import ctypes
import functools
import math
import os
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")

#: graphlet ids carried by the estimator, in output order
GRAPHLETS = (3, 4, 7, 8, 9, 10, 11, 12)
#: denominators D_i of X_i = (M/K) * sum N_i / D_i
DENOM = {3: 3, 4: 2, 7: 6, 8: 1, 9: 2, 10: 4, 11: 6, 12: 1}
Z95 = 1.96


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-std=gnu11", "-ffp-contract=off", src,
                    "-o", _SO + ".tmp", "-lm"], check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


@functools.lru_cache(maxsize=1)
def _lib() -> ctypes.CDLL:
    lib = ctypes.CDLL(build())
    P, I64, U64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
    lib.oracle_local_counts.argtypes = [I64, P, P, I64, P, I, P, P, P, P, P]
    lib.oracle_local_counts.restype = I
    lib.oracle_local_counts_literal_alg4.argtypes = [I64, P, P, I64, P, P, P, P, P, P]
    lib.oracle_local_counts_literal_alg4.restype = I
    lib.oracle_numerators.argtypes = [I64, P, P, P, P, P, P, P, P]
    lib.oracle_sample.argtypes = [I64, P, P, U64, U64, P, I64]
    lib.oracle_sample.restype = I64
    lib.oracle_splitmix64.argtypes = [U64]
    lib.oracle_splitmix64.restype = U64
    lib.oracle_micro.argtypes = [I64, I64, P, P, I64, P, ctypes.c_double, U64, P, P]
    lib.oracle_micro.restype = I
    lib.oracle_core_numbers.argtypes = [I64, P, P, P]
    lib.oracle_sample_weighted.argtypes = [I64, P, P, P, ctypes.c_double, U64, P, P, I64, P]
    lib.oracle_sample_weighted.restype = I64
    return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def splitmix64(x: int) -> int:
    return int(_lib().oracle_splitmix64(x & (2**64 - 1)))


def local_counts(row_ptr, col, pairs, four: bool = True, _literal_alg4: bool = False) -> dict:
    """Per-edge (t, a, b, k, q) for every pair of ``pairs`` (int32 [K, 2]).

    ``_literal_alg4`` runs Algorithm 4 exactly as printed (a planted mistake
    used only by the tests to show the printed test is wrong)."""
    row_ptr, col = _c(row_ptr, np.int64), _c(col, np.int32)
    pairs = _c(pairs, np.int32).reshape(-1, 2)
    k = len(pairs)
    out = {name: np.zeros(k, dtype=np.int64) for name in ("t", "a", "b", "k", "q")}
    ptrs = [out[x].ctypes.data for x in ("t", "a", "b", "k", "q")]
    if _literal_alg4:
        rc = _lib().oracle_local_counts_literal_alg4(len(row_ptr) - 1, row_ptr.ctypes.data,
                                                     col.ctypes.data, k, pairs.ctypes.data, *ptrs)
    else:
        rc = _lib().oracle_local_counts(len(row_ptr) - 1, row_ptr.ctypes.data, col.ctypes.data, k,
                                        pairs.ctypes.data, int(four), *ptrs)
    if rc != 0:
        raise ValueError("oracle: a sampled pair is not an edge of the graph")
    return out


#: micro-level statistics of Algorithm 7, in output column order
MICRO = tuple(range(3, 18))


def micro(row_ptr, col, pairs, p_e: float = 1.0, seed: int = 0):
    """Algorithm 7 (micro-level estimation) for every pair of ``pairs``: the
    per-edge vector (x3, ..., x17) as float64 [K, 15] and omega [K] (hits
    from S_u or S_v into T, which x15 uses). Each vertex w of the edge's
    neighbourhood probes ceil(d_w p_e) consecutive entries of N(w) from a
    seeded offset; p_e = 1 gives the exact per-edge statistics (see
    ``oracle_micro`` in oracle.c for the reading of every line)."""
    row_ptr, col = _c(row_ptr, np.int64), _c(col, np.int32)
    pairs = _c(pairs, np.int32).reshape(-1, 2)
    if not 0.0 < p_e <= 1.0:
        raise ValueError("p_e must lie in (0, 1]")
    k = len(pairs)
    x = np.zeros((k, 15), dtype=np.float64)
    om = np.zeros(k, dtype=np.float64)
    rc = _lib().oracle_micro(len(row_ptr) - 1, len(col) // 2, row_ptr.ctypes.data,
                             col.ctypes.data, k, pairs.ctypes.data, float(p_e),
                             seed & (2**64 - 1), x.ctypes.data, om.ctypes.data)
    if rc != 0:
        raise ValueError("oracle: a sampled pair is not an edge of the graph")
    return x, om


def core_numbers(row_ptr, col) -> np.ndarray:
    """k-core number of every vertex (int32 [n]), bucket peeling."""
    row_ptr, col = _c(row_ptr, np.int64), _c(col, np.int32)
    n = len(row_ptr) - 1
    out = np.zeros(max(n, 1), dtype=np.int32)
    _lib().oracle_core_numbers(n, row_ptr.ctypes.data, col.ctypes.data, out.ctypes.data)
    return out[:n].copy()


def sample_weighted(row_ptr, col, vertex_w, fraction: float, seed: int):
    """Weighted Bernoulli sample: edge (u < v) with weight w_e = min(w_u, w_v)
    kept with probability pi_e = min(1, s w_e), s = fraction M / sum_e w_e,
    by the same key as ``sample``. Returns (pairs int32 [K, 2], w_e int32
    [K], s)."""
    row_ptr, col = _c(row_ptr, np.int64), _c(col, np.int32)
    vw = _c(vertex_w, np.int32)
    if not (0.0 <= fraction <= 1.0) or (vw < 0).any():
        raise ValueError("fraction must lie in [0, 1] and weights must be >= 0")
    m = len(col) // 2
    out = np.zeros((max(m, 1), 2), dtype=np.int32)
    ow = np.zeros(max(m, 1), dtype=np.int32)
    scale = ctypes.c_double()
    kept = _lib().oracle_sample_weighted(len(row_ptr) - 1, row_ptr.ctypes.data, col.ctypes.data,
                                         vw.ctypes.data, float(fraction), seed & (2**64 - 1),
                                         out.ctypes.data, ow.ctypes.data, m, ctypes.byref(scale))
    return out[:kept].copy(), ow[:kept].copy(), scale.value


def inclusion_probability(weights, scale: float) -> list:
    """pi_e = min(1, s w_e), evaluated in FP64 as the samplers do."""
    return [min(1.0, scale * float(w)) for w in np.asarray(weights).tolist()]


def ht_estimate(lc: dict, weights, scale: float, m: int, z: float = Z95) -> dict:
    """Estimates under weighted Bernoulli (Poisson) sampling: with the
    per-edge inverse inclusion probability sigma_e = 1 / pi_e in place of
    Sec. 2.3's uniform sigma = M/K (Horvitz-Thompson),
        X_i = sum_e N_i(e) / (D_i pi_e),
        V_i = sum_e (1 - pi_e) N_i(e)^2 / (D_i^2 pi_e^2)
    (the unbiased variance estimator of independent inclusions), bounds
    X -/+ z sqrt(V) (Sec. 6.2); exact counts when every edge is sampled with
    pi = 1. Exact rationals (pi_e taken as its exact FP64 value), rounded
    once."""
    pis = [Fraction(p) for p in inclusion_probability(weights, scale)]
    _, _, nmat = numerators(lc, per_edge=True)
    k = len(pis)
    res = {}
    all_one = k == m and all(p == 1 for p in pis)
    for i, g in enumerate(GRAPHLETS):
        d = DENOM[g]
        col_i = nmat[:, i].tolist() if k else []
        X = sum((Fraction(v) / p for v, p in zip(col_i, pis)), Fraction(0)) / d
        V = sum((Fraction(v * v) * (1 - p) / (p * p) for v, p in zip(col_i, pis)),
                Fraction(0)) / (d * d)
        r = {"X": float(X), "V": float(V), "lb": math.nan, "ub": math.nan, "exact": None}
        half = z * math.sqrt(r["V"])
        r["lb"], r["ub"] = r["X"] - half, r["X"] + half
        if all_one:
            r["exact"] = int(X)
        res[g] = r
    return res


def _u128(lo: int, hi: int) -> int:
    return (int(hi) << 64) | int(lo)


def _i128(lo: int, hi: int) -> int:
    v = _u128(lo, hi)
    return v - (1 << 128) if v >> 127 else v


def numerators(lc: dict, per_edge: bool = False):
    """Exact sums {i: sum N_i}, {i: sum N_i^2} (Python ints) and optionally
    the per-edge numerator matrix int64 [K, 8]."""
    k = len(lc["t"])
    sums = np.zeros(16, dtype=np.uint64)
    sq = np.zeros(16, dtype=np.uint64)
    nmat = np.zeros((k, 8), dtype=np.int64) if per_edge else None
    _lib().oracle_numerators(k, *(lc[x].ctypes.data for x in ("t", "a", "b", "k", "q")),
                             nmat.ctypes.data if per_edge else None, sums.ctypes.data,
                             sq.ctypes.data)
    s = {g: _i128(sums[2 * i], sums[2 * i + 1]) for i, g in enumerate(GRAPHLETS)}
    s2 = {g: _u128(sq[2 * i], sq[2 * i + 1]) for i, g in enumerate(GRAPHLETS)}
    return (s, s2, nmat) if per_edge else (s, s2)


def sample(row_ptr, col, fraction: float, seed: int) -> np.ndarray:
    """Bernoulli(fraction) edge sample as int32 [K, 2] pairs (u < v)."""
    row_ptr, col = _c(row_ptr, np.int64), _c(col, np.int32)
    if not (0.0 <= fraction <= 1.0):
        raise ValueError("fraction must lie in [0, 1]")
    threshold = int(math.floor(fraction * 2.0**53))
    m = len(col) // 2
    out = np.zeros((max(m, 1), 2), dtype=np.int32)
    kept = _lib().oracle_sample(len(row_ptr) - 1, row_ptr.ctypes.data, col.ctypes.data,
                                threshold, seed & (2**64 - 1), out.ctypes.data, m)
    return out[:kept].copy()


def sample_keys(row_ptr, col, seed: int) -> np.ndarray:
    """The 53-bit sampler key (sm(seed ^ sm(i)) >> 11) of every canonical edge
    i (uint64 [M]), SplitMix64 evaluated in Python integers."""
    m = len(col) // 2
    mask = 2**64 - 1

    def sm(x):
        z = (x + 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        return z ^ (z >> 31)

    seed &= mask
    return np.array([sm(seed ^ sm(i)) >> 11 for i in range(m)], dtype=np.uint64)


def sample_fixed(row_ptr, col, k: int, seed: int) -> np.ndarray:
    """Uniform sample of exactly k distinct edges (Algorithm 1 with a sample
    size, without replacement): the k canonical edges with the smallest
    (key, i), key = the Bernoulli sampler's 53-bit key, listed in increasing
    i as int32 [k, 2]. Because the keys are those of ``sample``, the result
    is nested with every Bernoulli sample of the same seed."""
    from synth import upper_pairs  # input helper only: lists the edges
    m = len(col) // 2
    if not 0 <= k <= m:
        raise ValueError("k must lie in [0, M]")
    keys = sample_keys(row_ptr, col, seed)
    order = np.lexsort((np.arange(m), keys))[:k]
    return upper_pairs(np.asarray(row_ptr), np.asarray(col))[np.sort(order)].copy()


def estimate(s: dict, s2: dict, m: int, k: int, z: float = Z95) -> dict:
    """Estimates, variances and bounds per graphlet from exact sums.

    X = (M/K) * S / D                            (Sec. 2.3, sigma = |E|/|J|)
    V = M (M-K) (K S2 - S^2) / (K^2 (K-1) D^2)   (SRSWOR variance, K >= 2)
    lb, ub = X -/+ z sqrt(V)                     (Sec. 6.2, z = 1.96)
    exact = S / D when K == M (must divide).
    """
    res = {}
    for g in GRAPHLETS:
        d = DENOM[g]
        S, S2 = s[g], s2[g]
        r = {"X": math.nan, "V": math.nan, "lb": math.nan, "ub": math.nan, "exact": None}
        if k >= 1:
            r["X"] = float(Fraction(m * S, k * d))
        if k >= 2:
            Q = k * S2 - S * S
            assert Q >= 0
            r["V"] = float(Fraction(m * (m - k) * Q, k * k * (k - 1) * d * d))
            half = z * math.sqrt(r["V"])
            r["lb"] = r["X"] - half
            r["ub"] = r["X"] + half
        elif k == m == 1:
            r["V"] = 0.0
            r["lb"] = r["ub"] = r["X"]
        if k == m and k >= 1:
            if S % d != 0:
                raise ArithmeticError(f"sum N_{g} = {S} not divisible by {d} at K = M")
            r["exact"] = S // d
        res[g] = r
    return res


def sample_size(s: dict, s2: dict, m: int, k: int, rel_err: float, z: float = Z95) -> dict:
    """Sample size for a target error (Sec. 6.2: K = (z sqrt(Var) / margin)^2),
    read with the per-edge standard deviation of a pilot sample of k edges
    and a margin of rel_err |X| (relative error of the pilot estimate), with
    the finite-population correction of sampling without replacement:
        S^2 = (k sum N^2 - (sum N)^2) / (k (k - 1) D^2)   (sample variance of y)
        n0  = (z m S / (rel_err |X|))^2,   K = ceil(n0 / (1 + n0 / m)),
    capped to [1, m]; K = m when the pilot estimate is 0 and its spread is
    not (no relative target is reachable); K = k when the pilot's per-edge
    values do not vary. Exact rationals; None when the pilot has fewer than
    2 edges."""
    out = {}
    for g in GRAPHLETS:
        d = DENOM[g]
        if k < 2:
            out[g] = None
            continue
        S2 = Fraction(k * s2[g] - s[g] * s[g], k * (k - 1) * d * d)
        X = Fraction(m * s[g], k * d)
        if S2 == 0:
            out[g] = k
            continue
        if X == 0:
            out[g] = m
            continue
        h = Fraction(rel_err) * abs(X)
        zf = Fraction(z)
        n0 = zf * zf * m * m * S2 / (h * h)
        K = n0 / (1 + n0 / m)
        c = -((-K.numerator) // K.denominator)
        out[g] = max(1, min(m, c))
    return out


def exact_counts(row_ptr, col) -> dict:
    """Exact connected 3- and 4-node graphlet counts (all edges sampled)."""
    from synth import upper_pairs  # input helper only: lists the edges
    pairs = upper_pairs(np.asarray(row_ptr), np.asarray(col))
    lc = local_counts(row_ptr, col, pairs)
    s, s2 = numerators(lc)
    est = estimate(s, s2, len(pairs), len(pairs))
    return {g: est[g]["exact"] for g in GRAPHLETS}


def count_estimate(row_ptr, col, pairs, z: float = Z95) -> dict:
    """Full oracle pipeline on an explicit sampled-edge list."""
    lc = local_counts(row_ptr, col, pairs)
    s, s2 = numerators(lc)
    return {"sums": s, "sq": s2, "K": len(pairs), "M": len(col) // 2,
            "est": estimate(s, s2, len(col) // 2, len(pairs), z)}


#: disconnected graphlets, in output order
DISCONNECTED = (5, 6, 13, 14, 15, 16, 17)


def disconnected_estimate(row_ptr, col, pairs, z: float = Z95) -> dict:
    """Estimators of the disconnected graphlets over the sampled edges
    ``pairs`` (Sec. 2.3, sigma = M/K), read with corrected terms: with
    R_e = N - 2 - t - a - b (vertices adjacent to neither end of e),
    C5 = sum R, C13 = sum (a+b) R, C14 = sum t R, C15 = sum C(R,2),
    C16 = sum (M - d_u - d_v + 1),

        X5  = sigma C5
        X6  = C(N,3) - X3 - X4 - X5
        X13 = (sigma C14 - X9) / 3
        X14 = sigma C13 / 2 - X12
        X15 = sigma C16 / 2 - 3 X7 - 2 X8 - X9 - 2 X10 - X12
        X16 = sigma C15 - 2 X15
        X17 = C(N,4) - (X7 + X8 + ... + X16)

    with X3..X12 the connected estimators. Each X is a constant plus sigma
    times a sum over the sampled edges of a per-edge value y_e; V is the
    SRSWOR variance of that sum, M (M - K) (K sum y^2 - (sum y)^2) /
    (K^2 (K - 1)); lb, ub = X -/+ z sqrt(V); exact = X when K = M."""
    row_ptr = np.asarray(row_ptr)
    n = len(row_ptr) - 1
    m = len(col) // 2
    lc = local_counts(row_ptr, col, pairs)
    K = len(pairs)
    y = {g: [] for g in DISCONNECTED}  # 12 * y_e, integers
    for t, a, b, k, q in zip(*(lc[x].tolist() for x in ("t", "a", "b", "k", "q"))):
        R = n - 2 - t - a - b
        c16 = m - (a + t + 1) - (b + t + 1) + 1
        # per-edge parts of the connected estimators, times 12
        x3, x4, x7 = 4 * t, 6 * (a + b), 2 * k
        x8 = 12 * (t * (t - 1) // 2 - k)
        x9 = 6 * (t * (a + b)) - 2 * x8          # (C9 - 4 X8) / 2
        x10 = 3 * q
        x11 = (12 * (a * (a - 1) // 2 + b * (b - 1) // 2) - x9) // 3   # (C11 - X9) / 3
        x12 = 12 * (a * b - q)
        x5 = 12 * R
        x13 = (12 * t * R - x9) // 3
        x14 = 6 * (a + b) * R - x12
        x15 = 6 * c16 - 3 * x7 - 2 * x8 - x9 - 2 * x10 - x12
        x16 = 12 * (R * (R - 1) // 2) - 2 * x15
        y[5].append(x5)
        y[6].append(x3 + x4 + x5)               # X6 = C(N,3) - (...)
        y[13].append(x13)
        y[14].append(x14)
        y[15].append(x15)
        y[16].append(x16)
        y[17].append(x7 + x8 + x9 + x10 + x11 + x12 + x13 + x14 + x15 + x16)
    const = {6: math.comb(n, 3), 17: math.comb(n, 4)}
    res = {}
    for g in DISCONNECTED:
        S = sum(y[g])
        S2 = sum(v * v for v in y[g])
        r = {"X": math.nan, "V": math.nan, "lb": math.nan, "ub": math.nan, "exact": None}
        if K >= 1:
            lin = Fraction(m * S, K * 12)
            X = const[g] - lin if g in const else lin
            r["X"] = float(X)
            if K == m:
                if X.denominator != 1:
                    raise ArithmeticError(f"X_{g} = {X} is not an integer at K = M")
                r["exact"] = int(X)
        if K >= 2:
            V = Fraction(m * (m - K) * (K * S2 - S * S), K * K * (K - 1) * 144)
            r["V"] = float(V)
            half = z * math.sqrt(r["V"])
            r["lb"], r["ub"] = r["X"] - half, r["X"] + half
        elif K == m == 1:
            r["V"] = 0.0
            r["lb"] = r["ub"] = r["X"]
        res[g] = r
    return res


#: the 4-node graphlets over which Algorithm 8's objective takes its maximum
FOUR_NODE = (7, 8, 9, 10, 11, 12)


def adaptive_loss_graphlets(graphlets) -> tuple:
    """Graphlets whose relative change is Algorithm 8's loss: the objective
    of Sec. 4 takes the maximum over the 4-node graphlets G^(4); a request
    holding no 4-node graphlet falls back to its 3-node ones."""
    four = tuple(g for g in graphlets if g in FOUR_NODE)
    return four if four else tuple(graphlets)


def relative_change(x: float, prev: float) -> float:
    """|x - prev| / |prev| (the maximum-relative-error objective of Sec. 4
    with the previous estimate as reference); no change counts 0 even when
    both are 0, a change away from 0 counts as infinitely large."""
    if x == prev:
        return 0.0
    if prev == 0.0:
        return math.inf
    r = abs(x - prev) / abs(prev)
    return math.inf if math.isnan(r) else r


def adaptive_estimate(row_ptr, col, beta: float, t_max: int, phi: float, seed: int,
                      graphlets=GRAPHLETS, z: float = Z95) -> dict:
    """Algorithm 8: iteration t draws K_t = ceil(phi_t (M - |J|)) new edges
    uniformly without replacement from those not yet sampled -- the next
    K_t edges in sampler-key order, so J is always the |J| smallest keys
    (``sample_fixed``) -- recomputes the estimates from everything sampled
    so far, takes as loss the maximum relative change (``relative_change``)
    of the estimates of the 4-node graphlets among ``graphlets``
    (``adaptive_loss_graphlets``) since the previous iteration, and halves
    phi after the draw; it stops when the loss is at most beta or after
    t_max iterations. The first iteration has loss 1. phi <= 0 means
    1 / sqrt(M)."""
    from synth import upper_pairs  # input helper only: lists the edges
    m = len(col) // 2
    if not phi > 0:
        phi = 1.0 / math.sqrt(m) if m > 0 else 1.0
    loss_set = adaptive_loss_graphlets(graphlets)
    keys = sample_keys(row_ptr, col, seed)
    order = np.lexsort((np.arange(m), keys))
    up = upper_pairs(np.asarray(row_ptr), np.asarray(col))
    J, loss, t = 0, 1.0, 0
    prev = None
    pairs = np.zeros((0, 2), dtype=np.int32)
    est = s = s2 = None
    while loss > beta and t < t_max:
        K_t = int(math.ceil(phi * float(m - J)))
        J = min(m, J + K_t)
        pairs = up[np.sort(order[:J])]
        lc = local_counts(row_ptr, col, pairs)
        s, s2 = numerators(lc)
        est = estimate(s, s2, m, len(pairs), z)
        x = {g: est[g]["X"] for g in loss_set}
        if prev is None:
            loss = 1.0
        else:
            loss = max(relative_change(x[g], prev[g]) for g in loss_set)
        if len(pairs) > 0:
            prev = x
        phi *= 0.5
        t += 1
    return {"iters": t, "p": J / m if m else 0.0, "K": len(pairs), "sums": s, "sq": s2,
            "est": est}
