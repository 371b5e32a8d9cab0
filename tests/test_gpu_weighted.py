"""Weighted sampling (Sec. 3.1's weighted distribution F), k-core numbers and
the Horvitz-Thompson estimates on the GPU against the oracle.

k-core numbers and the weighted sample (pairs, weights, scale) are integer
or exactly specified FP64 work: bit-exact. Estimates within 1e-12 of the
magnitude of their terms (sum over the sample of |N_i| / (D_i pi_e)), exact
counts when every edge is kept with pi = 1. The extremal pipeline of Sec. 7
(k-core weighted sample, then the per-edge micro statistics and their
maxima) equals the oracle's on the same inputs."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1701_01772_gb300 as gs  # noqa: E402

REL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    yield


def _cores(g):
    out = torch.empty(g.info["n"], dtype=torch.int32, device="cuda")
    mx = gs.gs_core_numbers(g.handle, g.ws.handle, out)
    return out, mx


def _wsample(g, w, frac, seed):
    cap = g.m
    pairs = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    pw = torch.empty(cap, dtype=torch.int32, device="cuda")
    k, s = gs.gs_sample_weighted(g.handle, g.ws.handle, w, frac, seed, pairs, pw)
    return pairs[:k], pw[:k], s


GRAPHS = {
    "er_2000": lambda: synth.er_2000(),
    "chung_lu_20k": lambda: synth.chung_lu(20000, 150000, 2.1, 1500.0, seed=77),
    "rmat_13": lambda: synth.rmat(13, 12, seed=5),
    "clique_50": lambda: synth.from_pairs(60, *map(np.array, zip(*itertools.combinations(range(50), 2)))),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_core_numbers_equal_the_oracle(name):
    rp, col = GRAPHS[name]()
    g = gs.Graph.from_numpy(rp, col)
    core, mx = _cores(g)
    want = oracle.core_numbers(rp, col)
    assert np.array_equal(core.cpu().numpy(), want)
    assert mx == want.max()
    g.close()


@pytest.mark.parametrize("name", ["chung_lu_20k", "rmat_13"])
@pytest.mark.parametrize("weights", ["core", "degree"])
@pytest.mark.parametrize("frac,seed", [(0.01, 1), (0.2, 2**63 + 5)])
def test_weighted_sample_and_estimates_match_the_oracle(name, weights, frac, seed):
    rp, col = GRAPHS[name]()
    g = gs.Graph.from_numpy(rp, col)
    if weights == "core":
        w, _ = _cores(g)
        w_np = w.cpu().numpy()
    else:
        w_np = np.diff(rp).astype(np.int32)
        w = torch.as_tensor(w_np, device="cuda")
    pairs, pw, s = _wsample(g, w, frac, seed)
    want_pairs, want_w, want_s = oracle.sample_weighted(rp, col, w_np, frac, seed)
    assert s == want_s
    assert np.array_equal(pairs.cpu().numpy(), want_pairs)
    assert np.array_equal(pw.cpu().numpy(), want_w)
    res = gs.gs_count_weighted(g.handle, g.ws.handle, pairs, pairs.shape[0], w, s).as_dict()
    lc = oracle.local_counts(rp, col, want_pairs)
    ref = oracle.ht_estimate(lc, want_w, want_s, len(col) // 2)
    _, _, nmat = oracle.numerators(lc, per_edge=True)
    pis = np.array(oracle.inclusion_probability(want_w, want_s))
    for i, gid in enumerate(gs.GRAPHLETS):
        scale_x = float(np.sum(np.abs(nmat[:, i]) / pis)) / gs.DENOM[i] + 1.0
        scale_v = float(np.sum(nmat[:, i].astype(float) ** 2 / pis ** 2)) / gs.DENOM[i] ** 2 + 1
        assert abs(res[gid]["X"] - ref[gid]["X"]) <= REL * scale_x, gid
        assert abs(res[gid]["V"] - ref[gid]["V"]) <= REL * scale_v, gid
        assert res[gid]["exact"] is None
    g.close()


def test_equal_weights_give_the_uniform_sample_and_pi_one_gives_exact_counts():
    rp, col = GRAPHS["chung_lu_20k"]()
    g = gs.Graph.from_numpy(rp, col)
    ones = torch.full((g.info["n"],), 3, dtype=torch.int32, device="cuda")
    pairs, pw, s = _wsample(g, ones, 0.1, 7)
    assert torch.equal(pairs, g.sample(0.1, 7))
    pairs, pw, s = _wsample(g, ones, 1.0, 7)
    assert pairs.shape[0] == g.m
    res = gs.gs_count_weighted(g.handle, g.ws.handle, pairs, g.m, ones, s).as_dict()
    exact = oracle.exact_counts(rp, col)
    for gid in gs.GRAPHLETS:
        assert res[gid]["exact"] == exact[gid] and res[gid]["V"] == 0.0
    g.close()


def test_extremal_pipeline_kcore_against_uniform():
    """A clique of 30 planted in a sparse power-law graph (100,000 vertices,
    300,456 edges): the extremal statistics (Sec. 7) of a k-core weighted
    0.1% sample equal the oracle's on that sample, and its largest 4-clique
    count per edge is a clique edge's (C(28, 2) = 378), which the uniform
    0.1% sample of the same seed misses (its largest is 4) -- the effect the
    paper's Table 9 reports for k-core sampling."""
    rp0, col0 = synth.chung_lu(100000, 300000, 2.3, 300.0, seed=3)
    up = synth.upper_pairs(rp0, col0)
    clique = np.array(list(itertools.combinations(range(30), 2)))
    both = np.concatenate([up, clique])
    rp, col = synth.from_pairs(100000, both[:, 0], both[:, 1])
    g = gs.Graph.from_numpy(rp, col)
    core, _ = _cores(g)
    pairs, pw, s = _wsample(g, core, 0.001, 1)
    out = torch.empty((pairs.shape[0], 15), dtype=torch.float64, device="cuda")
    mx, arg = gs.gs_micro(g.handle, g.ws.handle, pairs, pairs.shape[0], 1.0, 0, out)
    want, _ = oracle.micro(rp, col, pairs.cpu().numpy(), 1.0, 0)
    assert np.array_equal(out.cpu().numpy(), want)
    assert np.array_equal(np.array(mx), want.max(0))
    col7 = gs.MICRO.index(7)
    assert mx[col7] == math.comb(28, 2)
    upairs = g.sample(0.001, 1)
    uout = torch.empty((upairs.shape[0], 15), dtype=torch.float64, device="cuda")
    umx, _ = gs.gs_micro(g.handle, g.ws.handle, upairs, upairs.shape[0], 1.0, 0, uout)
    assert umx[col7] == 4.0
    g.close()


def test_weighted_errors():
    rp, col = synth.er(300, 2000, seed=2)
    g = gs.Graph.from_numpy(rp, col)
    bad = torch.full((300,), 2, dtype=torch.int32, device="cuda")
    bad[5] = -1
    pairs = torch.empty((g.m, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(gs.GraphletError) as ei:
        gs.gs_sample_weighted(g.handle, g.ws.handle, bad, 0.5, 1, pairs)
    assert ei.value.status == 1
    zero = torch.zeros(300, dtype=torch.int32, device="cuda")
    with pytest.raises(gs.GraphletError) as ei:
        gs.gs_sample_weighted(g.handle, g.ws.handle, zero, 0.5, 1, pairs)
    assert ei.value.status == 1
    small = torch.empty((3, 2), dtype=torch.int32, device="cuda")
    ones = torch.ones(300, dtype=torch.int32, device="cuda")
    with pytest.raises(gs.GraphletError) as ei:
        gs.gs_sample_weighted(g.handle, g.ws.handle, ones, 0.5, 1, small)
    assert ei.value.status == 13
    k, s = gs.gs_sample_weighted(g.handle, g.ws.handle, ones, 0.5, 1, pairs)
    zw = ones.clone()
    zw[pairs[0, 0].item()] = 0  # a sampled edge of weight 0: pi = 0
    with pytest.raises(gs.GraphletError) as ei:
        gs.gs_count_weighted(g.handle, g.ws.handle, pairs[:k], k, zw, s)
    assert ei.value.status == 1
    g.close()


def test_core_numbers_and_weighted_sample_at_full_size():
    """R-MAT 24: core numbers of all 16.8M vertices and a 0.1% k-core
    weighted sample, bit-exact against the oracle."""
    rp, col = synth.rmat_24()
    g = gs.Graph.from_numpy(rp, col)
    core, mx = _cores(g)
    want = oracle.core_numbers(rp, col)
    assert np.array_equal(core.cpu().numpy(), want)
    pairs, pw, s = _wsample(g, core, 0.001, 3)
    wp, ww, ws_ = oracle.sample_weighted(rp, col, want, 0.001, 3)
    assert s == ws_ and np.array_equal(pairs.cpu().numpy(), wp)
    assert np.array_equal(pw.cpu().numpy(), ww)
    print("R-MAT 24: max core", mx, "weighted 0.1% sample", pairs.shape[0])
    g.close()


@pytest.mark.parametrize("name", ["er_2000", "chung_lu_20k"])
def test_fixed_size_sample_equals_the_oracle(name):
    rp, col = GRAPHS[name]()
    g = gs.Graph.from_numpy(rp, col)
    m = g.m
    buf = torch.empty((m, 2), dtype=torch.int32, device="cuda")
    for k, seed in ((0, 1), (1, 1), (17, 2), (m // 3, 3), (m - 1, 4), (m, 5)):
        got = gs.gs_sample_fixed(g.handle, g.ws.handle, k, seed, buf).cpu().numpy()
        assert np.array_equal(got, oracle.sample_fixed(rp, col, k, seed)), k
    g.close()


def test_fixed_size_samples_nest_with_bernoulli_at_full_size():
    """R-MAT 24 (260M edges): exactly k distinct edges, nested in k and
    between the Bernoulli samples of the same seed whose sizes bracket k."""
    rp, col = synth.rmat_24()
    g = gs.Graph.from_numpy(rp, col)
    lo, hi = g.sample(0.001, 9), g.sample(0.0012, 9)
    k = (lo.shape[0] + hi.shape[0]) // 2
    buf = torch.empty((k + 10, 2), dtype=torch.int32, device="cuda")
    fx = gs.gs_sample_fixed(g.handle, g.ws.handle, k, 9, buf).clone()
    n = g.info["n"]
    key = lambda p: (p[:, 0].long() * n + p[:, 1].long())  # noqa: E731
    kl, kf, kh = key(lo), key(fx), key(hi)
    assert fx.shape[0] == k and torch.unique(kf).numel() == k
    assert torch.all(kf[1:] > kf[:-1])  # increasing canonical order
    assert torch.isin(kl, kf).all() and torch.isin(kf, kh).all()
    fx2 = gs.gs_sample_fixed(g.handle, g.ws.handle, k - 1000, 9, buf)
    assert torch.isin(key(fx2), kf).all()
    g.close()


def test_rank_ranges_grow_a_sample_without_replacement():
    """Edges ranked [k_lo, k_hi) by sampler key: consecutive ranges
    partition the fixed-size sample of the last rank, in canonical order."""
    rp, col = GRAPHS["chung_lu_20k"]()
    g = gs.Graph.from_numpy(rp, col)
    m = g.m
    buf = torch.empty((m, 2), dtype=torch.int32, device="cuda")
    cuts = [0, 1, 500, 7000, 7001, m // 2]
    parts = []
    for lo, hi in zip(cuts, cuts[1:]):
        parts.append(gs.gs_sample_ranks(g.handle, g.ws.handle, lo, hi, 4, buf).cpu().numpy())
    whole = oracle.sample_fixed(rp, col, cuts[-1], 4)
    joined = np.concatenate(parts)
    joined = joined[np.lexsort((joined[:, 1], joined[:, 0]))]
    assert np.array_equal(joined, whole)
    for (lo, hi), p in zip(zip(cuts, cuts[1:]), parts):
        assert len(p) == hi - lo
        want_hi = {tuple(x) for x in oracle.sample_fixed(rp, col, hi, 4).tolist()}
        want_lo = {tuple(x) for x in oracle.sample_fixed(rp, col, lo, 4).tolist()}
        assert {tuple(x) for x in p.tolist()} == want_hi - want_lo
    g.close()
