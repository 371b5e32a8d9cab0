"""The exact 3-node pass over every edge through degree-oriented lists
(triangles listed once from their lowest vertex, per-edge t from
shared-memory counters and atomics) gives the same exact sums as the oracle
and as the general per-edge pass (which gs_count takes when per-edge output
is requested), on graphs of every shape, on cliques on either side of the
out-degree limit of the oriented lists, and at full size."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_sums_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1701_01772_gb300 as gs  # noqa: E402

THREE = (3, 4)


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    yield


def _both_paths(g):
    fast = g.count(None, gs.GS_THREE_NODE)
    per = torch.zeros((g.m, 3), dtype=torch.int64, device="cuda")
    general = g.count(None, gs.GS_THREE_NODE, per_edge=per)
    return fast, general


GRAPHS = {
    "er_2000": lambda: synth.er_2000(),
    "chung_lu_20k": lambda: synth.chung_lu(20000, 150000, 2.1, 1500.0, seed=77),
    "rmat_13": lambda: synth.rmat(13, 12, seed=5),
    "rgg_6k": lambda: synth.rgg(6000, 0.025, seed=3),
    "tiny": lambda: synth.from_pairs(50, np.array([3, 3, 4, 10]), np.array([4, 5, 5, 11])),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_oriented_exact_pass_equals_the_oracle_and_the_general_pass(name):
    rp, col = GRAPHS[name]()
    g = gs.Graph.from_numpy(rp, col)
    fast, general = _both_paths(g)
    lc = oracle.local_counts(rp, col, synth.upper_pairs(rp, col), four=False)
    s, s2 = oracle.numerators(lc)
    assert_sums_equal(fast, s, s2, THREE)
    assert fast.sums()[3] == general.sums()[3] and fast.sums()[4] == general.sums()[4]
    res = gs.gs_estimate(fast).as_dict()
    assert res[3]["exact"] * 3 == s[3]
    g.close()


@pytest.mark.parametrize("n", [3000, 4200])
def test_cliques_on_both_sides_of_the_out_degree_limit(n):
    """K_n: every edge lies in n - 2 triangles and no 2-star. K_3000 uses the
    oriented lists (largest out-degree 2,999), K_4200 the general pass."""
    a, b = zip(*itertools.combinations(range(n), 2))
    rp, col = synth.from_pairs(n, np.array(a), np.array(b))
    g = gs.Graph.from_numpy(rp, col)
    m = n * (n - 1) // 2
    fast, general = _both_paths(g)
    for s in (fast, general):
        got = s.sums()
        assert got[3] == (m * (n - 2), m * (n - 2) ** 2)
        assert got[4] == (0, 0)
    assert gs.gs_estimate(fast).as_dict()[3]["exact"] == math.comb(n, 3)
    g.close()


@pytest.mark.parametrize("maker", [synth.chung_lu_1m, synth.rmat_24], ids=["chung_lu_1m", "rmat_24"])
def test_oriented_exact_pass_at_full_size_equals_the_general_pass(maker):
    rp, col = maker()
    g = gs.Graph.from_numpy(rp, col)
    g.ws.set_timing(True)
    fast = g.count(None, gs.GS_THREE_NODE)
    st = g.ws.stats()
    print("oriented exact 3-node:", {k: st[k] for k in ("tri_tests", "ms_tri", "ms_fold")})
    per = torch.zeros((g.m, 3), dtype=torch.int64, device="cuda")
    general = g.count(None, gs.GS_THREE_NODE, per_edge=per)
    print("general exact 3-node:", {k: g.ws.stats()[k] for k in ("tri_tests", "ms_tri")})
    assert fast.sums()[3] == general.sums()[3] and fast.sums()[4] == general.sums()[4]
    # the per-edge t of the general pass sum to 3 T, as the oriented count does
    assert int(per[:, 0].sum().item()) == fast.sums()[3][0]
    g.close()
