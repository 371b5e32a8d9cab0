"""gs_count3_static, the counting entry point that allocates nothing.

Some callers cannot allocate device memory at the moment they count: a host
that gives the GPU a fixed memory pool when it starts and forbids growth
afterwards, or a latency path that cannot pay for a cudaMalloc / cudaFree
pair. gs_count3_static serves them from one fixed static device array. This
file checks, through the C ABI, that

  * two calls in a row give the same sums as gs_count (so the second call
    sees nothing left over from the first), and the same as the oracle;
  * a call at the fixed maximum sample size still matches gs_count;
  * the calls change the device's free memory by nothing;
  * samples above the fixed limit and invalid samples are refused.

The file is named so that pytest collects it last; it also passes when run
alone in a fresh process."""
import numpy as np
import pytest

import synth
from gpu_util import assert_sums_equal, oracle_sums

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1701_01772_gb300 as gs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    gs.build()
    yield


def _sums_equal(a, b, ids):
    sa, sb = a.sums(), b.sums()
    for i in ids:
        assert sa[i] == sb[i], (i, sa[i], sb[i])


def test_static_scratch_count_matches_gs_count_on_two_calls_in_a_row():
    rp, col = synth.chung_lu(20000, 150000, 2.1, 1500.0, seed=77)
    g = gs.Graph.from_numpy(rp, col)
    first_np = synth.explicit_sample(rp, col, 0.30, seed=5)
    second_np = synth.explicit_sample(rp, col, 0.02, seed=6)
    for pairs_np in (first_np, second_np):
        pairs = torch.as_tensor(pairs_np, device="cuda")
        want = g.count(pairs, gs.GS_THREE_NODE)
        got = gs.gs_count3_static(g.handle, pairs, pairs.shape[0], gs.GS_THREE_NODE)
        assert got.k == pairs.shape[0] and got.m == g.m
        _sums_equal(got, want, (3, 4))
        s, s2, _ = oracle_sums(rp, col, pairs_np)
        assert_sums_equal(got, s, s2, (3, 4))
        # estimates from the two paths agree exactly (same integer sums)
        ra, rb = gs.gs_estimate(got).as_dict(), gs.gs_estimate(want).as_dict()
        for i in (3, 4):
            assert ra[i]["X"] == rb[i]["X"] and ra[i]["V"] == rb[i]["V"]
    # single-graphlet masks and the full edge list of a second graph
    rp2, col2 = synth.er_2000()
    g2 = gs.Graph.from_numpy(rp2, col2)
    allp = torch.as_tensor(synth.upper_pairs(rp2, col2), device="cuda")
    for mask, ids in ((gs.GS_G3, (3,)), (gs.GS_G4, (4,))):
        _sums_equal(gs.gs_count3_static(g2.handle, allp, allp.shape[0], mask),
                    g2.count(allp, mask), ids)
    g.close()
    g2.close()


def test_static_scratch_at_the_maximum_sample_size_allocates_nothing():
    """k = GS_STATIC_MAX_PAIRS on a graph with more edges than that: the
    tightest scratch layout. Free device memory is read around two calls made
    after a first one (the first call may load the library's code onto the
    device, which is when the static array itself is reserved)."""
    rp, col = synth.chung_lu(200_000, 1_200_000, 2.1, 5000.0, seed=91)
    assert len(col) // 2 > gs.GS_STATIC_MAX_PAIRS
    g = gs.Graph.from_numpy(rp, col)
    pairs_np = synth.explicit_sample(rp, col, 0.95, seed=3)[:gs.GS_STATIC_MAX_PAIRS]
    assert len(pairs_np) == gs.GS_STATIC_MAX_PAIRS
    pairs = torch.as_tensor(np.ascontiguousarray(pairs_np), device="cuda")
    want = g.count(pairs, gs.GS_THREE_NODE)
    torch.cuda.synchronize()
    first = gs.gs_count3_static(g.handle, pairs, pairs.shape[0], gs.GS_THREE_NODE)
    _sums_equal(first, want, (3, 4))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    again = [gs.gs_count3_static(g.handle, pairs, pairs.shape[0], gs.GS_THREE_NODE)
             for _ in range(2)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    for s in again:
        _sums_equal(s, want, (3, 4))
    g.close()


def test_static_scratch_rejects_oversized_and_invalid_requests():
    rp, col = synth.er(3000, 30000, seed=4)
    g = gs.Graph.from_numpy(rp, col)
    pairs = torch.as_tensor(synth.upper_pairs(rp, col)[:100], device="cuda")
    # one row above the limit: refused before anything is read
    over = torch.zeros((gs.GS_STATIC_MAX_PAIRS + 1, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(gs.GraphletError) as ei:
        gs.gs_count3_static(g.handle, over, over.shape[0], gs.GS_THREE_NODE)
    assert ei.value.status == 13
    with pytest.raises(gs.GraphletError) as ei:
        gs.gs_count3_static(g.handle, pairs, pairs.shape[0], gs.GS_CONNECTED)
    assert ei.value.status == 1
    dup = torch.cat([pairs, pairs[:1].flip(1)]).contiguous()
    with pytest.raises(gs.GraphletError) as ei:
        gs.gs_count3_static(g.handle, dup, dup.shape[0], gs.GS_THREE_NODE)
    assert ei.value.status == 7
    # the binding refuses a k beyond the rows it was given
    with pytest.raises(ValueError):
        gs.gs_count3_static(g.handle, pairs, pairs.shape[0] + 1, gs.GS_THREE_NODE)
    # still usable after the errors
    _sums_equal(gs.gs_count3_static(g.handle, pairs, pairs.shape[0], gs.GS_THREE_NODE),
                g.count(pairs, gs.GS_THREE_NODE), (3, 4))
    g.close()
