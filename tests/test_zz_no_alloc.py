"""gs_count3_static, the counting entry point that allocates nothing.

It serves callers that cannot call cudaMalloc when they count (while a
stream is being captured into a CUDA graph, inside a fixed memory pool, or on
a latency path that cannot afford a device-wide allocation). Its scratch is a
fixed static device array, so this test checks that it gives the same sums as
gs_count on two calls in a row (the second call must not see stale data from
the first) and that it refuses samples larger than its fixed limit.

The file is named so that pytest collects it last."""
import pytest

import synth

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
    first = torch.as_tensor(synth.explicit_sample(rp, col, 0.30, seed=5), device="cuda")
    second = torch.as_tensor(synth.explicit_sample(rp, col, 0.02, seed=6), device="cuda")
    for pairs in (first, second):
        want = g.count(pairs, gs.GS_THREE_NODE)
        got = gs.gs_count3_static(g.handle, pairs, pairs.shape[0], gs.GS_THREE_NODE)
        assert got.k == pairs.shape[0] and got.m == g.m
        _sums_equal(got, want, (3, 4))
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


def test_static_scratch_rejects_oversized_and_invalid_requests():
    rp, col = synth.er(3000, 30000, seed=4)
    g = gs.Graph.from_numpy(rp, col)
    pairs = torch.as_tensor(synth.upper_pairs(rp, col)[:100], device="cuda")
    with pytest.raises(gs.GraphletError) as ei:
        gs.gs_count3_static(g.handle, pairs, gs.GS_STATIC_MAX_PAIRS + 1, gs.GS_THREE_NODE)
    assert ei.value.status == 13
    with pytest.raises(gs.GraphletError) as ei:
        gs.gs_count3_static(g.handle, pairs, pairs.shape[0], gs.GS_CONNECTED)
    assert ei.value.status == 1
    dup = torch.cat([pairs, pairs[:1].flip(1)]).contiguous()
    with pytest.raises(gs.GraphletError) as ei:
        gs.gs_count3_static(g.handle, dup, dup.shape[0], gs.GS_THREE_NODE)
    assert ei.value.status == 7
    # still usable after the errors
    _sums_equal(gs.gs_count3_static(g.handle, pairs, pairs.shape[0], gs.GS_THREE_NODE),
                g.count(pairs, gs.GS_THREE_NODE), (3, 4))
    g.close()
