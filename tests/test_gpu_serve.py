"""Serving path: requests over resident graphs, batched continuously; each
result equals the same request run alone (and the oracle's)."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_estimates_close, oracle_sums

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1701_01772_gb300 as gs  # noqa: E402

MASKS = [gs.GS_CONNECTED, gs.GS_THREE_NODE, gs.GS_G7 | gs.GS_G8, gs.GS_G10 | gs.GS_G12,
         gs.GS_G3 | gs.GS_G11, gs.GS_G9]


def _graphs():
    return [synth.er(2000, 20000, seed=101), synth.chung_lu(20000, 150000, 2.1, 1500.0, seed=7),
            synth.rmat(12, 8, seed=9), synth.er(2000, 20000, seed=102)]


def _same(a, b, mask):
    da, db = a.as_dict(), b.as_dict()
    for g in gs.GRAPHLETS:
        if not mask & (1 << g):
            continue
        for key in ("X", "V", "lb", "ub"):
            x, y = da[g][key], db[g][key]
            assert (math.isnan(x) and math.isnan(y)) or x == y, (g, key, x, y)


def test_served_results_equal_requests_run_alone():
    gs.build()
    graphs = _graphs()
    srv = gs.Server(hbm_budget_bytes=8 << 30, max_batch=16, lanes=2)
    ids = [srv.add_numpy(rp, col) for rp, col in graphs]
    srv.start()
    alone = [gs.Graph.from_numpy(rp, col) for rp, col in graphs]
    rng = np.random.default_rng(4)
    reqs = []
    for i in range(48):
        gi = int(rng.integers(0, len(graphs)))
        frac = float(10 ** rng.uniform(-3, -1))
        seed = int(rng.integers(1, 2**62))
        mask = MASKS[i % len(MASKS)]
        reqs.append((gi, frac, seed, mask, srv.submit(ids[gi], frac, seed, mask)))
    sizes = []
    for gi, frac, seed, mask, ticket in reqs:
        res, st = srv.wait(ticket)
        sizes.append(st["batch_size"])
        ref, k = alone[gi].count_estimate(frac, seed, mask)
        assert st["k"] == k
        _same(res, ref, mask)
    info = srv.info()
    assert info["completed"] == len(reqs)
    assert max(sizes) > 1, "requests were never batched together"
    # oracle check of a few served requests
    for gi, frac, seed, mask, _ in reqs[:4]:
        rp, col = graphs[gi]
        pairs = oracle.sample(rp, col, frac, seed)
        s, s2, _ = oracle_sums(rp, col, pairs)
        ref = oracle.estimate(s, s2, len(col) // 2, len(pairs))
        t = srv.submit(ids[gi], frac, seed, mask)
        res, _ = srv.wait(t)
        assert_estimates_close(res, ref, [g for g in gs.GRAPHLETS if mask & (1 << g)])
    srv.close()
    for g in alone:
        g.close()


def test_budget_limits_batches_and_rejects_oversized_requests():
    gs.build()
    graphs = _graphs()[:2]
    srv = gs.Server(hbm_budget_bytes=16 << 20, max_batch=8, lanes=2)
    ids = [srv.add_numpy(rp, col) for rp, col in graphs]
    srv.start()
    with pytest.raises(gs.GraphletError) as ei:
        srv.submit(ids[1], 1.0, 1)  # all 150k edges of the 20k-vertex graph: over 16 MiB
    assert ei.value.status == 10
    tickets = [srv.submit(ids[i % 2], 0.01, 100 + i) for i in range(12)]
    for t in tickets:
        srv.wait(t)
    info = srv.info()
    assert info["peak_reserved_bytes"] <= info["budget_bytes"]
    srv.close()
