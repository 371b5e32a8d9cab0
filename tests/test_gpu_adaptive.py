"""Algorithm 8 (adaptive estimation) on the GPU against the oracle: same
iterations, same number of sampled edges, same exact sums, and the same
result as one count of the fixed-size sample of that size (the samples are
the smallest sampler keys, so the iterations nest)."""
import math

import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1701_01772_gb300 as gs  # noqa: E402


@pytest.mark.parametrize("maker,beta,t_max,phi,seed", [
    (lambda: synth.er_2000(), 0.02, 12, 0.05, 3),
    (lambda: synth.er_2000(), 0.0, 5, 0.05, 4),
    (lambda: synth.chung_lu(20000, 150000, 2.1, 1500.0, seed=77), 0.01, 10, 0.02, 7),
    (lambda: synth.rmat(12, 10, seed=3), 0.005, 8, 0.0, 11),
], ids=["er_beta_0.02", "er_tmax", "chung_lu_20k", "rmat_12_default_phi"])
def test_adaptive_matches_oracle(maker, beta, t_max, phi, seed):
    rp, col = maker()
    g = gs.Graph.from_numpy(rp, col)
    sums, res, iters, frac = gs.gs_count_adaptive(g.handle, g.ws.handle, beta, t_max, phi, seed)
    want = oracle.adaptive_estimate(rp, col, beta, t_max, phi, seed)
    assert iters == want["iters"] and frac == want["p"] and sums.k == want["K"]
    got = sums.sums()
    for gid in gs.GRAPHLETS:
        assert got[gid] == (want["sums"][gid], want["sq"][gid]), gid
    est = res.as_dict()
    for gid in gs.GRAPHLETS:
        a, b = est[gid]["X"], want["est"][gid]["X"]
        assert abs(a - b) <= 1e-12 * max(abs(a), abs(b), 1.0), gid
    # the fixed-size sample of the final size counts to the same sums
    buf = torch.empty((max(sums.k, 1), 2), dtype=torch.int32, device="cuda")
    pairs = gs.gs_sample_fixed(g.handle, g.ws.handle, sums.k, seed, buf)
    assert g.count(pairs).sums() == got
    g.close()
