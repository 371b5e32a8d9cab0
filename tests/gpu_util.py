"""Helpers shared by the GPU parity tests: run the library and the oracle on
the same inputs and compare."""
import math

import numpy as np

import oracle

REL = 1e-12  # FP64 estimates: relative tolerance against the exact-rational oracle


def oracle_sums(row_ptr, col, pairs):
    lc = oracle.local_counts(row_ptr, col, pairs)
    s, s2 = oracle.numerators(lc)
    return s, s2, lc


def assert_sums_equal(gpu_sums, s, s2, mask_ids):
    got = gpu_sums.sums()
    for g in mask_ids:
        assert got[g][0] == s[g], (g, got[g][0], s[g])
        assert got[g][1] == s2[g], (g, got[g][1], s2[g])


def assert_estimates_close(gpu_res, ref, mask_ids):
    got = gpu_res.as_dict()
    for g in mask_ids:
        r, x = ref[g], got[g]
        if r["exact"] is not None:
            assert x["exact"] == r["exact"], g
        for key in ("X", "V"):
            if math.isnan(r[key]):
                assert math.isnan(x[key]), (g, key)
            else:
                assert abs(x[key] - r[key]) <= REL * abs(r[key]), (g, key, x[key], r[key])
        if not math.isnan(r["V"]):
            scale = abs(r["X"]) + 1.96 * math.sqrt(r["V"])
            assert abs(x["lb"] - r["lb"]) <= REL * scale, g
            assert abs(x["ub"] - r["ub"]) <= REL * scale, g


def per_edge_reference(lc):
    return np.stack([lc["t"], lc["k"], lc["q"]], axis=1)
