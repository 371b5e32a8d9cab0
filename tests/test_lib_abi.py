"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/graphlet.h declares; the binding
refuses to run without it (no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "graphlet.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("gs_graph_create", "gs_graph_destroy", "gs_sample", "gs_count", "gs_estimate",
                 "gs_count_estimate", "gs_workspace_create", "gs_last_error"):
        assert want in names


def test_library_builds_and_exports_every_declared_symbol():
    import paper_1701_01772_gb300 as gs
    path = gs.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_calls_need_no_gpu():
    import paper_1701_01772_gb300 as gs
    gs.build()
    assert "libgraphlet" in gs.gs_version()
    L = gs.lib()
    L.gs_last_error()


def test_estimate_is_host_only_and_exact_at_full_sample():
    """gs_estimate runs on the host: K = M gives exact counts and zero variance."""
    import paper_1701_01772_gb300 as gs
    gs.build()
    s = gs.GsSums()
    s.k = s.m = 10
    s.mask = gs.GS_CONNECTED
    vals = [30, 20, 6, 1, 2, 4, 6, 1]
    for i, v in enumerate(vals):
        s.sum[i][0] = v
        s.sumsq[i][0] = v * v
    r = gs.gs_estimate(s).as_dict()
    for i, g in enumerate(gs.GRAPHLETS):
        assert r[g]["exact"] == vals[i] // gs.DENOM[i]
        assert r[g]["V"] == 0.0


def test_estimate_matches_oracle_rational_arithmetic():
    """Host FP64 estimator vs the oracle's exact-rational estimator on the
    same integer sums (relative 1e-12)."""
    import math

    import numpy as np

    import oracle
    import paper_1701_01772_gb300 as gs
    import synth
    gs.build()
    rp, col = synth.chung_lu(3000, 20000, 2.1, 400.0, seed=5)
    pairs = oracle.sample(rp, col, 0.07, 9)
    lc = oracle.local_counts(rp, col, pairs)
    s1, s2 = oracle.numerators(lc)
    ref = oracle.estimate(s1, s2, len(col) // 2, len(pairs))
    s = gs.GsSums()
    s.k, s.m, s.mask = len(pairs), len(col) // 2, gs.GS_CONNECTED
    for i, g in enumerate(gs.GRAPHLETS):
        v = s1[g] % (1 << 128)
        s.sum[i][0], s.sum[i][1] = v & (2**64 - 1), v >> 64
        s.sumsq[i][0], s.sumsq[i][1] = s2[g] & (2**64 - 1), s2[g] >> 64
    got = gs.gs_estimate(s).as_dict()
    for g in gs.GRAPHLETS:
        for key in ("X", "V"):
            assert got[g][key] == pytest.approx(ref[g][key], rel=1e-12, abs=0.0), (g, key)
        half = 1.96 * math.sqrt(ref[g]["V"])
        scale = abs(ref[g]["X"]) + half
        assert abs(got[g]["lb"] - ref[g]["lb"]) <= 1e-12 * scale
        assert abs(got[g]["ub"] - ref[g]["ub"]) <= 1e-12 * scale
    assert np.isfinite([got[g]["V"] for g in gs.GRAPHLETS]).all()


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_1701_01772_gb300 as gs
    monkeypatch.setattr(gs, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(gs, "_lib_handle", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        gs.lib()


def test_header_is_plain_c_and_struct_layouts_match_the_binding(tmp_path):
    """include/graphlet.h compiles as C99 (no C++ or CUDA types in the
    boundary), and the sizes of its result structs equal the binding's."""
    import shutil
    import subprocess

    import paper_1701_01772_gb300 as gs
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text('#include <stdio.h>\n#include "graphlet.h"\nint main(void) {\n'
                   '  printf("%zu %zu %zu %zu %zu\\n", sizeof(gs_sums), sizeof(gs_result),\n'
                   '         sizeof(gs_sums_disc), sizeof(gs_result_disc), sizeof(gs_stats));\n'
                   '  return 0;\n}\n')
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True)
    sizes = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                            check=True).stdout.split()]
    want = [ctypes.sizeof(c) for c in (gs.GsSums, gs.GsResult, gs.GsSumsDisc, gs.GsResultDisc,
                                       gs.GsStats)]
    assert sizes == want
