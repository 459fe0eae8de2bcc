"""Host multigrid hierarchy (make_mg_levels, make_mg_tables in csrc/plan.cpp) built from the
planner's own offsets, layout and NK stencil: its Galerkin operators must be
symmetric, and as a V(1,1) preconditioner of CG on the PE Poisson problem it
must reach the plain-CG solution in far fewer iterations.  The harness
(tests/mg_check.cpp) compiles with the host C++ compiler; no GPU."""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2011_07209_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("mg") / "mg_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "mg_check.cpp"), os.path.join(CSRC, "plan.cpp"), "-o", exe],
                   check=True)
    return exe


def _run(exe, *args):
    out = subprocess.run([exe, *map(str, args)], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


@pytest.mark.parametrize("cell, n_stcl", [((23.5, 0.0, 0.0, 120), 19), ((29.6, 0.1, 0.05, 150), 37)])
def test_vcycle_preconditioned_cg(harness, cell, n_stcl):
    r = _run(harness, *cell, 6.0, 8.0)
    assert r["n_stcl"] == n_stcl
    lv = r["levels"]
    assert len(lv) >= 3 and lv[-1] <= 600 and all(a > 4 * b for a, b in zip(lv, lv[1:]))
    assert r["asym"] < 1e-13                        # P^T A P of a symmetric A
    assert r["cg_iter"] > 150                       # plain CG to 1e-9
    assert 0 < r["pcg_iter"] <= 20                  # V(1,1)-preconditioned CG to 1e-9
    assert r["rel_diff"] < 1e-8                     # the same discrete solution
    # the device form of the hierarchy (interior / explicit rows, padded boxes,
    # dense inverse on the coarsest level), applied in FP32 as the solver does
    assert r["tables_levels"] == len(lv) + 1         # down to <= 200 points
    assert 0 < r["tables_pcg_iter"] <= 20
    assert r["tables_rel_diff"] < 1e-8
    assert 0 < r["tables_level1_explicit"] < r["tables_level1_n"]
    # the run forms the solver uses on level 1 (float4 weights per window position for
    # runs with explicit rows; the fine restriction from aligned groups of four) give
    # the row forms up to FP32 summation order
    assert r["runs_rel_diff"] < 1e-5
    assert r["restrict_runs_rel_diff"] < 1e-5 and r["restrict_runs_aligned"] == 1
    # pass D's prolongation onto the fine groups (level-1 rows from the per-group table)
    assert r["prolong_groups_rel_diff"] < 1e-6
    assert r["pinfo_even"] == 1                      # pass D reads each parents' row start as a float2
    # the sparsified device operators of the small coarse levels stay symmetric positive definite
    assert r["coarse_checked"] >= 1 and r["coarse_spd"] == 1 and r["coarse_asym"] < 1e-6
    # and level 2 onto the level-1 runs (pinfo1)
    assert r["prolong_runs1_rel_diff"] < 1e-6
