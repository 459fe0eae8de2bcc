"""Host logic of the schedule autotuner (exx_plan_autotune): the candidate
schedules and the pick among measured solver times, driven with fake timings
through a host harness (tests/sched_check.cpp, compiled with the host C++
compiler; no GPU)."""
import json
import math
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
    exe = str(tmp_path_factory.mktemp("sched") / "sched_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "sched_check.cpp"), os.path.join(CSRC, "plan.cpp"), "-o", exe],
                   check=True)
    return exe


def _run(exe, mg, *ms):
    out = subprocess.run([exe, str(int(mg)), *map(str, ms)], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


def test_candidates(harness):
    r = _run(harness, True)
    # MG with omega 0.8, 0.7, 0.6 (inner_shift 14, 18 each), then plain CG
    assert r["n"] == 8
    assert r["cand"][0] == [1, 0.8, 14] and r["cand"][1] == [1, 0.8, 18]
    assert [c[1] for c in r["cand"][:6:2]] == [0.8, 0.7, 0.6]
    assert r["cand"][6] == [0, 0.7, 14] and r["cand"][7] == [0, 0.7, 18]
    plain = _run(harness, False)
    assert plain["n"] == 2 and all(c[0] == 0 for c in plain["cand"])


def test_pick_fastest_first_on_ties_and_skips_failures(harness):
    assert _run(harness, True, 5.0, 3.0, 4.0, 3.0, 9, 9, 9, 9)["pick"] == 1       # tie: the earlier
    assert _run(harness, True, "inf", "inf", 7.5, "inf", 8, 9, 9, 9)["pick"] == 2  # failed candidates skipped
    assert _run(harness, True, "nan", 2.0)["pick"] == 1
    assert _run(harness, True, "inf", "inf")["pick"] == -1                      # nothing converged
    assert _run(harness, False, 1e300, 4.0)["pick"] == 1                        # the "failed" marker
