"""Host logic of bench.py that needs no GPU: the algorithmic byte count of a
solver launch and the rule that DRAM traffic is reported only from a profile
taken on the current kernel source."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_mixed_and_fp64():
    n_pairs, it, ref, n_pe, n_me = 3, 100, 7, 1000, 2500
    per_pair = 2 * n_me * 8 + 2 * n_me * 16 + 8 * n_pe
    # mixed: 7 FP32 accesses per CG point-iteration, 20 B per point for a
    # double-float true residual (v and 4 pi rho pairs read, r written in FP32)
    assert bench.algorithmic_bytes(n_pairs, it, ref, n_pe, n_me, 4) == it * 7 * n_pe * 4 + ref * 20 * n_pe \
        + n_pairs * per_pair
    # FP64: 7 FP64 accesses, 24 B per point for an FP64 residual
    assert bench.algorithmic_bytes(n_pairs, it, ref, n_pe, n_me, 8) == it * 7 * n_pe * 8 + ref * 24 * n_pe \
        + n_pairs * per_pair


def _profile(sha, traffic):
    return (f"# k_pair_solve summary\n\nkernel_source_sha256: {sha}\n\n"
            f"dram_bytes_per_full_launch: {traffic}\n")


def test_traffic_only_from_a_profile_of_the_current_source(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    sha = "ab" * 32
    (tmp_path / "profiles" / "k_pair_solve_case.md").write_text(_profile(sha, "6.25e12"))
    (tmp_path / "profiles" / "other_kernel.md").write_text(_profile("cd" * 32, "1e9"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic(sha) == 6.25e12
    assert bench.profile_traffic("cd" * 32) is None        # only k_pair_solve summaries count
    assert bench.profile_traffic("ef" * 32) is None        # a changed kernel has no traffic figure


def test_kernel_sha_covers_the_solver_sources(tmp_path, monkeypatch):
    src = tmp_path / "paper_2011_07209_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in ("kernels.cu", "exx_dev.h", "kernels.h", "pair_rule.cuh"):
        (src / f).write_text(f"// {f}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    a = bench.kernel_sha()
    (src / "exx_dev.h").write_text("// changed\n")
    assert bench.kernel_sha() != a


def test_algorithmic_bytes_multigrid():
    n_pairs, it, ref, n_pe, n_me = 2, 15, 3, 1000, 2500
    per_pair = 2 * n_me * 8 + 2 * n_me * 16 + 8 * n_pe
    levels = [1000, 140, 20]
    # 13 FP32 accesses per fine point-iteration, 8 per coarse point
    assert bench.algorithmic_bytes(n_pairs, it, ref, n_pe, n_me, 4, levels) == \
        it * (13 * n_pe * 4 + 8 * 4 * 160) + ref * 20 * n_pe + n_pairs * per_pair
