#!/usr/bin/env python
"""Benchmark of the EXX pair path on one GB300 (or N replicas under torchrun).

Headline workload (the largest single-GPU cell): a 10-step trajectory of 256
water-like molecules (1024 orbitals) in the triclinic cell
h = 37.3 [[1,0,0],[0.08,1,0],[0.04,0.06,1]] bohr on a 190^3 grid; per MD step a
symmetric strain N(0, 1e-3) and centre moves N(0, 0.05) bohr, orbitals
re-sampled; frozen proto-subdomains (offsets of step 0, Sec. III B 2),
R_pair / R_PE / R_ME = 8 / 6 / 8 bohr, 37-point NK stencil, CG tol 1e-9.  One
bench step = one full EXX evaluation of the next MD step (pair list -> every
pair's Poisson solve -> E_xx, D_xx, sigma_xx / Pi_xx) with the orbitals
resident in HBM, the mixed FP32/FP64 path.  The same line carries the plain
FP64 GPU path on a pair sample of MD step 0 (with the mixed path on the same
sample), both paths' errors against the FP64 oracle on that sample, the
end-to-end rate through the C ABI with host buffers, and the oracle's own rate
on the host cores.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload trajectory256|water64|triclinic128|batch3]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair Poisson solves/s and ms per EXX step (E_xx+D_xx+sigma_xx), %HBM roofline"
UNIT = "pair_solves/s"
WORKLOAD = ("water64_cubic23.5bohr_n120: 256 MLWFs, R_pair/R_PE/R_ME = 8/6/8 bohr, n = 3 (19-point stencil), "
            "l_max = 6, CG tol 1e-9, mixed FP32/FP64")
TRAJ_WORKLOAD = ("water256_triclinic37.3bohr_n190 trajectory: 1024 MLWFs, h = 37.3 [[1,0,0],[0.08,1,0],[0.04,0.06,1]] "
                 "bohr, 190^3 grid, 10 MD steps (symmetric strain N(0,1e-3), centres += N(0,0.05) bohr, orbitals "
                 "re-sampled), frozen offsets, R_pair/R_PE/R_ME = 8/6/8 bohr, 37-point NK stencil, l_max = 6, "
                 "CG tol 1e-9, E_xx + D_xx + sigma_xx per step")
N_MD = 10                 # MD steps of the trajectory; bench steps cycle through them
PRECONDS = {"mg": 1, "none": 0}   # exx PRECOND_MG / PRECOND_NONE
TRAJ_SEED_OFFSET = 500
FALLBACK_HBM = 6800.0


_T0 = time.time()


def log(msg: str) -> None:
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.time() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def measured_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.samples = []
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for p in self.samples:
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def profile_traffic(kernel_src_sha, workload="water64"):
    """DRAM bytes per launch of the pair solver from the committed ncu summary
    of this workload, if it was taken on the current kernel source."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    for f in sorted(os.listdir(d)):
        if not f.startswith("k_pair_solve") or not f.endswith(".md"):
            continue
        txt = open(os.path.join(d, f)).read()
        m_w = re.search(r"workload_key:\s*(\S+)", txt)
        if (m_w.group(1) if m_w else "water64") != workload:
            continue
        m_sha = re.search(r"kernel_source_sha256:\s*([0-9a-f]{64})", txt)
        m_b = re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
        if m_sha and m_b and m_sha.group(1) == kernel_src_sha:
            return float(m_b.group(1))
    return None


def kernel_sha():
    h = hashlib.sha256()
    for f in ("kernels.cu", "exx_dev.h", "kernels.h", "pair_rule.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2011_07209_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def rank_seed(rank: int) -> int:
    """Seed of the water64 cell solved by `rank`: every rank solves its own
    independent cell (weak scaling), rank 0 the seed of the single-GPU run."""
    return 7209 + 2 + 1000 * rank


def reduce_over_ranks(elapsed_ms: float, n_pairs: int, dist, device):
    """The slowest rank's timed region and the pairs of all ranks (one all-reduce
    each; the only collectives of a multi-rank run)."""
    if dist is None:
        return elapsed_ms, n_pairs
    import torch
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(n_pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(n.item()))


def algorithmic_bytes(n_pairs, total_iter, total_refine, n_pe, n_me, s, mg_points=None):
    """Bytes the pair solver must move per launch:
    CG: 7 N_PE s per iteration (x, r, p read + written, p read by the stencil);
    multigrid-preconditioned CG (mg_points = the active points of every level,
    fine first): 13 N_PE s per iteration (x, r, p read + written, p read by
    the stencil, and the V-cycle's fine level: r read by each of its two
    stencil passes, z0 written and read, z written and read) plus 8 n_l s on
    every coarse level (its R, Z, T boxes written and read, Z read once more
    by the prolongation, T by the restriction);
    true residual: FP64 path 24 N_PE (v, rho read, r written in FP64), mixed
    path 20 N_PE (v and 4 pi rho read as double-float pairs, r written in FP32);
    per pair: gather 2 N_ME 8, D read-modify-write 2 N_ME 16, rho 8 N_PE."""
    per_residual = 20.0 if s == 4 else 24.0
    if mg_points:
        per_iter = 13.0 * n_pe * s + 8.0 * s * sum(mg_points[1:])
    else:
        per_iter = 7.0 * n_pe * s
    return (total_iter * per_iter + total_refine * per_residual * n_pe
            + n_pairs * (2.0 * n_me * 8.0 + 2.0 * n_me * 16.0 + 8.0 * n_pe))


def mg_of(plan):
    """Multigrid level sizes when the plan's schedule uses the preconditioner."""
    if plan.schedule()["precond"] != "mg":
        return None
    return plan.info()["mg_points"] or None


def cpu_baseline(ws, n_sample, seed=7209):
    import numpy as np

    import oracle
    rows = oracle.pair_list(ws.lattice, ws.n, ws.centres, 8.0)
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(len(rows), size=min(n_sample, len(rows)), replace=False)).astype(np.int32)
    cores = os.cpu_count() or 1
    p = oracle.make_params(r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-9, n_threads=cores)
    t0 = time.perf_counter()
    oracle.exx(ws, p, sel=sel, want_d=False)
    dt = time.perf_counter() - t0
    return {"value": len(sel) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(sel)} seeded pairs of the same workload (FP64 CG to 1e-9, OpenMP over pairs), "
                      f"{dt:.1f} s wall"}


def run_reference(args, rank, world):
    """The oracle, as it stands, on bounded seeded samples of the headline
    workload's MD step 0 (one sample per step) on the host cores."""
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    import paper_2011_07209_gb300.synth as synth
    c = synth.CONFIGS[5]
    ws = synth.make_config(5)
    rows = oracle.pair_list(ws.lattice, ws.n, ws.centres, c["r_pair"])
    cores = os.cpu_count() or 1
    p = oracle.make_params(r_pair=c["r_pair"], r_pe=c["r_pe"], r_me=c["r_me"], tol=c["tol"], n_threads=cores,
                           lattice0=ws.lattice)
    rng = np.random.default_rng(7209)
    per_step = max(cores, args.ref_sample)
    times = []
    for it in range(args.warmup + args.steps):
        sel = np.sort(rng.choice(len(rows), size=per_step, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        oracle.exx(ws, p, sel=sel, want_d=False)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    tot = sum(times)
    val = per_step * len(times) / tot
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": TRAJ_WORKLOAD, "pairs_per_step": per_step, "total_pairs_in_cell": int(len(rows)),
                       "note": "each step is a bounded seeded sample of the pairs of MD step 0"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} seeded pairs of MD step 0 per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2011_07209_gb300.synth as synth
    from paper_2011_07209_gb300 import driver, exx

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    c = synth.CONFIGS[2]
    seed = rank_seed(rank)       # independent cell per rank (weak scaling)
    ws = synth.water_cell(c["lattice"], c["n"], c["n_mol"], seed)
    if args.subset > 0:
        ws = ws.subset(args.subset)
    ctx = exx.Context(local_rank)
    if args.solver == "cluster":
        ctx.set_solver(exx.SOLVER_CLUSTER)
    p = exx.make_params(r_pair=c["r_pair"], r_pe=c["r_pe"], r_me=c["r_me"], tol=c["tol"], precision=exx.MIXED,
                        precond=PRECONDS[args.precond])
    cr = driver.prepare(ctx, ws, p, device=local_rank)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ctx.set_timing(True)
    for _ in range(args.warmup):
        out = driver.run(ctx, cr, pair_outputs=False, stream=sh)
    torch.cuda.synchronize()
    info = cr.plan.info()      # after a solve: the persistent grid is known

    gpu_id = None
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        gpu_id = cvd.split(",")[local_rank].strip()
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    solve_ms, n_pairs, tot_iter, tot_ref = [], 0, 0, 0
    for _ in range(args.steps):
        out = driver.run(ctx, cr, pair_outputs=False, stream=sh)
        t = ctx.timing()
        solve_ms.append(t["solve_ms"])
        n_pairs = out["n_pairs"]
        tot_iter = out["total_cg_iter"]
        tot_ref = out["total_refine"]
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    elapsed, all_pairs = reduce_over_ranks(ev0.elapsed_time(ev1), n_pairs, dist, "cuda")
    ms_step = elapsed / args.steps
    value = all_pairs * args.steps / (elapsed / 1e3)

    # roofline of the dominant kernel (the persistent pair solver)
    s_bytes = 4.0
    bytes_launch = algorithmic_bytes(n_pairs, tot_iter, tot_ref, info["n_pe_pair"], info["n_me_pair"], s_bytes,
                                     mg_of(cr.plan))
    avg_solve = sum(solve_ms) / len(solve_ms)
    achieved = bytes_launch / (avg_solve / 1e3) / 1e9
    peak, peak_kind = measured_hbm()
    traffic = profile_traffic(kernel_sha())

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e = None
    if not args.no_e2e:
        phi_h = torch.empty(ws.phi.shape, dtype=torch.float64, pin_memory=True).numpy()
        phi_h[...] = ws.phi
        cen_h = torch.empty(ws.centres.shape, dtype=torch.float64, pin_memory=True).numpy()
        cen_h[...] = ws.centres
        lo_h = torch.empty(ws.box_lo.shape, dtype=torch.int32, pin_memory=True).numpy()
        lo_h[...] = ws.box_lo
        dxx_h = torch.empty((ws.n_orb,) + tuple(int(x) for x in cr.dbox), dtype=torch.float64,
                            pin_memory=True).numpy()
        dlo_h = torch.empty(cr.dbox_lo_np.shape, dtype=torch.int32, pin_memory=True).numpy()
        dlo_h[...] = cr.dbox_lo_np
        orb = exx.make_orbitals(ws.n_orb, ws.box, cen_h, lo_h, phi_h, exx.MEM_HOST)
        res = exx.make_result(dxx_h, cr.dbox, dlo_h, exx.MEM_HOST)
        exx.solve(ctx, cr.plan, ws.lattice, ws.n, orb, res, stream=sh)     # warm (allocates staging)
        n_e2e = max(2, min(args.steps, 3))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_e2e):
            exx.solve(ctx, cr.plan, ws.lattice, ws.n, orb, res, stream=sh)
        e1.record(stream)
        torch.cuda.synchronize()
        et, e2e_pairs = reduce_over_ranks(e0.elapsed_time(e1) / n_e2e, res.n_pairs, dist, "cuda")
        h2d = phi_h.nbytes + cen_h.nbytes + lo_h.nbytes + dlo_h.nbytes
        d2h = dxx_h.nbytes + 19 * 8
        e2e = {"value": e2e_pairs / (et / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": et}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(ws, args.cpu_sample)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "mixed-f32-f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + (f" [profiling subset: first {args.subset} MLWFs]" if args.subset else ""),
                       "pairs_per_step": n_pairs, "n_pe": info["n_pe_pair"],
                       "n_me": info["n_me_pair"], "n_stcl": info["n_stcl"],
                       "mean_cg_iter": tot_iter / max(n_pairs, 1), "mean_true_residuals": tot_ref / max(n_pairs, 1),
                       "ctas": info["ctas"], "threads": info["threads"], "ctas_per_pair": info["cluster"],
                       "l2": "inputs larger than L2 (orbital boxes 512 MB, D_xx 3.5 GB per step)",
                       "parallelism": f"replicas{world}" if world > 1 else "single-gpu"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic if args.solver == "cta" else None,
                         "kernel": "k_pair_solve<float>" if args.solver == "cta" else "k_pair_solve_cluster",
                         "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_ms": avg_solve,
                         "peak_kind": f"{peak_kind} HBM copy bandwidth"},
            "clocks": clocks,
            "gpu_launches": 5 * args.steps,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def traj_cell(rank: int):
    """Step-0 cell of the trajectory solved by `rank` (rank 0: the seeded
    config; other ranks: an independent cell of the same size, weak scaling)."""
    import paper_2011_07209_gb300.synth as synth
    if rank == 0:
        return synth.make_config(5)
    c = synth.CONFIGS[5]
    return synth.water_cell(c["lattice"], c["n"], c["n_mol"], synth.SEED_BASE + 5 + 1000 * rank)


def traj_steps(ws0, rank: int):
    """The N_MD cells of the trajectory, on boxes of one common size."""
    import numpy as np

    import paper_2011_07209_gb300.synth as synth
    steps = synth.trajectory(ws0, N_MD, seed=synth.SEED_BASE + TRAJ_SEED_OFFSET + 1000 * rank)
    box = np.max([w.box for w in steps], axis=0)
    return [w if np.array_equal(w.box, box) else w.padded(box) for w in steps]


def accuracy_sample(pairs, n_sample, d_orbs=(0, 1), seed=7209):
    """Pair indices for the oracle comparison: every pair touching the orbitals
    whose D_xx is checked, plus seeded random pairs up to n_sample."""
    import numpy as np
    touch = np.nonzero(np.isin(pairs[:, 0], d_orbs) | np.isin(pairs[:, 1], d_orbs))[0]
    rest = np.setdiff1d(np.arange(len(pairs)), touch)
    rng = np.random.default_rng(seed)
    k = max(0, min(n_sample - len(touch), len(rest)))
    extra = rng.choice(rest, size=k, replace=False) if k else np.empty(0, np.int64)
    return np.sort(np.concatenate([touch, extra])).astype(np.int32)


def compare_with_oracle(g, o, sel, lattice, dxx_gpu=None, dxx_orc=None, d_orbs=(0, 1)):
    """Largest errors of the GPU's per-pair results on the sampled pairs: E_pair
    relative, the pair's contribution to Pi (Ha/bohr^3, absolute), and D_xx
    (max abs over the boxes of the checked orbitals)."""
    import numpy as np
    h = np.asarray(lattice, float).T
    vol = abs(np.linalg.det(h))
    rel_e, d_pi = 0.0, 0.0
    for k in sel:
        i, j = int(o["pairs"][k][0]), int(o["pairs"][k][1])
        w = 1.0 if i == j else 2.0
        ref = o["pair_e"][k]
        rel_e = max(rel_e, abs(g["pair_e"][k] - ref) / abs(ref))
        dsig = -2.0 * w * (g["pair_sig"][k] - o["pair_sig"][k])     # sigma^{a alpha} contribution
        d_pi = max(d_pi, float(np.abs(-(dsig @ h.T) / vol).max()))
    out = {"pairs": int(len(sel)), "max_rel_err_e_pair": rel_e, "max_abs_err_pi_pair_ha_bohr3": d_pi}
    if dxx_gpu is not None:
        out["max_abs_err_dxx"] = float(max(np.abs(dxx_gpu[i] - dxx_orc[i]).max() for i in d_orbs))
        out["dxx_orbitals"] = list(d_orbs)
    return out


def run_trajectory(args, rank, world, local_rank):
    """Headline: the 1024-orbital triclinic trajectory (see the module docstring)."""
    import numpy as np
    import torch

    import paper_2011_07209_gb300.synth as synth
    from paper_2011_07209_gb300 import driver, exx

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    c = synth.CONFIGS[5]
    shard = args.shard and world > 1
    log("generating the trajectory")
    ws0 = traj_cell(0 if shard else rank)      # sharded: every rank holds the same cell
    steps = traj_steps(ws0, 0 if shard else rank)
    log("trajectory ready; plan and device inputs")
    box = steps[0].box
    ctx = exx.Context(local_rank)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    # a pair that fails to converge stops at 3000 iterations (plain CG needs about 250)
    mk = dict(r_pair=c["r_pair"], r_pe=c["r_pe"], r_me=c["r_me"], tol=c["tol"], frozen=True, max_iter=3000)
    pc = PRECONDS[args.precond]
    p = exx.make_params(precision=exx.MIXED, warm_start=args.warm, precond=pc, **mk)
    plan = exx.Plan(ctx, ws0.lattice, ws0.n, p, ws0.n_orb, box)
    if shard:
        plan.set_shard(rank, world)
    dbox = np.max([exx.dbox_layout(w.lattice, w.n, w.centres, p)[0] for w in steps], axis=0)
    dxx = torch.zeros((ws0.n_orb,) + tuple(int(b) for b in dbox), dtype=torch.float64, device="cuda")
    runs = [driver.prepare(ctx, w, p, plan=plan, dxx=dxx, device=local_rank) for w in steps]
    ctx.set_timing(True)
    if args.autotune:
        w0 = runs[0]
        sched = plan.autotune(ctx, w0.ws.lattice, w0.ws.n, w0.orbitals(), sample_pairs=args.autotune, stream=sh)
        log(f"autotuned schedule {sched}")
    log("warm-up")
    for k in range(args.warmup):
        driver.run(ctx, runs[k % N_MD], pair_outputs=False, stream=sh)
    torch.cuda.synchronize()
    info = plan.info()
    log("timed steps")

    gpu_id = None
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES")
    if cvd:
        gpu_id = cvd.split(",")[local_rank].strip()
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    solve_ms, n_pairs, tot_iter, tot_ref, bytes_launch = [], 0, 0, 0, 0.0
    for k in range(args.steps):
        out = driver.run(ctx, runs[k % N_MD], pair_outputs=False, stream=sh)
        solve_ms.append(ctx.timing()["solve_ms"])
        if shard:   # E_xx, sigma, Pi and D_xx summed over the ranks (NCCL all-reduce)
            driver.reduce_shards(out, runs[k % N_MD].dxx, dist)
        n_pairs += out["n_pairs"]
        tot_iter += out["total_cg_iter"]
        tot_ref += out["total_refine"]
        bytes_launch += algorithmic_bytes(out["n_pairs"], out["total_cg_iter"], out["total_refine"],
                                          info["n_pe_pair"], info["n_me_pair"], 4.0, mg_of(plan))
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    elapsed, all_pairs = reduce_over_ranks(ev0.elapsed_time(ev1), n_pairs, dist, "cuda")
    if shard:
        all_pairs = n_pairs          # one cell shared by the ranks: its pairs count once
    ms_step = elapsed / args.steps
    value = all_pairs / (elapsed / 1e3)
    avg_solve = sum(solve_ms) / len(solve_ms)
    achieved = bytes_launch / args.steps / (avg_solve / 1e3) / 1e9
    peak, peak_kind = measured_hbm()
    traffic = profile_traffic(kernel_sha(), "trajectory256")
    log(f"timed: {ms_step:.1f} ms per step, {value:.1f} pair solves/s")

    # end to end through the C ABI with pinned host buffers: every step copies its
    # orbitals in and its D_xx out inside the timed region
    e2e = None
    if not args.no_e2e and not shard:
        log("end-to-end leg: pinned host buffers")
        n_e2e = min(args.steps, N_MD)
        n_buf = min(n_e2e, 4)
        host = []
        for si, w in enumerate(steps[:n_buf]):
            phi_h = torch.empty(w.phi.shape, dtype=torch.float64, pin_memory=True).numpy()
            phi_h[...] = w.phi
            cen_h = torch.empty(w.centres.shape, dtype=torch.float64, pin_memory=True).numpy()
            cen_h[...] = w.centres
            lo_h = torch.empty(w.box_lo.shape, dtype=torch.int32, pin_memory=True).numpy()
            lo_h[...] = w.box_lo
            dlo_h = torch.empty(runs[0].dbox_lo_np.shape, dtype=torch.int32, pin_memory=True).numpy()
            dlo_h[...] = runs[si].dbox_lo_np
            # the orbitals structure holds raw pointers: keep the buffers alive beside it
            host.append((w, exx.make_orbitals(w.n_orb, w.box, cen_h, lo_h, phi_h, exx.MEM_HOST), dlo_h,
                         phi_h.nbytes + cen_h.nbytes + lo_h.nbytes + dlo_h.nbytes, (phi_h, cen_h, lo_h)))
        del dxx, runs
        torch.cuda.empty_cache()
        dxx_h = torch.empty((ws0.n_orb,) + tuple(int(x) for x in dbox), dtype=torch.float64, pin_memory=True).numpy()
        w, orb, dlo_h, _, _ = host[0]
        log("end-to-end leg: warm call")
        exx.solve(ctx, plan, w.lattice, w.n, orb, exx.make_result(dxx_h, dbox, dlo_h, exx.MEM_HOST), stream=sh)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_pairs, h2d = 0, 0
        for k in range(n_e2e):
            w, orb, dlo_h, nb, _ = host[k % n_buf]
            res = exx.make_result(dxx_h, dbox, dlo_h, exx.MEM_HOST)
            exx.solve(ctx, plan, w.lattice, w.n, orb, res, stream=sh)
            e2e_pairs += res.n_pairs
            h2d += nb
        e1.record(stream)
        torch.cuda.synchronize()
        et, e2e_all = reduce_over_ranks(e0.elapsed_time(e1), e2e_pairs, dist, "cuda")
        e2e = {"value": e2e_all / (et / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d // n_e2e),
               "d2h_bytes_per_step": int(dxx_h.nbytes + 19 * 8), "ms_per_step": et / n_e2e, "steps": n_e2e,
               "note": f"MD steps 0..{n_e2e - 1} of the trajectory, host inputs from {n_buf} pinned buffers"}
        del host, dxx_h
    else:
        del dxx, runs
        torch.cuda.empty_cache()

    # plain FP64 GPU path beside the mixed one on a pair sample of MD step 0 (the
    # pairs of its first --arm-orbitals MLWFs), and both against the FP64 oracle
    arms, accuracy, cpu = None, None, None
    if rank == 0 and not args.no_arms and not shard:
        sub = steps[0].subset(args.arm_orbitals) if args.arm_orbitals < ws0.n_orb else steps[0]
        arms, gouts, gruns = {}, {}, {}
        # the FP64 path at the same stopping rule, and at tol 1e-8 (closer to the mixed
        # path's own accuracy, which its FP32 moment tables set near 1e-8 in E)
        for name, prec, tol in (("mixed", exx.MIXED, c["tol"]), ("fp64", exx.FP64, c["tol"]),
                                ("fp64_tol1e-8", exx.FP64, 1e-8)):
            log(f"{name} arm on {sub.n_orb} MLWFs of MD step 0")
            pp = exx.make_params(precision=prec, precond=pc, **dict(mk, tol=tol))
            pl = exx.Plan(ctx, ws0.lattice, ws0.n, pp, sub.n_orb, box)
            cr = driver.prepare(ctx, sub, pp, plan=pl, device=local_rank)
            driver.run(ctx, cr, pair_outputs=False, stream=sh)       # warm (allocates the solver's slots)
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            o = driver.run(ctx, cr, pair_outputs=True, stream=sh)
            a1.record(stream)
            torch.cuda.synchronize()
            ms = a0.elapsed_time(a1)
            arms[name] = {"value": o["n_pairs"] / (ms / 1e3), "unit": UNIT, "ms": ms, "pairs": o["n_pairs"],
                          "mean_cg_iter": o["total_cg_iter"] / max(o["n_pairs"], 1), "cg_tol": tol}
            gouts[name] = o
            gruns[name] = cr
        arms["mixed_over_fp64_speed"] = arms["mixed"]["value"] / arms["fp64"]["value"]
        arms["mixed_over_fp64_tol1e-8_speed"] = arms["mixed"]["value"] / arms["fp64_tol1e-8"]["value"]
        arms["sample"] = (f"all {arms['mixed']['pairs']} pairs of the first {sub.n_orb} MLWFs of MD step 0 "
                          f"(same cell, frozen plan), one timed solve each after one warm-up")
        if not args.no_cpu:
            import oracle
            log("oracle on the accuracy sample")
            g0 = gouts["mixed"]
            sel = accuracy_sample(g0["pairs"], args.cpu_sample)
            cores = os.cpu_count() or 1
            op = oracle.make_params(r_pair=c["r_pair"], r_pe=c["r_pe"], r_me=c["r_me"], tol=c["tol"],
                                    n_threads=cores, lattice0=ws0.lattice)
            t0 = time.perf_counter()
            o = oracle.exx(sub, op, sel=sel, want_d=True, dbox=gruns["mixed"].dbox, dbox_lo=gruns["mixed"].dbox_lo_np)
            dt = time.perf_counter() - t0
            assert np.array_equal(o["pairs"], g0["pairs"]), "pair list differs from the oracle's"
            cpu = {"value": len(sel) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{len(sel)} pairs of MD step 0 (every pair of MLWFs 0 and 1, the rest seeded random; "
                             f"FP64 CG to {c['tol']:g}, OpenMP over pairs, D_xx on), {dt:.1f} s wall"}
            accuracy = {"oracle": f"FP64 oracle, CG tol {c['tol']:g}, same pairs"}
            for name in ("mixed", "fp64", "fp64_tol1e-8"):
                d_g = gruns[name].dxx.cpu().numpy()[:2]
                accuracy[name] = compare_with_oracle(gouts[name], o, sel, sub.lattice, d_g, o["dxx"][:2])

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "strong" if shard else "weak",
            "vs_baseline": None, "dtype": "mixed-f32-f64", "data": "synthetic",
            "config": {"workload": TRAJ_WORKLOAD, "md_steps_cycled": N_MD, "schedule": plan.schedule(),
                       "pairs_per_step": n_pairs / args.steps, "autotuned": bool(args.autotune), "n_pe": info["n_pe_pair"],
                       "n_me": info["n_me_pair"], "n_stcl": info["n_stcl"],
                       "mean_cg_iter": tot_iter / max(n_pairs, 1), "mean_true_residuals": tot_ref / max(n_pairs, 1),
                       "ctas": info["ctas"], "threads": info["threads"], "ctas_per_pair": info["cluster"],
                       "l2": "inputs larger than L2 (orbital boxes 2 GB per MD step, D_xx 16.8 GB)",
                       "parallelism": (f"pair-sharded{world}" if shard else f"replicas{world}") if world > 1
                       else "single-gpu"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": "k_pair_solve<float>",
                         "algorithmic_bytes_per_launch": bytes_launch / args.steps, "avg_launch_ms": avg_solve,
                         "peak_kind": f"{peak_kind} HBM copy bandwidth"},
            "clocks": clocks,
            "gpu_launches": 9 * args.steps,
            "e2e": e2e,
            "fp64_arm": arms,
            "accuracy_vs_oracle": accuracy,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


WORKLOADS = {
    "triclinic128": "water128_triclinic29.6bohr_n150: 512 MLWFs, R_pair/R_PE/R_ME = 8/6/8 bohr, 37-point NK "
                    "stencil (3 aux directions), CG tol 1e-9",
    "batch3": "three cells in one launch: water32 cubic 18.6 (93^3), water96 26.8x26.8x28.0 (134x134x140), "
              "water192 monoclinic 33.9 shear 0.12 (169x169x171); R_PE from {5,6,7} per cell, R_ME 8, CG tol 1e-9",
}


def run_workload(args, rank, world, local_rank):
    """The other benchmark cells (one JSON line; no e2e or CPU arm)."""
    import numpy as np
    import torch

    import paper_2011_07209_gb300.synth as synth
    from paper_2011_07209_gb300 import driver, exx

    torch.cuda.set_device(local_rank)
    ctx = exx.Context(local_rank)
    prec = exx.FP64 if args.precision == "fp64" else exx.MIXED
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    ctx.set_timing(True)
    n_total = args.warmup + args.steps
    if args.workload == "triclinic128":
        c = synth.CONFIGS[3]
        ws = synth.make_config(3)
        if args.subset > 0:
            ws = ws.subset(args.subset)
        p = exx.make_params(r_pair=8.0, r_pe=6.0, r_me=8.0, tol=c["tol"], precision=prec,
                            precond=PRECONDS[args.precond])
        cr = driver.prepare(ctx, ws, p)
        step_runs = [[cr]] * n_total
    elif args.workload == "batch3":
        runs = []
        for name, ws, r_pe in synth.make_batch(4):
            p = exx.make_params(r_pair=8.0, r_pe=r_pe, r_me=8.0, tol=1e-9, precision=prec,
                                precond=PRECONDS[args.precond])
            runs.append(driver.prepare(ctx, ws, p))
        step_runs = [runs] * n_total
    else:
        raise ValueError(args.workload)

    schedules = []
    if args.autotune:
        for r in step_runs[0]:
            schedules.append(r.plan.autotune(ctx, r.ws.lattice, r.ws.n, r.orbitals(), sample_pairs=args.autotune,
                                             stream=sh))
    else:
        schedules = [r.plan.schedule() for r in step_runs[0]]

    def one(runs):
        if len(runs) == 1:
            o = driver.run(ctx, runs[0], pair_outputs=False, stream=sh)
            return [o], ctx.timing()["solve_ms"]
        o = driver.run_batch(ctx, runs, stream=sh)
        return o, ctx.timing()["solve_ms"]

    for k in range(args.warmup):
        one(step_runs[k])
    torch.cuda.synchronize()
    sampler = ClockSampler(None)
    sampler.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    n_pairs = tot_iter = tot_ref = n_warm = 0
    solve_ms = []
    bytes_launch = 0.0
    for k in range(args.warmup, n_total):
        outs, ms = one(step_runs[k])
        solve_ms.append(ms)
        for o, r in zip(outs, step_runs[k]):
            info = r.plan.info()
            n_pairs += o["n_pairs"]
            tot_iter += o["total_cg_iter"]
            tot_ref += o["total_refine"]
            n_warm += o.get("n_warm", 0)
            bytes_launch += algorithmic_bytes(o["n_pairs"], o["total_cg_iter"], o["total_refine"], info["n_pe_pair"],
                                              info["n_me_pair"], 8.0 if prec == exx.FP64 else 4.0, mg_of(r.plan))
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    elapsed = ev0.elapsed_time(ev1)
    peak, peak_kind = measured_hbm()
    avg_solve = sum(solve_ms) / len(solve_ms)
    achieved = bytes_launch / args.steps / (avg_solve / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": n_pairs / (elapsed / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == exx.FP64 else "mixed-f32-f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload] + (f" [profiling subset: first {args.subset} MLWFs]"
                                                             if args.subset else ""),
                   "pairs_per_step": n_pairs / args.steps,
                   "schedules": schedules, "autotuned": bool(args.autotune),
                   "mean_cg_iter": tot_iter / max(n_pairs, 1), "mean_true_residuals": tot_ref / max(n_pairs, 1),
                   "warm_started_pairs_per_step": n_warm / args.steps},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_pair_solve", "avg_launch_ms": avg_solve,
                     "peak_kind": f"{peak_kind} HBM copy bandwidth"},
        "clocks": clocks, "gpu_launches": 5 * args.steps, "e2e": None, "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=256, help="oracle pairs of the CPU baseline (about 10 s)")
    ap.add_argument("--ref-sample", type=int, default=16, help="oracle pairs per step of --impl reference")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-arms", action="store_true", help="skip the FP64 arm and the oracle comparison")
    ap.add_argument("--arm-orbitals", type=int, default=256,
                    help="the FP64 arm and the accuracy check solve the pairs of the first K MLWFs of MD step 0")
    ap.add_argument("--warm", action="store_true", help="trajectory256 with warm-started CG (previous MD step)")
    ap.add_argument("--shard", action="store_true",
                    help="trajectory256 under torchrun: the ranks share one cell's pairs (LPT partition, all-reduce "
                         "of E, sigma and D per step; strong scaling) instead of solving one cell each")
    ap.add_argument("--autotune", type=int, default=1216,
                    help="autotune each plan's solver schedule on this many pairs first (0: the default schedule)")
    ap.add_argument("--workload", default="trajectory256", choices=["trajectory256", "water64"] + sorted(WORKLOADS),
                    help="trajectory256 is the headline workload; the others print their own line")
    ap.add_argument("--precond", default="mg", choices=sorted(PRECONDS),
                    help="mixed path's CG: multigrid-preconditioned (default) or plain")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="for --workload triclinic128 and batch3")
    ap.add_argument("--solver", default="cta", choices=["cta", "cluster"],
                    help="water64: one CTA per pair (default) or one 16-CTA cluster per pair")
    ap.add_argument("--subset", type=int, default=0,
                    help="water64, triclinic128: solve only the pairs of the first K MLWFs (a small case for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "trajectory256":
        return run_trajectory(args, rank, world, local_rank)
    if args.workload == "water64":
        return run_gpu(args, rank, world, local_rank)
    if world > 1:
        print(json.dumps({"error": f"--workload {args.workload} runs on one GPU"}))
        return 1
    return run_workload(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
