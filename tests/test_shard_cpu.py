"""Pair sharding of one cell over ranks, on CPU with two gloo ranks.

The paper distributes the unique pairs over MPI processes and sums E_xx and
sigma_xx over them, each process returning its D_ji contributions (Sec. III A,
Steps II and V).  Here every rank computes the same longest-processing-time
partition of the pair list (exx_pair_partition, host code of the library),
forms its partial results, and driver.reduce_shards sums them with one
all-reduce of 20 doubles and one of the D boxes.  The rank-local partial
results are the oracle's (stored per-pair values of the 64-molecule cell; the
oracle run on each rank's own pairs of the 4-molecule cell for D_xx), so the
check needs no GPU: the partition covers every pair exactly once, the loads
balance, and the reduced sums are the single-rank results.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_water64.npz")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _partials(g, mine):
    """-sum w E_pair, sigma = -2 sum w sig_pair, Pi = -sigma h^T / V over the given pairs."""
    rows = g["rows"].astype(np.int64)
    w = np.where(rows[:, 0] == rows[:, 1], 1.0, 2.0)[mine]
    e = -float((w * g["pair_e"][mine]).sum())
    sig = -2.0 * np.einsum("p,pab->ab", w, g["pair_sig"][mine])
    h = np.asarray(g["lattice"], float).T
    pi = -(sig @ h.T) / abs(np.linalg.det(h))
    return {"e_xx": e, "dedh": sig, "stress": pi, "p_int": float(np.trace(pi)) / 3.0}


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ["OMP_NUM_THREADS"] = "2"
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2011_07209_gb300 import driver, exx, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {}
    # 64-molecule cell: the partition and the E / sigma / Pi reduction
    g = dict(np.load(GOLDEN))
    p = exx.make_params(r_pair=float(g["r_pair"]), r_pe=float(g["r_pe"]), r_me=float(g["r_me"]))
    owner = exx.pair_partition(g["lattice"], g["n"], p, g["rows"], world)
    all_owners = [torch.zeros(len(owner), dtype=torch.int32) for _ in range(world)]
    dist.all_gather(all_owners, torch.as_tensor(owner))
    res["same_partition"] = all(np.array_equal(o.numpy(), owner) for o in all_owners)
    res["counts"] = np.bincount(owner, minlength=world).tolist()
    mine = np.nonzero(owner == rank)[0]
    red = driver.reduce_shards(_partials(g, mine), None, dist)
    res["e_xx"] = red["e_xx"]
    res["e_xx_ref"] = float(g["e_xx"])
    res["dedh_err"] = float(np.abs(red["dedh"] - g["dedh"]).max())
    res["stress_err"] = float(np.abs(red["stress"] - g["stress"]).max())
    # 4-molecule cell: D_xx boxes summed over the ranks' own pairs
    ws = synth.make_config(1)
    op = oracle.make_params(r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-10)
    rows = oracle.pair_list(ws.lattice, ws.n, ws.centres, 8.0)
    own1 = np.nonzero(exx.pair_partition(ws.lattice, ws.n, exx.make_params(), rows, world) == rank)[0]
    full = oracle.exx(ws, op)
    part = oracle.exx(ws, op, sel=own1.astype(np.int32), dbox=full["dbox"], dbox_lo=full["dbox_lo"])
    dxx = torch.as_tensor(part["dxx"].copy())
    out = {"e_xx": part["e_xx"], "dedh": part["dedh"], "stress": part["stress"], "p_int": 0.0}
    red1 = driver.reduce_shards(out, dxx, dist)
    res["d_err"] = float(np.abs(dxx.numpy() - full["dxx"]).max())
    res["d_max"] = float(np.abs(full["dxx"]).max())
    res["e1_rel"] = abs(red1["e_xx"] / full["e_xx"] - 1.0)
    res["n_own1"] = int(len(own1))
    dist.barrier()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_one_cell(tmp_path):
    if not os.path.exists(GOLDEN):
        pytest.skip("stored oracle results not generated")
    mp = pytest.importorskip("torch.multiprocessing")
    from paper_2011_07209_gb300 import build
    build.build()
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    for x in r:
        assert x["same_partition"]
        c0, c1 = x["counts"]
        assert abs(c0 - c1) <= 1                      # equal-cost pairs: LPT alternates
        assert x["e_xx"] == pytest.approx(x["e_xx_ref"], rel=1e-12)
        assert x["dedh_err"] < 1e-12 * 10 and x["stress_err"] < 1e-15
        assert x["d_err"] <= 1e-12 * x["d_max"]
        assert x["e1_rel"] < 1e-12
    assert r[0]["n_own1"] > 0 and r[1]["n_own1"] > 0


def test_lpt_partition_two_cost_classes():
    """Self pairs with a larger subdomain go first; the loads stay within one pair's cost."""
    from paper_2011_07209_gb300 import build, exx
    build.build()
    lat = np.diag([23.5] * 3)
    n = (120, 120, 120)
    p = exx.make_params(r_pe_self=6.0, r_me_self=8.0, r_pe=5.0, r_me=7.0)
    rng = np.random.default_rng(1)
    rows = np.zeros((200, 8), np.int32)
    rows[:, 0] = rng.integers(0, 50, 200)
    rows[:, 1] = np.where(rng.random(200) < 0.2, rows[:, 0], rows[:, 0] + 1)
    geo = exx.geometry(lat, n, p)
    cost = np.where(rows[:, 0] == rows[:, 1], geo["n_pe_self"], geo["n_pe_pair"]).astype(float)
    for world in (1, 3, 4):
        owner = exx.pair_partition(lat, n, p, rows, world)
        loads = np.bincount(owner, weights=cost, minlength=world)
        assert owner.min() >= 0 and owner.max() < world
        assert loads.max() - loads.min() <= cost.max()
