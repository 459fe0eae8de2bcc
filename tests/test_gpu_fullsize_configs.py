"""Full-size parity on the other benchmark cells, in the launch configuration of
the benchmark (mixed precision, one persistent launch per solve):

  * triclinic 128-molecule cell (512 MLWFs, 150^3, 37-point NK stencil);
  * three uneven cells (32 / 96 / 192 molecules, R_PE drawn from {5, 6, 7})
    solved together in one batched launch;
  * the first two steps of the 256-molecule triclinic trajectory (1024 MLWFs,
    190^3) with frozen offsets and warm-started CG.

As in the 64-molecule test, the pair lists are compared bit for bit, a seeded
sample of pairs is solved by the oracle one by one, and every pair must
converge.
"""
import numpy as np
import pytest

import oracle
import paper_2011_07209_gb300.synth as synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_07209_gb300 import exx
    c = exx.Context(0)
    yield c
    c.close()


def _sample(out, k, seed):
    rng = np.random.default_rng(seed)
    n = out["n_pairs"]
    sel = rng.choice(n, size=min(k, n), replace=False)
    selfs = np.nonzero(out["pairs"][:, 0] == out["pairs"][:, 1])[0]
    return np.unique(np.concatenate([sel, selfs[:1]])).astype(np.int32)


def _check_sampled(out, o, sel, rel=1e-7):
    for k in sel:
        assert out["pair_e"][k] == pytest.approx(o["pair_e"][k], rel=rel)
        scale = np.abs(o["pair_sig"][k]).max()
        assert np.abs(out["pair_sig"][k] - o["pair_sig"][k]).max() < 1e-6 * scale


def test_triclinic_128_molecules(ctx):
    from paper_2011_07209_gb300 import driver, exx
    c = synth.CONFIGS[3]
    ws = synth.make_config(3)
    p = exx.make_params(r_pair=c["r_pair"], r_pe=c["r_pe"], r_me=c["r_me"], tol=c["tol"], precision=exx.MIXED)
    out = driver.run(ctx, driver.prepare(ctx, ws, p, want_d=False))
    assert out["status"] == 0 and out["failed_pair"] == -1
    assert out["n_aux"] == 3 and out["n_stcl"] == 37
    assert np.array_equal(out["pairs"], oracle.pair_list(ws.lattice, ws.n, ws.centres, c["r_pair"]))
    assert out["pair_iter"].max() < 1000
    sel = _sample(out, 8, 3)
    o = oracle.exx(ws, oracle.make_params(r_pair=c["r_pair"], r_pe=c["r_pe"], r_me=c["r_me"], tol=c["tol"]),
                   sel=sel, want_d=False)
    _check_sampled(out, o, sel)


def test_batched_three_cells(ctx):
    from paper_2011_07209_gb300 import driver, exx
    runs, cells = [], synth.make_batch(4)
    for name, ws, r_pe in cells:
        p = exx.make_params(r_pair=8.0, r_pe=r_pe, r_me=8.0, tol=1e-9, precision=exx.MIXED)
        runs.append(driver.prepare(ctx, ws, p, want_d=False))
    outs = driver.run_batch(ctx, runs, pair_outputs=True)
    for (name, ws, r_pe), out in zip(cells, outs):
        assert out["status"] == 0, name
        pairs = runs[[c[0] for c in cells].index(name)].plan.pair_list()
        assert np.array_equal(pairs, oracle.pair_list(ws.lattice, ws.n, ws.centres, 8.0)), name
        assert out["n_pairs"] == len(pairs)
    # sampled pairs of each cell against the oracle with that cell's R_PE
    for ci, ((name, ws, r_pe), out, run) in enumerate(zip(cells, outs, runs)):
        e = run.pair_e[:out["n_pairs"]].cpu().numpy()
        sig = run.pair_sig[:out["n_pairs"]].cpu().numpy()
        pairs = run.plan.pair_list()
        view = {"pair_e": e, "pair_sig": sig, "pairs": pairs, "n_pairs": out["n_pairs"]}
        sel = _sample(view, 4, 40 + ci)
        o = oracle.exx(ws, oracle.make_params(r_pair=8.0, r_pe=r_pe, r_me=8.0, tol=1e-9), sel=sel, want_d=False)
        _check_sampled(view, o, sel)


def test_trajectory_first_steps_frozen_warm(ctx):
    from paper_2011_07209_gb300 import driver, exx
    c = synth.CONFIGS[5]
    ws0 = synth.make_config(5)
    steps = synth.trajectory(ws0, 2, seed=synth.SEED_BASE + 500)
    box = np.max([w.box for w in steps], axis=0)
    steps = [w.padded(box) for w in steps]
    lat0 = ws0.lattice
    # guess off: every pair of the second step keeps its previous solution as the start
    p = exx.make_params(r_pair=c["r_pair"], r_pe=c["r_pe"], r_me=c["r_me"], tol=c["tol"], precision=exx.MIXED,
                        frozen=True, warm_start=True, guess=False)
    plan = exx.Plan(ctx, lat0, ws0.n, p, ws0.n_orb, box)
    outs = []
    for ws in steps:
        out = driver.run(ctx, driver.prepare(ctx, ws, p, plan=plan, want_d=False))
        assert out["status"] == 0 and out["failed_pair"] == -1
        outs.append(out)
    assert outs[0]["n_warm"] == 0 and outs[1]["n_warm"] > 0.9 * outs[1]["n_pairs"]
    ws = steps[1]
    assert np.array_equal(outs[1]["pairs"], oracle.pair_list(ws.lattice, ws.n, ws.centres, c["r_pair"]))
    sel = _sample(outs[1], 6, 5)
    o = oracle.exx(ws, oracle.make_params(r_pair=c["r_pair"], r_pe=c["r_pe"], r_me=c["r_me"], tol=c["tol"],
                                          lattice0=lat0), sel=sel, want_d=False)
    _check_sampled(outs[1], o, sel)
