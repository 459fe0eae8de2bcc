"""Full-size parity against stored oracle results: every pair of every
benchmark cell, in the launch configuration the benchmark times.

The stored results (``tests/golden/oracle_<cell>.npz``) were written by
``tests/golden/make_oracle_golden.py``, which calls only the FP64 CPU oracle,
at CG tolerance 1e-13 (the discrete truth).  Checked here, per cell:

  * the pair list, bit for bit;
  * every pair's E_pair = int_PE rho v, relative to that pair's own value;
  * every pair's contribution to Pi (Ha/bohr^3, absolute);
  * the cell totals E_xx (relative) and Pi_xx (Ha/bohr^3, absolute);
  * D_xx elementwise on the whole D boxes of a few orbitals, against the oracle
    run on every pair that touches them (so those D^i are complete);
  * on the 64-molecule cell, the plain FP64 GPU path as well.

Bounds (tolerances of the workloads): E_xx 1e-7 relative (mixed) and 1e-9
(FP64); Pi_xx 1e-8 Ha/bohr^3; D_xx 1e-6 absolute.  Per pair, E within 1e-7
(mixed) or 1e-9 (FP64) of its own value: a stopping rule |b - A v| <= tol |b|
bounds the relative error of int rho v by sqrt(cond A) tol (about 6e-8 at
cond A ~ 3e3 and tol 1e-9) when the start is not zero, and the solves here
start from the multipole guess; the FP64 runs use tol 1e-11 so that this bound
sits below 1e-9.  A pair's contribution to Pi within 1e-10 Ha/bohr^3.

Set EXX_ACCURACY_REPORT to a directory to have the measured errors written
there as JSON (one file per cell and precision).
"""
import json
import os
import sys

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_oracle_golden as golden  # noqa: E402

pytestmark = pytest.mark.gpu

E_REL = {"mixed": 1e-7, "fp64": 1e-9}
PI_ABS = 1e-8
PI_PAIR_ABS = 1e-10
D_ABS = 1e-6


def load(stem):
    path = os.path.join(HERE, "golden", f"oracle_{stem}.npz")
    if not os.path.exists(path):
        pytest.skip(f"stored oracle results {os.path.basename(path)} not generated")
    return dict(np.load(path))


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_07209_gb300 import exx
    c = exx.Context(0)
    yield c
    c.close()


def pi_of(sig_pairs, rows, lattice):
    """Per-pair contribution to Pi = -(1/V) sigma h^T, sigma = -2 w pair_sig."""
    h = np.asarray(lattice, float).T
    vol = abs(np.linalg.det(h))
    w = np.where(rows[:, 0] == rows[:, 1], 1.0, 2.0)
    sig = -2.0 * w[:, None, None] * sig_pairs
    return -np.einsum("pab,cb->pac", sig, h) / vol


def d_orbitals(rows, k, seed):
    """k orbitals, the first of them the one with the most pairs."""
    cnt = np.bincount(np.concatenate([rows[:, 0], rows[:, 1]]).astype(np.int64))
    rng = np.random.default_rng(seed)
    pick = [int(np.argmax(cnt))] + [int(x) for x in rng.choice(len(cnt), size=k, replace=False)]
    return sorted(set(pick))[:k]


def check_cell(name, prec, g, ws, lattice, out, dxx_gpu, dbox, dbox_lo, p_oracle, d_orbs):
    rows = g["rows"].astype(np.int32)
    assert np.array_equal(out["pairs"], rows), f"{name}: pair list differs from the oracle's"
    assert out["status"] == 0 and out["failed_pair"] == -1
    n = len(rows)
    e_g, e_o = out["pair_e"][:n], g["pair_e"]
    rel = np.abs(e_g - e_o) / np.abs(e_o)
    pi_pair = np.abs(pi_of(out["pair_sig"][:n], rows, lattice) - pi_of(g["pair_sig"], rows, lattice))
    rel_exx = abs(out["e_xx"] / float(g["e_xx"]) - 1.0)
    d_pi = float(np.abs(out["stress"] - g["stress"]).max())
    rep = {"cell": name, "precision": prec, "pairs": int(n), "max_rel_err_e_pair": float(rel.max()),
           "median_rel_err_e_pair": float(np.median(rel)), "rel_err_e_xx": rel_exx,
           "max_abs_err_pi_pair": float(pi_pair.max()), "max_abs_err_pi": d_pi,
           "oracle_tol": float(g["tol"])}
    if d_orbs is not None:
        sel = np.nonzero(np.isin(rows[:, 0], d_orbs) | np.isin(rows[:, 1], d_orbs))[0].astype(np.int32)
        o = oracle.exx(ws, p_oracle, sel=sel, want_d=True, dbox=dbox, dbox_lo=dbox_lo)
        dd = max(float(np.abs(dxx_gpu[i] - o["dxx"][i]).max()) for i in d_orbs)
        rep["max_abs_err_dxx"] = dd
        rep["dxx_orbitals"] = [int(i) for i in d_orbs]
        rep["dxx_max_abs"] = max(float(np.abs(o["dxx"][i]).max()) for i in d_orbs)
    outdir = os.environ.get("EXX_ACCURACY_REPORT")
    if outdir:
        os.makedirs(outdir, exist_ok=True)
        with open(os.path.join(outdir, f"accuracy_{name}_{prec}.json"), "w") as f:
            json.dump(rep, f, indent=1)
    print(json.dumps(rep))
    assert rel.max() <= E_REL[prec], rep
    assert rel_exx <= E_REL[prec], rep
    if prec == "mixed":
        # tighter regression guard on the mixed path's measured error budget (about
        # 8e-9, a same-sign bias from its FP32 moment and far-field tables)
        assert rel_exx <= 1e-8, rep
    assert pi_pair.max() <= PI_PAIR_ABS, rep
    assert d_pi <= PI_ABS, rep
    if d_orbs is not None:
        assert rep["max_abs_err_dxx"] <= D_ABS, rep


def solve_one(ctx, ws, prec, r_pair, r_pe, r_me, lattice0=None, tol=None):
    from paper_2011_07209_gb300 import driver, exx
    p = exx.make_params(r_pair=r_pair, r_pe=r_pe, r_me=r_me, tol=tol, frozen=lattice0 is not None,
                        precision=exx.MIXED if prec == "mixed" else exx.FP64)
    plan = exx.Plan(ctx, ws.lattice if lattice0 is None else lattice0, ws.n, p, ws.n_orb, ws.box)
    cr = driver.prepare(ctx, ws, p, plan=plan)
    out = driver.run(ctx, cr)
    return cr, out


def tol_for(prec):
    return 1e-9 if prec == "mixed" else 1e-11


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_water64_every_pair(ctx, prec):
    g = load("water64")
    [(stem, ws, r_pair, r_pe, r_me, lat0)] = golden.cells("water64")
    assert golden.sha(ws.centres) == str(g["centres_sha256"])
    cr, out = solve_one(ctx, ws, prec, r_pair, r_pe, r_me, tol=tol_for(prec))
    d_orbs = d_orbitals(g["rows"], 4, 2)
    dxx = {i: cr.dxx[i].cpu().numpy() for i in d_orbs}
    p_o = oracle.make_params(r_pair=r_pair, r_pe=r_pe, r_me=r_me, tol=1e-11)
    check_cell(stem, prec, g, ws, ws.lattice, out, dxx, cr.dbox, cr.dbox_lo_np, p_o, d_orbs)


def test_triclinic128_every_pair(ctx):
    g = load("triclinic128")
    [(stem, ws, r_pair, r_pe, r_me, lat0)] = golden.cells("triclinic128")
    assert golden.sha(ws.centres) == str(g["centres_sha256"])
    cr, out = solve_one(ctx, ws, "mixed", r_pair, r_pe, r_me, tol=1e-9)
    assert out["n_stcl"] == int(g["n_stcl"]) == 37
    d_orbs = d_orbitals(g["rows"], 3, 3)
    dxx = {i: cr.dxx[i].cpu().numpy() for i in d_orbs}
    p_o = oracle.make_params(r_pair=r_pair, r_pe=r_pe, r_me=r_me, tol=1e-11)
    check_cell(stem, "mixed", g, ws, ws.lattice, out, dxx, cr.dbox, cr.dbox_lo_np, p_o, d_orbs)


def test_batch3_every_pair(ctx):
    """The three uneven cells in one persistent launch."""
    from paper_2011_07209_gb300 import driver, exx
    cells = golden.cells("batch3")
    gs = [load(stem) for stem, *_ in cells]
    runs = []
    for stem, ws, r_pair, r_pe, r_me, lat0 in cells:
        p = exx.make_params(r_pair=r_pair, r_pe=r_pe, r_me=r_me, tol=1e-9, precision=exx.MIXED)
        runs.append(driver.prepare(ctx, ws, p))
    outs = driver.run_batch(ctx, runs, pair_outputs=True)
    for ci, ((stem, ws, r_pair, r_pe, r_me, lat0), g, cr, o) in enumerate(zip(cells, gs, runs, outs)):
        assert golden.sha(ws.centres) == str(g["centres_sha256"])
        n = o["n_pairs"]
        o = dict(o, pairs=cr.plan.pair_list(), pair_e=cr.pair_e[:n].cpu().numpy(),
                 pair_sig=cr.pair_sig[:n].cpu().numpy())
        d_orbs = d_orbitals(g["rows"], 2, 10 + ci)
        dxx = {i: cr.dxx[i].cpu().numpy() for i in d_orbs}
        p_o = oracle.make_params(r_pair=r_pair, r_pe=r_pe, r_me=r_me, tol=1e-11)
        check_cell(stem, "mixed", g, ws, ws.lattice, o, dxx, cr.dbox, cr.dbox_lo_np, p_o, d_orbs)


@pytest.mark.parametrize("step", [0, 1])
def test_trajectory256_every_pair(ctx, step):
    """MD steps 0 and 1 of the 1024-orbital triclinic trajectory, frozen offsets
    of step 0 (Sec. III B 2)."""
    name = f"traj256_s{step}"
    g = load(name)
    [(stem, ws, r_pair, r_pe, r_me, lat0)] = golden.cells(name)
    assert golden.sha(ws.centres) == str(g["centres_sha256"])
    lattice0 = np.asarray(g["lattice0"])
    cr, out = solve_one(ctx, ws, "mixed", r_pair, r_pe, r_me, lattice0=lattice0, tol=1e-9)
    d_orbs = d_orbitals(g["rows"], 2, 20 + step)
    dxx = {i: cr.dxx[i].cpu().numpy() for i in d_orbs}
    p_o = oracle.make_params(r_pair=r_pair, r_pe=r_pe, r_me=r_me, tol=1e-11, lattice0=lattice0)
    check_cell(stem, "mixed", g, ws, ws.lattice, out, dxx, cr.dbox, cr.dbox_lo_np, p_o, d_orbs)
