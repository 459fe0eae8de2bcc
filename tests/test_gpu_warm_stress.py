"""GPU: warm-started CG along a frozen-offset trajectory, and the stress modes.

Warm start (the previous step's solution as the CG starting guess, Sec. III B 2)
changes only where CG starts: every result must match the cold start to the
CG tolerance, and the warm solves must take fewer iterations.  The stress
modes follow Sec. II C ("Isotropic Constraints"): p_int = Tr Pi / 3
(Eq. pxx_working) and, in a simple cubic cell, p_int = E_xx / (3V)
(Eq. liq_press).
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
    exx.lib()
    c = exx.Context(0)
    yield c
    c.close()


def _trajectory(n_steps=3):
    ws0 = synth.make_config(1)
    steps = synth.trajectory(ws0, n_steps, seed=synth.SEED_BASE + 50, strain_sigma=1e-3, centre_sigma=0.02)
    box = np.max([w.box for w in steps], axis=0)
    return ws0.lattice.copy(), [w.padded(box) for w in steps]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_warm_start_matches_cold_start_with_fewer_iterations(ctx, precision):
    from paper_2011_07209_gb300 import driver, exx
    lat0, steps = _trajectory(3)
    prec = exx.FP64 if precision == "fp64" else exx.MIXED
    # against a CG that starts from zero (no multipole guess)
    kw = dict(r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-10, precision=prec, frozen=True, guess=False)
    p_cold = exx.make_params(**kw)
    p_warm = exx.make_params(**kw, warm_start=True)
    n_orb, box, n = steps[0].n_orb, steps[0].box, steps[0].n
    plan_cold = exx.Plan(ctx, lat0, n, p_cold, n_orb, box)
    plan_warm = exx.Plan(ctx, lat0, n, p_warm, n_orb, box)
    for k, ws in enumerate(steps):
        cc = driver.prepare(ctx, ws, p_cold, plan=plan_cold)
        cw = driver.prepare(ctx, ws, p_warm, plan=plan_warm)
        c = driver.run(ctx, cc)
        w = driver.run(ctx, cw)
        assert c["status"] == 0 and w["status"] == 0
        assert np.array_equal(c["pairs"], w["pairs"])
        assert w["e_xx"] == pytest.approx(c["e_xx"], rel=1e-8)
        assert np.abs(w["stress"] - c["stress"]).max() < 1e-10
        assert np.abs(w["pair_e"] - c["pair_e"]).max() < 1e-8 * np.abs(c["pair_e"]).max()
        assert np.abs(cw.dxx.cpu().numpy() - cc.dxx.cpu().numpy()).max() < 1e-8
        if k == 0:
            assert w["n_warm"] == 0
            assert w["total_cg_iter"] == c["total_cg_iter"]
        else:
            assert w["n_warm"] >= 0.9 * w["n_pairs"]
            assert w["total_cg_iter"] < 0.95 * c["total_cg_iter"], (w["total_cg_iter"], c["total_cg_iter"])
    # the last step also against the oracle (frozen offsets of the first cell)
    ws = steps[-1]
    o = oracle.exx(ws, oracle.make_params(r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-10, lattice0=lat0), want_d=False)
    assert np.array_equal(w["pairs"], o["pairs"])
    assert w["e_xx"] == pytest.approx(o["e_xx"], rel=1e-7 if precision == "mixed" else 1e-9)
    assert np.abs(w["stress"] - o["stress"]).max() < 1e-8


def test_stress_modes_in_a_cubic_cell(ctx):
    from paper_2011_07209_gb300 import driver, exx
    ws = synth.make_config(1)
    out = {}
    for mode in (exx.STRESS_FULL, exx.STRESS_ISOTROPIC, exx.STRESS_CUBIC):
        p = exx.make_params(r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-10, precision=exx.FP64, stress_mode=mode)
        out[mode] = driver.run(ctx, driver.prepare(ctx, ws, p, want_d=False))
    full, iso, cub = out[exx.STRESS_FULL], out[exx.STRESS_ISOTROPIC], out[exx.STRESS_CUBIC]
    L = ws.lattice[0, 0]
    V = L ** 3
    E = full["e_xx"]
    assert iso["e_xx"] == pytest.approx(E, rel=1e-13) and cub["e_xx"] == pytest.approx(E, rel=1e-13)
    # Eq. pxx_working
    p_full = np.trace(full["stress"]) / 3.0
    assert full["p_int"] == pytest.approx(p_full, rel=1e-14)
    assert iso["p_int"] == pytest.approx(p_full, rel=1e-12)
    assert np.allclose(iso["stress"], iso["p_int"] * np.eye(3), rtol=0, atol=1e-18)
    assert np.allclose(iso["dedh"], full["dedh"], rtol=1e-10, atol=0)
    # Eq. liq_press and Eq. dexxdL: exact for the shortcut
    assert cub["p_int"] == pytest.approx(E / (3.0 * V), rel=1e-14)
    assert np.allclose(cub["stress"], cub["p_int"] * np.eye(3), rtol=0, atol=1e-18)
    assert np.trace(cub["dedh"]) == pytest.approx(-E / L, rel=1e-14)
    # the analytic sigma obeys E(lambda h) = E / lambda up to discretization error
    assert p_full == pytest.approx(E / (3.0 * V), rel=5e-3)
    # and p_int of the full path matches the oracle's Tr Pi / 3
    o = oracle.exx(ws, oracle.make_params(r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-10), want_d=False)
    assert full["p_int"] == pytest.approx(np.trace(o["stress"]) / 3.0, abs=1e-9)


def test_cubic_shortcut_rejects_other_cells(ctx):
    from paper_2011_07209_gb300 import driver, exx
    lat = 14.0 * np.array([[1.0, 0.0, 0.0], [0.1, 1.0, 0.0], [0.05, -0.08, 1.0]])
    ws = synth.water_cell(lat, (56, 56, 56), 2, 11)
    p = exx.make_params(r_pair=8.0, r_pe=5.0, r_me=6.5, tol=1e-8, precision=exx.MIXED, stress_mode=exx.STRESS_CUBIC)
    cr = driver.prepare(ctx, ws, p, want_d=False)
    with pytest.raises(exx.ExxError) as ei:
        driver.run(ctx, cr)
    assert ei.value.code == exx.ERR_ARG


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multipole_guess_same_results_fewer_iterations(ctx, precision):
    # the starting point is the free-space multipole potential of rho_ij: CG ends at the
    # same solution (same stopping rule) in fewer iterations
    from paper_2011_07209_gb300 import driver, exx
    ws = synth.make_config(1)
    prec = exx.FP64 if precision == "fp64" else exx.MIXED
    out = {}
    for g in (False, True):
        p = exx.make_params(r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-10, precision=prec, guess=g)
        cr = driver.prepare(ctx, ws, p)
        out[g] = driver.run(ctx, cr)
        out[g]["dxx"] = cr.dxx.cpu().numpy()
        out[g]["dbox"], out[g]["dbox_lo"] = cr.dbox, cr.dbox_lo_np
    a, b = out[True], out[False]
    assert a["status"] == 0 and b["status"] == 0
    assert a["e_xx"] == pytest.approx(b["e_xx"], rel=1e-8)
    assert np.abs(a["stress"] - b["stress"]).max() < 1e-10
    assert np.abs(a["dxx"] - b["dxx"]).max() < 1e-8
    assert a["total_cg_iter"] < 0.9 * b["total_cg_iter"], (a["total_cg_iter"], b["total_cg_iter"])
    o = oracle.exx(ws, oracle.make_params(r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-10), dbox=a["dbox"],
                   dbox_lo=a["dbox_lo"])
    assert a["e_xx"] == pytest.approx(o["e_xx"], rel=1e-7 if precision == "mixed" else 1e-9)
    assert np.abs(a["stress"] - o["stress"]).max() < 1e-8
    assert np.abs(a["dxx"] - o["dxx"]).max() < 1e-6


def test_warm_start_falls_back_to_multipole_guess_for_large_steps(ctx):
    # centres moved by 0.15 bohr: previous solutions start worse than the multipole
    # potential, so (guess on) most pairs start from the latter; results unchanged
    from paper_2011_07209_gb300 import driver, exx
    ws0 = synth.make_config(1)
    steps = synth.trajectory(ws0, 2, seed=synth.SEED_BASE + 52, strain_sigma=1e-3, centre_sigma=0.15)
    box = np.max([w.box for w in steps], axis=0)
    steps = [w.padded(box) for w in steps]
    kw = dict(r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-10, precision=exx.MIXED, frozen=True)
    plan_w = exx.Plan(ctx, ws0.lattice, ws0.n, exx.make_params(**kw, warm_start=True), ws0.n_orb, box)
    plan_g = exx.Plan(ctx, ws0.lattice, ws0.n, exx.make_params(**kw), ws0.n_orb, box)
    for k, ws in enumerate(steps):
        w = driver.run(ctx, driver.prepare(ctx, ws, exx.make_params(**kw, warm_start=True), plan=plan_w,
                                           want_d=False))
        g = driver.run(ctx, driver.prepare(ctx, ws, exx.make_params(**kw), plan=plan_g, want_d=False))
        assert w["status"] == 0 and g["status"] == 0
        assert w["e_xx"] == pytest.approx(g["e_xx"], rel=1e-8)
        if k == 1:
            assert w["n_warm"] < 0.5 * w["n_pairs"]
            assert w["total_cg_iter"] < 1.1 * g["total_cg_iter"]


def test_strain_triggered_reassembly(ctx):
    """Frozen proto-subdomains along a trajectory whose strain grows step by step
    (Sec. III B 2): once the Green-Lagrange strain against the plan's reference
    cell exceeds the threshold, the subdomains are re-assembled from the current
    cell (a new plan, no warm start carried over); the step after that matches
    the oracle with the new reference cell, and the steps before it the oracle
    with the old one."""
    from paper_2011_07209_gb300 import driver, exx
    ws0 = synth.make_config(1)
    eps = np.array([[3e-3, 1e-3, 0.0], [1e-3, -2e-3, 1e-3], [0.0, 1e-3, 2e-3]])   # per step
    steps, ws = [ws0], ws0
    for _ in range(3):
        ws = synth.strained(ws, eps)
        steps.append(ws)
    policy = exx.Reassembly(eps_max=6e-3)
    kw = dict(r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-10, precision=exx.MIXED, frozen=True, warm_start=True)
    p = exx.make_params(**kw)
    lat_ref, since = ws0.lattice.copy(), 0
    plan = exx.Plan(ctx, lat_ref, ws0.n, p, ws0.n_orb, ws0.box)
    reassembled_at = None
    for k, ws in enumerate(steps):
        if policy.due(lat_ref, ws.lattice, since):
            plan.close()
            lat_ref, since = ws.lattice.copy(), 0
            plan = exx.Plan(ctx, lat_ref, ws.n, p, ws.n_orb, ws.box)
            reassembled_at = k if reassembled_at is None else reassembled_at
        cr = driver.prepare(ctx, ws, p, plan=plan)
        g = driver.run(ctx, cr)
        assert g["status"] == 0
        if since == 0 and k > 0:
            assert g["n_warm"] == 0          # a fresh plan starts without previous solutions
        o = oracle.exx(ws, oracle.make_params(r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-10, lattice0=lat_ref),
                       dbox=cr.dbox, dbox_lo=cr.dbox_lo_np)
        assert np.array_equal(g["pairs"], o["pairs"])
        assert g["e_xx"] == pytest.approx(o["e_xx"], rel=1e-7)
        assert np.abs(g["stress"] - o["stress"]).max() < 1e-8
        assert np.abs(cr.dxx.cpu().numpy() - o["dxx"]).max() < 1e-6
        since += 1
    assert reassembled_at == 2                 # strain ~4e-3 after one step, ~8e-3 after two
