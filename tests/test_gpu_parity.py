"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (the target accuracy of the path):
  pair list            bit-exact (integers)
  E_xx                 1e-9 relative (FP64 path), 1e-7 relative (mixed path)
  D_xx                 1e-6 max-abs
  Pi_xx                1e-8 Ha/bohr^3 max-abs
Mixed-path errors are measured against the oracle run at the same CG
tolerance.
"""
import numpy as np
import pytest

import oracle
import paper_2011_07209_gb300.synth as synth

pytestmark = pytest.mark.gpu

E_TOL = {"fp64": 1e-9, "mixed": 1e-7}
# per pair, relative to the pair's own E: the oracle and the GPU both stop at
# |b - A v| <= tol |b| (tol 1e-10 here), which bounds each one's relative error in
# int rho v by sqrt(cond A) tol ~ 6e-9; the mixed path adds its FP32 moments
PAIR_TOL = {"fp64": 2e-8, "mixed": 1e-7}
D_TOL = 1e-6
PI_TOL = 1e-8


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


def _gpu(ctx, ws, r_pair, r_pe, r_me, tol, precision, frozen=False, lattice0=None, max_iter=20000):
    from paper_2011_07209_gb300 import driver, exx
    prec = exx.FP64 if precision == "fp64" else exx.MIXED
    p = exx.make_params(r_pair=r_pair, r_pe=r_pe, r_me=r_me, tol=tol, precision=prec, frozen=frozen,
                        max_iter=max_iter)
    if lattice0 is not None:
        plan = exx.Plan(ctx, lattice0, ws.n, p, ws.n_orb, ws.box)
        cr = driver.prepare(ctx, ws, p, plan=plan)
    else:
        cr = driver.prepare(ctx, ws, p)
    out = driver.run(ctx, cr)
    out["dxx"] = cr.dxx.cpu().numpy()
    out["dbox"] = cr.dbox
    out["dbox_lo"] = cr.dbox_lo_np
    out["info"] = cr.plan.info()
    return out


def _oracle(ws, r_pair, r_pe, r_me, tol, dbox, dbox_lo, sel=None, lattice0=None, freeze_aux=False):
    p = oracle.make_params(r_pair=r_pair, r_pe=r_pe, r_me=r_me, tol=tol, lattice0=lattice0, freeze_aux=freeze_aux)
    return oracle.exx(ws, p, sel=sel, dbox=dbox, dbox_lo=dbox_lo, want_d=sel is None)


def _compare(g, o, precision, per_pair=True):
    assert np.array_equal(g["pairs"], o["pairs"]), "pair list differs"
    assert g["n_aux"] == o["n_aux"] and g["n_stcl"] == o["n_stcl"]
    assert g["e_xx"] == pytest.approx(o["e_xx"], rel=E_TOL[precision])
    assert np.abs(g["stress"] - o["stress"]).max() < PI_TOL
    if per_pair:
        # every pair against its own value (not the cell's largest), so that a distant
        # pair with a tiny E_pair is held to the same relative bound
        rel = np.abs(g["pair_e"] - o["pair_e"]) / np.abs(o["pair_e"])
        assert rel.max() < PAIR_TOL[precision], rel.max()
    if o["dxx"] is not None:
        assert np.abs(g["dxx"] - o["dxx"]).max() < D_TOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config1_cubic_water(ctx, precision):
    ws = synth.make_config(1)
    g = _gpu(ctx, ws, 8.0, 6.0, 8.0, 1e-10, precision)
    o = _oracle(ws, 8.0, 6.0, 8.0, 1e-10, g["dbox"], g["dbox_lo"])
    _compare(g, o, precision)
    assert g["status"] == 0 and g["failed_pair"] == -1


def _small_triclinic(n_mol=4, scale=14.0, n=56, seed=3):
    lat = scale * np.array([[1.0, 0, 0], [0.1, 1.0, 0], [0.05, -0.08, 1.0]])
    return synth.water_cell(lat, (n, n, n), n_mol, seed)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_triclinic_nk3d(ctx, precision):
    ws = _small_triclinic()
    g = _gpu(ctx, ws, 7.0, 5.0, 6.5, 1e-10, precision)
    o = _oracle(ws, 7.0, 5.0, 6.5, 1e-10, g["dbox"], g["dbox_lo"])
    assert g["n_aux"] == 3 and g["n_stcl"] == 37
    _compare(g, o, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_monoclinic_nk2d_ragged(ctx, precision):
    lat = 13.0 * np.array([[1.0, 0, 0], [0, 1.0, 0], [0.12, 0, 1.0]])
    ws = synth.water_cell(lat, (45, 47, 46), 3, 9)     # ragged grid sizes
    g = _gpu(ctx, ws, 7.0, 5.0, 6.5, 1e-10, precision)
    o = _oracle(ws, 7.0, 5.0, 6.5, 1e-10, g["dbox"], g["dbox_lo"])
    assert g["n_aux"] == 1 and g["n_stcl"] == 25
    _compare(g, o, precision)


def test_frozen_strained_cell(ctx):
    lat0 = 14.0 * np.array([[1.0, 0, 0], [0.1, 1.0, 0], [0.05, -0.08, 1.0]])
    ws0 = synth.water_cell(lat0, (56, 56, 56), 3, 5)
    eps = np.array([[2e-3, 1e-3, 0], [1e-3, -1e-3, 5e-4], [0, 5e-4, 1e-3]])
    ws = synth.strained(ws0, eps)
    g = _gpu(ctx, ws, 7.0, 5.0, 6.5, 1e-10, "fp64", frozen=True, lattice0=lat0)
    o = _oracle(ws, 7.0, 5.0, 6.5, 1e-10, g["dbox"], g["dbox_lo"], lattice0=lat0)
    _compare(g, o, "fp64")


def test_frozen_aux_directions(ctx):
    # frozen = 2: the plan cell's aux directions are kept under strain as well
    lat0 = 14.0 * np.array([[1.0, 0, 0], [0.1, 1.0, 0], [0.05, -0.08, 1.0]])
    ws0 = synth.water_cell(lat0, (56, 56, 56), 3, 5)
    eps = np.array([[-1e-3, 5e-4, 2e-4], [5e-4, 2e-3, 0], [2e-4, 0, -5e-4]])
    ws = synth.strained(ws0, eps)
    g = _gpu(ctx, ws, 7.0, 5.0, 6.5, 1e-10, "mixed", frozen=2, lattice0=lat0)
    o = _oracle(ws, 7.0, 5.0, 6.5, 1e-10, g["dbox"], g["dbox_lo"], lattice0=lat0, freeze_aux=True)
    _compare(g, o, "mixed")


def test_frozen_cubic_plan_cell_under_strain(ctx):
    # a cubic plan cell has no aux directions; a strained step needs three, chosen
    # for that step (Algorithm 1 at every MD step) while the offsets stay frozen
    lat0 = np.diag([12.0] * 3)
    ws0 = synth.water_cell(lat0, (40, 40, 40), 2, 31)
    eps = np.array([[1e-3, 4e-4, -3e-4], [4e-4, -2e-3, 6e-4], [-3e-4, 6e-4, 5e-4]])
    ws = synth.strained(ws0, eps)
    g = _gpu(ctx, ws, 7.0, 5.0, 6.5, 1e-10, "fp64", frozen=True, lattice0=lat0)
    assert g["n_aux"] == 3
    o = _oracle(ws, 7.0, 5.0, 6.5, 1e-10, g["dbox"], g["dbox_lo"], lattice0=lat0)
    _compare(g, o, "fp64")


def test_batched_uneven_cells(ctx):
    from paper_2011_07209_gb300 import driver, exx
    cells = [
        (synth.water_cell(np.diag([12.0] * 3), (40, 40, 40), 2, 21), 5.0),
        (synth.water_cell(np.diag([12.5, 12.5, 13.0]), (42, 42, 44), 3, 22), 4.5),
        (synth.water_cell(13.0 * np.array([[1.0, 0, 0], [0, 1.0, 0], [0.12, 0, 1.0]]), (44, 44, 45), 3, 23), 5.5),
    ]
    runs = []
    for ws, rpe in cells:
        p = exx.make_params(r_pair=7.0, r_pe=rpe, r_me=rpe + 1.6, tol=1e-10, precision=exx.MIXED)
        runs.append(driver.prepare(ctx, ws, p))
    outs = driver.run_batch(ctx, runs)
    for (ws, rpe), cr, g in zip(cells, runs, outs):
        o = _oracle(ws, 7.0, rpe, rpe + 1.6, 1e-10, cr.dbox, cr.dbox_lo_np)
        assert g["n_pairs"] == len(o["pairs"])
        assert g["e_xx"] == pytest.approx(o["e_xx"], rel=E_TOL["mixed"])
        assert np.abs(g["stress"] - o["stress"]).max() < PI_TOL
        assert np.abs(cr.dxx.cpu().numpy() - o["dxx"]).max() < D_TOL
        assert np.array_equal(cr.plan.pair_list(), o["pairs"])


def test_host_memory_path_matches_device(ctx):
    from paper_2011_07209_gb300 import driver, exx
    ws = synth.make_config(1)
    p = exx.make_params(tol=1e-10, precision=exx.MIXED)
    cr = driver.prepare(ctx, ws, p)
    dev = driver.run(ctx, cr)
    host = driver.run_host(ctx, cr.plan, ws, p)
    assert host["e_xx"] == pytest.approx(dev["e_xx"], rel=1e-12)
    assert np.abs(host["dxx"] - cr.dxx.cpu().numpy()).max() < 1e-12


def test_edge_cases(ctx):
    from paper_2011_07209_gb300 import driver, exx
    L = 10.0
    # one orbital, self pair only
    g1 = synth.gaussian_set(np.diag([L] * 3), (32,) * 3, [[1.0, 1.0, 1.0]])
    out = _gpu(ctx, g1, 6.0, 4.0, 5.5, 1e-10, "fp64")
    o = _oracle(g1, 6.0, 4.0, 5.5, 1e-10, out["dbox"], out["dbox_lo"])
    assert out["n_pairs"] == 1
    assert out["e_xx"] == pytest.approx(o["e_xx"], rel=1e-9)
    # R_pair below every separation -> self pairs only
    g2 = synth.gaussian_set(np.diag([L] * 3), (32,) * 3, [[1.0, 1.0, 1.0], [6.0, 6.0, 6.0]])
    out = _gpu(ctx, g2, 0.5, 4.0, 5.5, 1e-10, "mixed")
    assert [tuple(x[:2]) for x in out["pairs"]] == [(0, 0), (1, 1)]
    # halo too small -> EXX_ERR_HALO at plan creation
    with pytest.raises(exx.ExxError) as e:
        exx.Plan(ctx, g2.lattice, g2.n, exx.make_params(r_pe=4.0, r_me=4.2), 2, g2.box)
    assert e.value.code == exx.ERR_HALO
    # left-handed cell
    with pytest.raises(exx.ExxError) as e:
        exx.Plan(ctx, np.diag([L, L, -L]), g2.n, exx.make_params(r_pe=4.0, r_me=5.5), 2, g2.box)
    assert e.value.code == exx.ERR_CELL
    # iteration cap -> EXX_ERR_CG_NOT_CONVERGED with the failing pair reported
    p = exx.make_params(r_pair=6.0, r_pe=4.0, r_me=5.5, tol=1e-10, precision=exx.FP64, max_iter=3)
    cr = driver.prepare(ctx, g2, p)
    out = driver.run(ctx, cr, check=False)
    assert out["status"] == exx.ERR_CG and out["failed_pair"] == 0
    # D box too small for a non-zero contribution -> EXX_ERR_BOX
    p = exx.make_params(r_pair=6.0, r_pe=4.0, r_me=5.5, tol=1e-10, precision=exx.MIXED)
    cr = driver.prepare(ctx, g2, p)
    small = exx.make_result(cr.dxx, [3, 3, 3], cr.dbox_lo, exx.MEM_DEVICE)
    code = exx.solve(ctx, cr.plan, g2.lattice, g2.n, cr.orbitals(), small, check=False)
    assert code == exx.ERR_BOX
    # no orbitals at all
    g0 = synth.gaussian_set(np.diag([L] * 3), (32,) * 3, np.zeros((0, 3)))
    pl = exx.Plan(ctx, g0.lattice, g0.n, exx.make_params(r_pe=4.0, r_me=5.5), 1, g0.box)
    orb = exx.make_orbitals(0, g0.box, None, None, None)
    res = exx.make_result()
    exx.solve(ctx, pl, g0.lattice, g0.n, orb, res)
    assert res.n_pairs == 0 and res.e_xx == 0.0


def test_plan_matches_oracle_geometry(ctx):
    from paper_2011_07209_gb300 import exx
    for k in (1, 2, 3, 5):
        c = synth.CONFIGS[k]
        p = exx.make_params(r_pe=c["r_pe"], r_me=c["r_me"])
        plan = exx.Plan(ctx, c["lattice"], c["n"], p, 1, (8, 8, 8))
        info = plan.info()
        st = oracle.stencil_info(c["lattice"], c["n"])
        npe, m = oracle.offsets(c["lattice"], c["n"], c["r_pe"], c["r_me"])
        assert info["n_pe_pair"] == npe and info["n_me_pair"] == m.shape[0]
        assert np.array_equal(info["dirs"], st["dirs"])
        assert np.allclose(info["coef"], st["coef"], rtol=1e-12)


@pytest.mark.parametrize("cell", ["cubic", "triclinic", "monoclinic"])
def test_multigrid_preconditioned_cg(ctx, cell):
    """The mixed path with and without the multigrid preconditioner: the same
    discrete solution (both against the oracle at the parity tolerances) from
    far fewer iterations."""
    from paper_2011_07209_gb300 import driver, exx
    if cell == "cubic":
        ws, rp = synth.make_config(1), (8.0, 6.0, 8.0)
    elif cell == "triclinic":
        ws, rp = _small_triclinic(), (7.0, 5.0, 6.5)
    else:
        lat = 13.0 * np.array([[1.0, 0, 0], [0, 1.0, 0], [0.12, 0, 1.0]])
        ws, rp = synth.water_cell(lat, (45, 47, 46), 3, 9), (7.0, 5.0, 6.5)
    outs = {}
    for pc in (exx.PRECOND_NONE, exx.PRECOND_MG):
        p = exx.make_params(r_pair=rp[0], r_pe=rp[1], r_me=rp[2], tol=1e-10, precision=exx.MIXED, precond=pc)
        cr = driver.prepare(ctx, ws, p)
        g = driver.run(ctx, cr)
        g["dxx"] = cr.dxx.cpu().numpy()
        outs[pc] = (g, cr)
    g_mg, cr = outs[exx.PRECOND_MG]
    g_cg, _ = outs[exx.PRECOND_NONE]
    o = _oracle(ws, *rp, 1e-10, cr.dbox, cr.dbox_lo_np)
    _compare(g_mg, o, "mixed")
    _compare(g_cg, o, "mixed")
    assert g_mg["status"] == 0
    assert g_mg["total_cg_iter"] < 0.25 * g_cg["total_cg_iter"], (g_mg["total_cg_iter"], g_cg["total_cg_iter"])
    assert g_mg["max_cg_iter"] <= 40


def test_sharded_solves_sum_to_the_whole(ctx):
    """exx_plan_set_shard on one GPU: the shards of 3 ranks, solved one after the
    other, hold every pair once (per-pair outputs of other ranks' pairs are
    zero), and their partial E_xx, Pi and D_xx add up to the unsharded solve."""
    from paper_2011_07209_gb300 import driver, exx
    ws = _small_triclinic()
    p = exx.make_params(r_pair=7.0, r_pe=5.0, r_me=6.5, tol=1e-10, precision=exx.MIXED)
    cr = driver.prepare(ctx, ws, p)
    whole = driver.run(ctx, cr)
    d_whole = cr.dxx.cpu().numpy()
    owner = exx.pair_partition(ws.lattice, ws.n, p, whole["pairs"], 3)
    e_sum, pi_sum, d_sum, seen = 0.0, 0.0, 0.0, np.zeros(whole["n_pairs"], int)
    for rank in range(3):
        crr = driver.prepare(ctx, ws, p)
        crr.plan.set_shard(rank, 3)
        part = driver.run(ctx, crr)
        assert part["n_pairs"] == whole["n_pairs"]
        mine = owner == rank
        assert np.all(part["pair_e"][~mine] == 0.0)
        assert np.allclose(part["pair_e"][mine], whole["pair_e"][mine], rtol=1e-7, atol=0)
        seen += mine
        e_sum += part["e_xx"]
        pi_sum = pi_sum + part["stress"]
        d_sum = d_sum + crr.dxx.cpu().numpy()
    assert np.all(seen == 1)
    assert e_sum == pytest.approx(whole["e_xx"], rel=1e-7)
    assert np.abs(pi_sum - whole["stress"]).max() < 1e-10
    assert np.abs(d_sum - d_whole).max() < 1e-8
