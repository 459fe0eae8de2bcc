"""Pins for the oracle's whole pair path: Poisson solve, E_xx, sigma_xx, D_xx.

* Gaussian densities have closed-form potentials erf(r/s)/r and Coulomb
  energies; the error must fall at the stencil's sixth order.
* E(lambda h) = E(h) / lambda exactly for the discrete method with frozen
  subdomains (Eqs. exx_drv_Sspace_key, dexxdL), hence sum sigma h = -E for the
  finite-difference derivative of E; the analytic sigma of Eq. sxx_working
  agrees with it to discretization error, shrinking at sixth order.
* Rotation invariance, i <-> j symmetry, and D_xx as the orbital gradient.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2011_07209_gb300.synth as synth

S2PI = math.sqrt(2.0) / math.sqrt(math.pi)


def _coulomb_gauss(cen, s, rows):
    E = 0.0
    for r in rows:
        i, j = int(r[0]), int(r[1])
        d2 = float(((cen[i] - cen[j]) ** 2).sum())
        w = 1.0 if i == j else 2.0
        E -= w * math.exp(-d2 / (2 * s * s)) * S2PI / s
    return E


def test_gaussian_potential_is_erf_over_r():
    L, n = 12.0, 48
    c = np.array([5.13, 6.21, 5.72])
    g = synth.gaussian_set(np.diag([L] * 3), (n,) * 3, [c], s=0.7)
    p = oracle.make_params(r_pe=5.0, r_me=6.5, tol=1e-12)
    rows = oracle.pair_list(g.lattice, g.n, g.centres, 8.0)
    out = oracle.pair_potential(g, 0, 0, rows[0][5:8], p)
    h = g.lattice.T
    rbar = (out["m"] / n) @ h.T
    centre_grid = h @ (rows[0][5:8] / n)
    delta = c - centre_grid
    r = np.linalg.norm(rbar - delta, axis=1)
    from scipy.special import erf
    exact = erf(r / 0.7) / r
    err = np.abs(out["v"] - exact) / exact
    assert err[: out["n_pe"]].max() < 2e-3
    assert err[out["n_pe"]:].max() < 1e-6          # far field of a spherical charge


def test_gaussian_energy_sixth_order():
    L = 12.0
    errs = []
    for n in (28, 42, 56):
        g = synth.gaussian_set(np.diag([L] * 3), (n,) * 3, [[5.1, 6.2, 5.7]], s=1.0)
        p = oracle.make_params(r_pe=5.0, r_me=6.5, tol=1e-12)
        r = oracle.exx(g, p, want_d=False)
        errs.append(abs(r["e_xx"] / (-S2PI / 1.0) - 1.0))
    order = math.log(errs[0] / errs[2]) / math.log(2.0)
    assert errs[2] < 2e-6
    assert 5.0 < order < 7.5, (order, errs)


@pytest.mark.parametrize("cell", ["cubic", "triclinic"])
def test_gaussian_set_closed_form_and_isotropic_stress(cell):
    if cell == "cubic":
        lat = np.diag([14.7] * 3)
        n = (48, 48, 48)
    else:
        lat = 14.7 * np.array([[1.0, 0, 0], [0.1, 1.0, 0], [0.05, -0.08, 1.0]])
        n = (56, 56, 56)
    cen = np.array([[3.0, 4.0, 5.0], [4.2, 4.5, 5.3], [9.0, 9.0, 9.0], [3.5, 4.9, 4.3]])
    g = synth.gaussian_set(lat, n, cen, s=0.7)
    r = oracle.exx(g, oracle.make_params(r_pe=6.0, r_me=8.0, tol=1e-11), want_d=False)
    E = _coulomb_gauss(cen, 0.7, r["pairs"])
    assert r["e_xx"] == pytest.approx(E, rel=2e-4)
    V = abs(np.linalg.det(lat))
    # every pair density is spherical about its midpoint, so Pi_xx = E/(3V) 1 in any cell
    # (Eq. liq_press in the simple cubic case)
    assert np.allclose(r["stress"], np.eye(3) * r["e_xx"] / (3 * V), atol=3e-3 * abs(E) / V)


def _small_water(n, seed=11):
    lat0 = 10.0 * np.array([[1.0, 0, 0], [0.1, 1.0, 0], [0.05, -0.08, 1.0]])
    ws = synth.water_cell(lat0, (n,) * 3, 1, seed)
    # derivatives of the discrete energy along one stencil family: aux directions frozen too
    p = oracle.make_params(r_pe=4.0, r_me=5.5, r_pair=6.0, tol=1e-12, lattice0=lat0, freeze_aux=True)
    return lat0, ws, p


def test_homogeneity_exact():
    lat0, ws, p = _small_water(32)
    E = oracle.exx(ws, p, want_d=False)["e_xx"]
    for lam in (0.98, 1.03):
        E2 = oracle.exx(synth.strained(ws, (lam - 1) * np.eye(3)), p, want_d=False)["e_xx"]
        assert E2 * lam == pytest.approx(E, rel=1e-11)


def _fd_sigma(ws, p, lat0, d=1e-4):
    h0 = lat0.T
    fd = np.zeros((3, 3))
    for a in range(3):
        for al in range(3):
            vals = []
            for sgn in (1, -1):
                h = h0.copy()
                h[a, al] += sgn * d
                eps = h @ np.linalg.inv(h0) - np.eye(3)
                vals.append(oracle.exx(synth.strained(ws, eps), p, want_d=False)["e_xx"])
            fd[a, al] = (vals[0] - vals[1]) / (2 * d)
    return fd


def test_stress_against_finite_differences_and_virial():
    errs = []
    for n in (32, 48):
        lat0, ws, p = _small_water(n)
        r = oracle.exx(ws, p, want_d=False)
        fd = _fd_sigma(ws, p, lat0)
        h0 = lat0.T
        # the derivative of the discrete energy obeys the virial identity exactly
        assert (fd * h0).sum() == pytest.approx(-r["e_xx"], rel=1e-8)
        # analytic sigma (Eq. sxx_working) vs derivative: discretization error only
        errs.append(np.abs(r["dedh"] - fd).max() / np.abs(fd).max())
        assert (r["dedh"] * h0).sum() == pytest.approx(-r["e_xx"], rel=3e-3)
        # Pi from sigma (Eq. pixx_working)
        V = np.linalg.det(h0)
        assert np.allclose(r["stress"], -(r["dedh"] @ h0.T) / V, atol=1e-15)
    assert errs[0] < 3e-3
    order = math.log(errs[0] / errs[1]) / math.log(48 / 32)
    assert order > 4.5, (order, errs)


def test_rotation_invariance():
    lat0, ws, p0 = _small_water(32)
    th = 0.7
    Q = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1.0]])
    Q = Q @ np.array([[1, 0, 0], [0, math.cos(0.3), -math.sin(0.3)], [0, math.sin(0.3), math.cos(0.3)]])
    p = oracle.make_params(r_pe=4.0, r_me=5.5, r_pair=6.0, tol=1e-12)
    r = oracle.exx(ws, p, want_d=False)
    ws2 = synth.MLWFSet(lattice=lat0 @ Q.T, n=ws.n, centres=ws.centres @ Q.T, a=ws.a, box=ws.box,
                        box_lo=ws.box_lo, phi=ws.phi, s=ws.s)
    r2 = oracle.exx(ws2, p, want_d=False)
    assert r2["e_xx"] == pytest.approx(r["e_xx"], rel=1e-10)
    assert np.allclose(r2["stress"], Q @ r["stress"] @ Q.T, atol=1e-10 * np.abs(r["stress"]).max())
    assert np.allclose(r2["dedh"], Q @ r["dedh"], atol=1e-10 * np.abs(r["dedh"]).max())


def test_pair_symmetry():
    ws = synth.make_config(1)
    p = oracle.make_params(tol=1e-11)
    sel = list(range(0, 119, 7))
    r = oracle.exx(ws, p, sel=sel, want_d=False)
    rev = synth.MLWFSet(lattice=ws.lattice, n=ws.n, centres=ws.centres[::-1].copy(), a=ws.a[::-1].copy(),
                        box=ws.box, box_lo=ws.box_lo[::-1].copy(), phi=ws.phi[::-1].copy(), s=ws.s)
    r2 = oracle.exx(rev, p, want_d=False)
    N = ws.n_orb
    idx = {(int(a[0]), int(a[1])): k for k, a in enumerate(r2["pairs"])}
    for k in sel:
        i, j = int(r["pairs"][k][0]), int(r["pairs"][k][1])
        k2 = idx[(N - 1 - j, N - 1 - i)]
        assert r2["pair_e"][k2] == pytest.approx(r["pair_e"][k], rel=1e-9)


def test_dxx_is_orbital_gradient_of_energy():
    """D^i = sum_j v_ij phi_j (Eq. Dxx) is, up to the factor 4 of a closed-shell
    real-orbital gradient (and up to the tiny asymmetry of the boundary terms), the
    derivative dE/dphi_i: dE = -4 dV <D^i, dphi_i>."""
    L, n = 10.0, 40
    ws = synth.water_cell(np.diag([L] * 3), (n,) * 3, 1, 3)
    p = oracle.make_params(r_pe=4.5, r_me=6.0, r_pair=6.0, tol=1e-12)
    r = oracle.exx(ws, p)
    i = 1
    rng = np.random.default_rng(0)
    u = [np.arange(b) for b in ws.box]
    grid = np.stack(np.meshgrid(*u, indexing="ij"), -1).astype(float)
    cen = np.array(ws.box) // 2
    bump = np.exp(-((grid - cen) ** 2).sum(-1) / (2 * 4.0 ** 2)) * np.cos(0.4 * (grid[..., 0] - cen[0]))
    t = 1e-4
    Es = []
    for sgn in (1, -1):
        phi = ws.phi.copy()
        phi[i] += sgn * t * bump
        w2 = synth.MLWFSet(lattice=ws.lattice, n=ws.n, centres=ws.centres, a=ws.a, box=ws.box,
                           box_lo=ws.box_lo, phi=phi, s=ws.s)
        Es.append(oracle.exx(w2, p, want_d=False)["e_xx"])
    dE = (Es[0] - Es[1]) / (2 * t)
    # D^i on its box; bring bump onto the D box by global index
    Nn = np.asarray(ws.n)
    gidx = (ws.box_lo[i] + grid.astype(int)) % Nn
    dl = (gidx - r["dbox_lo"][i]) % Nn
    inside = np.all(dl < r["dbox"], axis=-1)
    Dv = np.zeros(bump.shape)
    Dv[inside] = r["dxx"][i][tuple(dl[inside].T)]
    pred = -4.0 * ws.dv * float((Dv * bump).sum())
    assert pred == pytest.approx(dE, rel=1e-6)


def test_edge_cases():
    L = 10.0
    # no orbitals
    g = synth.gaussian_set(np.diag([L] * 3), (32,) * 3, np.zeros((0, 3)))
    r = oracle.exx(g, oracle.make_params(r_pe=4.0, r_me=5.5), want_d=False)
    assert r["e_xx"] == 0.0 and len(r["pairs"]) == 0
    # R_pair below every separation: self pairs only
    g = synth.gaussian_set(np.diag([L] * 3), (32,) * 3, [[1.0, 1.0, 1.0], [6.0, 6.0, 6.0]])
    r = oracle.exx(g, oracle.make_params(r_pair=0.5, r_pe=4.0, r_me=5.5), want_d=False)
    assert [tuple(x[:2]) for x in r["pairs"]] == [(0, 0), (1, 1)]
    # R_ME too small for the halo -> error 3
    with pytest.raises(oracle.OracleError) as e:
        oracle.exx(g, oracle.make_params(r_pe=4.0, r_me=4.2), want_d=False)
    assert e.value.code == 3
    # left-handed cell -> error 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.exx(synth.MLWFSet(lattice=np.diag([L, L, -L]), n=g.n, centres=g.centres, a=g.a, box=g.box,
                                 box_lo=g.box_lo, phi=g.phi), oracle.make_params(r_pe=4.0, r_me=5.5), want_d=False)
    assert e.value.code == 2
    # CG iteration cap -> error 5
    with pytest.raises(oracle.OracleError) as e:
        oracle.exx(g, oracle.make_params(r_pe=4.0, r_me=5.5, max_iter=3), want_d=False)
    assert e.value.code == 5


@pytest.mark.parametrize("cell", ["cubic", "triclinic"])
def test_cg_matches_dense_direct_solve(cell):
    """Step IV on a tiny subdomain: the oracle's CG potential equals the direct
    solution of the dense system A v = 4 pi rho + L_shell v_shell (Eq. pe with
    the Dirichlet data of Eq. me), where A = -L restricted to PE is assembled
    here from the stencil's directions, coefficients and weights (Eqs. d2_1,
    lapG_mod_nk3d).  The pair density is non-spherical (a != 0 orbitals, i != j),
    so moments with l > 0 feed the boundary values."""
    if cell == "cubic":
        lat = np.diag([7.0, 7.0, 7.0])
    else:
        lat = 7.0 * np.array([[1.0, 0, 0], [0.1, 1.0, 0], [0.05, -0.08, 1.0]])
    n = (35, 35, 35)
    ws = synth.water_cell(lat, n, 1, 11, r_phi=3.0)
    r_pe, r_me = 1.1, 2.4
    p = oracle.make_params(r_pair=4.0, r_pe=r_pe, r_me=r_me, tol=1e-13, lmax=6)
    rows = oracle.pair_list(ws.lattice, ws.n, ws.centres, 4.0)
    i, j, g = 0, 1, None
    for r in rows:
        if r[0] == i and r[1] == j:
            g = np.asarray(r[5:8])
    assert g is not None
    out = oracle.pair_potential(ws, i, j, g, p)
    npe, m = out["n_pe"], out["m"]
    assert 300 < npe < 1200
    nn = np.asarray(n)
    h = ws.lattice.T
    # pair density on PE from the orbital boxes
    def phi_at(k, pts):
        u = (pts - ws.box_lo[k]) % nn
        ok = np.all(u < ws.box, axis=1)
        v = np.zeros(len(pts))
        v[ok] = ws.phi[k][u[ok, 0], u[ok, 1], u[ok, 2]]
        return v
    pts = (g + m) % nn
    rho = (phi_at(i, pts) * phi_at(j, pts))[:npe]
    # the far field on the shell is the oracle's multipole expansion (pinned separately)
    rbar = (m / nn) @ h.T
    Q = oracle.multipoles(6, rbar[:npe], rho * ws.dv)
    assert np.abs(Q[1:]).max() > 1e-3 * abs(Q[0])       # l > 0 moments matter here
    v_sh = oracle.farfield(6, Q, rbar[npe:])
    assert np.allclose(out["v"][npe:], v_sh, rtol=1e-12, atol=0)
    # dense A = -L on PE, with the shell coupling moved to the right-hand side
    st = oracle.stencil_info(ws.lattice, n, 3)
    w2 = oracle.fd2_weights(3)
    index = {tuple(x): k for k, x in enumerate(m)}
    A = np.zeros((npe, npe))
    b = 4 * math.pi * rho.copy()
    for k in range(npe):
        for d, c in zip(st["dirs"], st["coef"]):
            for s in range(-3, 4):
                q = index[tuple(m[k] + s * np.asarray(d))]
                wgt = c * w2[abs(s)]
                if q < npe:
                    A[k, q] -= wgt
                else:
                    b[k] += wgt * out["v"][q]
    assert np.allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
    v = np.linalg.solve(A, b)
    assert np.abs(out["v"][:npe] - v).max() <= 1e-10 * np.abs(v).max()
    assert out["e_pair"] == pytest.approx(float(rho @ v) * ws.dv, rel=1e-10)
