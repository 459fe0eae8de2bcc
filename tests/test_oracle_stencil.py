"""Pins for the oracle's finite differences, cell metric and Natan-Kronik stencil.

Each test checks the oracle against something it does not compute itself:
the weights printed in the paper, exactness on polynomials (derived here with
exact fractions), the analytic Laplacian of Gaussians (convergence order),
the stencil sizes of Table 2, and the indefinite naive bisector choice the
paper reports for ice II.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_weights():
    out = {1: {}, 2: {}}
    for line in open(os.path.join(GOLD, "fd_weights_n3.txt")):
        if line.startswith("#") or not line.strip():
            continue
        d, q, num, den = (int(x) for x in line.split())
        out[d][q] = num / den
    return out


def test_printed_weights_n3():
    g = _golden_weights()
    w2 = oracle.fd2_weights(3)
    w1 = oracle.fd1_weights(3)
    for q in range(4):
        assert w2[q] == pytest.approx(g[2][q], rel=1e-15, abs=1e-15)
        assert w1[q] == pytest.approx(g[1][q], rel=1e-15, abs=1e-15)


def _exact_central_weights(n, order):
    """Solve the moment conditions of the (2n+1)-point central formula in fractions.

    order 2: sum_{q=-n..n} w_|q| q^k = 2 delta_{k,2} for k = 0, 2, ..., 2n;
    order 1: sum_{q=-n..n} sign(q) w_|q| q^k = delta_{k,1} for k = 1, 3, ..., 2n-1.
    """
    if order == 2:
        ks = list(range(0, 2 * n + 1, 2))
        cols = list(range(n + 1))
        A = [[(Fraction(1) if k == 0 else Fraction(0)) if q == 0 else 2 * Fraction(q) ** k for q in cols]
             for k in ks]
        rhs = [Fraction(2) if k == 2 else Fraction(0) for k in ks]
    else:
        ks = list(range(1, 2 * n, 2))
        cols = list(range(1, n + 1))
        A = [[2 * Fraction(q) ** k for q in cols] for k in ks]
        rhs = [Fraction(1) if k == 1 else Fraction(0) for k in ks]
    m = len(rhs)
    M = [A[r][:] + [rhs[r]] for r in range(m)]
    for c in range(m):
        p = next(r for r in range(c, m) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [x / piv for x in M[c]]
        for r in range(m):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    sol = {q: M[i][-1] for i, q in enumerate(cols)}
    if order == 1:
        sol[0] = Fraction(0)
    return sol


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_weights_are_exact_on_polynomials(n):
    w2 = oracle.fd2_weights(n)
    w1 = oracle.fd1_weights(n)
    e2 = _exact_central_weights(n, 2)
    e1 = _exact_central_weights(n, 1)
    for q in range(n + 1):
        assert w2[q] == pytest.approx(float(e2[q]), rel=1e-13, abs=1e-15)
        assert w1[q] == pytest.approx(float(e1[q]), rel=1e-13, abs=1e-15)


def test_metric_basic():
    lat = 29.6 * np.array([[1.0, 0.0, 0.0], [0.1, 1.0, 0.0], [0.05, -0.08, 1.0]])
    m = oracle.metric(lat, (150, 150, 150))
    h = lat.T
    assert np.allclose(m["h"], h)
    assert np.allclose(m["hinv"] @ h, np.eye(3), atol=1e-14)
    assert m["vol"] == pytest.approx(np.linalg.det(h), rel=1e-14)
    # grad_r = J grad_xi with xi_alpha = |L_alpha| s_alpha: check on a linear function
    L = np.linalg.norm(lat, axis=1)
    k = np.array([0.3, -1.2, 0.7])
    # f(r) = k.r; d f / d xi_alpha = k . L^_alpha
    dxi = lat @ k / L
    assert np.allclose(m["J"] @ dxi, k, atol=1e-14)
    assert np.allclose(m["F"], m["J"].T @ m["J"], atol=1e-14)


CELLS = {
    "cubic": (np.diag([14.7, 14.7, 14.7]), (48, 48, 48)),
    "ortho": (np.diag([26.8, 26.8, 28.0]), (134, 134, 140)),
    "monoclinic": (33.9 * np.array([[1.0, 0, 0], [0, 1.0, 0], [0.12, 0, 1.0]]), (169, 169, 171)),
    "triclinic": (29.6 * np.array([[1.0, 0, 0], [0.1, 1.0, 0], [0.05, -0.08, 1.0]]), (150, 150, 150)),
    "triclinic5": (37.3 * np.array([[1.0, 0, 0], [0.08, 1.0, 0], [0.04, 0.06, 1.0]]), (190, 190, 190)),
}


def _golden_counts():
    d = {}
    for line in open(os.path.join(GOLD, "nk_counts.txt")):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        d[parts[0]] = [int(x) for x in parts[1:]]
    return d


def test_stencil_counts_match_table2():
    g = _golden_counts()
    expect = {"cubic": "orthorhombic", "ortho": "orthorhombic", "monoclinic": "monoclinic",
              "triclinic": "triclinic", "triclinic5": "triclinic"}
    for name, (lat, n) in CELLS.items():
        st = oracle.stencil_info(lat, n)
        n_aux, n_pure, n_stcl = g[expect[name]]
        assert st["n_aux"] == n_aux, name
        assert st["dirs"].shape[0] == n_pure, name
        assert st["n_stcl"] == n_stcl, name


def test_first_shell_has_ten_non_axial_directions():
    g = _golden_counts()
    lat, n = CELLS["cubic"]
    nq = g["default_nq"][0]
    n1 = g["first_shell_non_axial"][0]
    m, ln = oracle.nk_candidates(lat, n, nq=nq)
    # N_q candidates, all non-axial and sorted by spacing; in a cubic grid every
    # second-shell point is longer than sqrt(3) spacings, so the first shell's
    # non-axial directions come first and the second shell fills the rest
    assert m.shape[0] == nq
    assert all(np.count_nonzero(r) >= 2 for r in m)
    assert np.all(np.diff(ln) >= 0)
    assert np.all(np.abs(m[:n1]).max(axis=1) == 1)
    assert np.all(np.abs(m[n1:]).max(axis=1) == 2)
    # one of +-m kept: first non-zero component positive
    assert all(r[np.nonzero(r)[0][0]] > 0 for r in m)


def _sample(lat, n, half, fn):
    """Sample fn on grid offsets |m| <= half around the origin (r = h m / N)."""
    h = np.asarray(lat, float).T
    ax = [np.arange(-half, half + 1)] * 3
    mm = np.stack(np.meshgrid(*ax, indexing="ij"), axis=-1).astype(float)
    r = (mm / np.asarray(n, float)) @ h.T
    return fn(r), r


@pytest.mark.parametrize("name", list(CELLS))
def test_laplacian_exact_on_degree7_polynomials(name):
    """L is exact on every polynomial of total degree <= 2n+1 = 7: each pure
    second difference is exact along its line, and the NK combination of pure
    derivatives reproduces the metric Laplacian (Eqs. lapG, lapG_mod_nk3d)."""
    lat, n = CELLS[name]
    rng = np.random.default_rng(3)
    terms = [(rng.normal(size=3), m, rng.normal()) for m in (2, 3, 4, 5, 6, 7) for _ in range(2)]
    scale = 0.4

    def f(r):
        out = np.zeros(r.shape[:-1])
        for k, m, c in terms:
            out += c * ((r @ k) * scale) ** m
        return out

    def lap_f(r):
        out = np.zeros(r.shape[:-1])
        for k, m, c in terms:
            out += c * m * (m - 1) * (k @ k) * scale ** 2 * ((r @ k) * scale) ** (m - 2)
        return out

    vals, r = _sample(lat, n, 8, f)
    lap = oracle.apply_lap(lat, n, vals)
    ok = np.isfinite(lap)
    assert ok.sum() > 100
    ref = lap_f(r)[ok]
    err = np.abs(lap[ok] - ref).max() / np.abs(ref).max()
    assert err < 1e-8, err


@pytest.mark.parametrize("name", ["cubic", "monoclinic", "triclinic"])
def test_laplacian_sixth_order_on_gaussian(name):
    lat, n0 = CELLS[name]
    errs = []
    hs = []
    sig = 0.9
    for k in (1.0, 1.5, 2.0):
        n = tuple(int(round(x * k * 0.5)) for x in n0)
        g = lambda r: np.exp(-(r * r).sum(-1) / (2 * sig * sig))
        vals, r = _sample(lat, n, int(round(12 * k)), g)
        lap = oracle.apply_lap(lat, n, vals)
        r2 = (r * r).sum(-1)
        ref = (r2 / sig ** 4 - 3 / sig ** 2) * np.exp(-r2 / (2 * sig * sig))
        ok = np.isfinite(lap) & (r2 < 2.0 ** 2)
        errs.append(np.abs(lap[ok] - ref[ok]).max())
        hs.append(1.0 / k)
    order = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert 5.3 < order < 7.0, (order, errs)


def _naive_bisectors(lat):
    aux = []
    for a, b in ((0, 1), (0, 2), (1, 2)):
        m = [0, 0, 0]
        m[a] = 1
        m[b] = -1 if np.dot(lat[a], lat[b]) > 0 else 1
        aux.append(m)
    return np.array(aux)


def _rhombohedral(angle_deg, a=10.0):
    t = math.radians(angle_deg)
    c = math.cos(t)
    a1 = [1.0, 0.0, 0.0]
    a2 = [c, math.sin(t), 0.0]
    cy = (c - c * c) / math.sin(t)
    a3 = [c, cy, math.sqrt(1 - c * c - cy * cy)]
    return a * np.array([a1, a2, a3])


def test_naive_bisector_indefinite_for_ice_II_like_cell():
    ang = None
    for line in open(os.path.join(GOLD, "paper_numbers.txt")):
        if line.startswith("rhombohedral_angle_deg"):
            ang = float(line.split()[1])
    lat = _rhombohedral(ang)
    n = (40, 40, 40)
    assert oracle.stencil_code(lat, n, aux=_naive_bisectors(lat)) == 4
    st = oracle.stencil_info(lat, n)
    assert st["n_aux"] == 3
    # Algorithm 1 uses the grid-resolved trigonal axis
    assert [1, 1, 1] in st["dirs"].tolist()


def test_two_d_rule_matches_eq_lapG_nk2d():
    """For one non-orthogonal pair the coefficients are those of Eq. lapG_nk2d."""
    lat, n = CELLS["monoclinic"]
    m = oracle.metric(lat, n)
    st = oracle.stencil_info(lat, n)
    F, dxi = m["F"], m["dxi"]
    al, be = 0, 2
    L = np.linalg.norm(lat, axis=1)
    cosab = np.dot(lat[al], lat[be]) / (L[al] * L[be])
    kappa = -(dxi[be] / dxi[al]) * np.sign(cosab)
    Lh = lat / L[:, None]
    d = np.linalg.norm(Lh[al] + kappa * Lh[be])
    c_al = F[al, al] - F[al, be] / kappa
    c_be = F[be, be] - kappa * F[al, be]
    c_aux = F[al, be] * d * d / kappa
    coef = st["coef"]
    assert coef[al] * dxi[al] ** 2 == pytest.approx(c_al, rel=1e-12)
    assert coef[be] * dxi[be] ** 2 == pytest.approx(c_be, rel=1e-12)
    # aux step length is dxi_alpha * d
    assert coef[3] * (dxi[al] * d) ** 2 == pytest.approx(c_aux, rel=1e-12)
    assert coef[1] * dxi[1] ** 2 == pytest.approx(F[1, 1], rel=1e-12)
