"""Pins for the oracle's solid harmonics, multipole expansion and pair list.

Harmonics: low-order closed forms, the addition theorem (which fixes every
normalization and the relative phase of each m), and orthonormality under a
product quadrature.  Multipoles: the far field (Eq. me) against a direct
Coulomb sum, with the truncation error falling as l_max grows.  Pair list:
brute force over all 27 images.
"""
import math

import numpy as np
import pytest

import oracle


def _legendre(l, x):
    p0, p1 = np.ones_like(x), x
    if l == 0:
        return p0
    for k in range(2, l + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    return p1


def test_low_order_closed_forms():
    rng = np.random.default_rng(0)
    xyz = rng.normal(size=(50, 3))
    S = oracle.solid_harmonics(2, xyz)
    x, y, z = xyz.T
    r2 = (xyz ** 2).sum(1)
    c1 = math.sqrt(3 / (4 * math.pi))
    assert np.allclose(S[:, 0], 1 / math.sqrt(4 * math.pi))
    assert np.allclose(S[:, 1], c1 * y)      # l=1, m=-1
    assert np.allclose(S[:, 2], c1 * z)      # l=1, m=0
    assert np.allclose(S[:, 3], c1 * x)      # l=1, m=+1
    assert np.allclose(S[:, 6], math.sqrt(5 / (16 * math.pi)) * (3 * z * z - r2))
    assert np.allclose(S[:, 8], math.sqrt(15 / (16 * math.pi)) * (x * x - y * y))
    assert np.allclose(S[:, 4], math.sqrt(15 / (4 * math.pi)) * x * y)


def test_addition_theorem_l_le_6():
    rng = np.random.default_rng(1)
    a = rng.normal(size=(40, 3))
    b = rng.normal(size=(40, 3))
    a /= np.linalg.norm(a, axis=1)[:, None]
    b /= np.linalg.norm(b, axis=1)[:, None]
    Sa = oracle.solid_harmonics(6, a)
    Sb = oracle.solid_harmonics(6, b)
    cg = (a * b).sum(1)
    for l in range(7):
        s = (Sa[:, l * l:(l + 1) ** 2] * Sb[:, l * l:(l + 1) ** 2]).sum(1)
        assert np.allclose(s, (2 * l + 1) / (4 * math.pi) * _legendre(l, cg), atol=1e-12), l


def test_orthonormal_on_sphere():
    xg, wg = np.polynomial.legendre.leggauss(16)
    nphi = 32
    ph = 2 * math.pi * np.arange(nphi) / nphi
    ct = np.repeat(xg, nphi)
    w = np.repeat(wg, nphi) * (2 * math.pi / nphi)
    st = np.sqrt(1 - ct ** 2)
    pp = np.tile(ph, xg.size)
    pts = np.stack([st * np.cos(pp), st * np.sin(pp), ct], axis=1)
    S = oracle.solid_harmonics(6, pts)
    G = (S * w[:, None]).T @ S
    assert np.allclose(G, np.eye(49), atol=1e-12)


def test_solid_harmonic_at_origin():
    S = oracle.solid_harmonics(6, np.zeros((1, 3)))
    assert S[0, 0] == pytest.approx(1 / math.sqrt(4 * math.pi))
    assert np.all(S[0, 1:] == 0.0)


def test_far_field_matches_direct_coulomb_sum():
    """Eqs. me and mepole: the truncated expansion converges to the direct sum
    like (a / r)^(l_max + 1) outside the charge cloud."""
    rng = np.random.default_rng(2)
    src = rng.normal(scale=0.6, size=(400, 3))
    q = rng.normal(size=400)
    q -= q.mean() * 0.5
    dirs = rng.normal(size=(60, 3))
    dirs /= np.linalg.norm(dirs, axis=1)[:, None]
    tgt = 6.0 * dirs
    direct = np.array([(q / np.linalg.norm(src - t, axis=1)).sum() for t in tgt])
    errs = []
    for lmax in range(0, 7):
        Q = oracle.multipoles(lmax, src, q)
        v = oracle.farfield(lmax, Q, tgt)
        errs.append(np.abs(v - direct).max())
    # textbook truncation bound of the multipole series of 1/|r - r'|
    a = np.linalg.norm(src, axis=1).max()
    r = 6.0
    for lmax in range(7):
        bound = np.abs(q).sum() * (a / r) ** (lmax + 1) / (r - a)
        assert errs[lmax] <= bound, (lmax, errs[lmax], bound)
    assert errs[6] < 1e-3 * np.abs(direct).max()
    assert all(errs[k + 2] < errs[k] for k in range(0, 5))


def _brute_pairs(lattice, n, centres, r_pair):
    h = np.asarray(lattice, float).T
    hinv = np.linalg.inv(h)
    out = {}
    N = len(centres)
    for i in range(N):
        for j in range(i, N):
            best = None
            s = hinv @ (centres[j] - centres[i])
            s -= np.round(s)
            for k in np.ndindex(5, 5, 5):
                kk = np.array(k) - 2
                d = h @ (s + kk)
                dd = float(d @ d)
                if best is None or dd < best[0]:
                    best = (dd, d)
            if best[0] <= r_pair * r_pair:
                out[(i, j)] = best
    return out


@pytest.mark.parametrize("cell", ["cubic", "triclinic"])
def test_pair_list_brute_force(cell):
    rng = np.random.default_rng(5)
    if cell == "cubic":
        lat = np.diag([14.7] * 3)
        n = (48, 48, 48)
    else:
        lat = 18.0 * np.array([[1.0, 0, 0], [0.1, 1.0, 0], [0.05, -0.08, 1.0]])
        n = (90, 90, 90)
    cen = (rng.random((60, 3)) * 1.2 - 0.1) @ lat   # some centres outside the cell
    rows = oracle.pair_list(lat, n, cen, 8.0)
    ref = _brute_pairs(lat, n, cen, 8.0)
    got = {(int(r[0]), int(r[1])): r for r in rows}
    assert set(got) == set(ref)
    h = lat.T
    hinv = np.linalg.inv(h)
    for (i, j), r in got.items():
        # the stored image reproduces the minimum-image distance
        s = hinv @ (cen[j] - cen[i])
        s = s - np.round(s) + r[2:5]
        assert float((h @ s) @ (h @ s)) == pytest.approx(ref[(i, j)][0], rel=1e-12, abs=1e-12)
        # g_ij is the grid point nearest (in fractional index) to the midpoint
        mid = hinv @ cen[i] + 0.5 * s
        g = np.asarray(r[5:8])
        dn = (np.asarray(n) * mid - g) / np.asarray(n)
        dn -= np.round(dn)
        assert np.all(np.abs(dn * np.asarray(n)) <= 0.5 + 1e-9)
        assert np.all((g >= 0) & (g < np.asarray(n)))
    # canonical order i <= j, lexicographic
    keys = [(int(r[0]), int(r[1])) for r in rows]
    assert keys == sorted(keys) and all(i <= j for i, j in keys)


def test_offsets_sets():
    lat = 29.6 * np.array([[1.0, 0, 0], [0.1, 1.0, 0], [0.05, -0.08, 1.0]])
    n = (75, 75, 75)
    npe, m = oracle.offsets(lat, n, 6.0, 8.0)
    h = lat.T
    r = (m / np.asarray(n)) @ h.T
    d = np.sqrt((r ** 2).sum(1))
    assert np.all(d[:npe] <= 6.0 + 1e-12)
    assert np.all((d[npe:] > 6.0 - 1e-12) & (d[npe:] <= 8.0 + 1e-12))
    # brute force count over a generous box
    H = 40
    ax = np.arange(-H, H + 1)
    mm = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    rr = (mm / np.asarray(n)) @ h.T
    dd = (rr ** 2).sum(1)
    assert npe == int((dd <= 36.0).sum())
    assert m.shape[0] == int((dd <= 64.0).sum())
    # lexicographic within each part
    for part in (m[:npe], m[npe:]):
        t = [tuple(x) for x in part]
        assert t == sorted(t)
    # volume: the PE count approaches the sphere volume over dV
    dv = np.linalg.det(h) / np.prod(n)
    assert npe * dv == pytest.approx(4 / 3 * math.pi * 6.0 ** 3, rel=0.02)


def test_pair_centre_rounds_half_away_from_zero():
    """Eq. l2g's NINT: a pair midpoint that lands exactly on a half grid index
    rounds away from zero (Fortran NINT), before the MOD.  In an 8 bohr cubic
    cell with 8 points every quantity below is exact in binary, so the three
    plausible rules separate: +2.5 -> 3 (round-half-even would give 2) and
    -2.5 -> -3 = 5 mod 8 (floor(x + 0.5) and half-even would give -2 = 6)."""
    lat = np.diag([8.0, 8.0, 8.0])
    n = (8, 8, 8)
    cases = [  # (C_i, C_j, expected g_ij)
        ([2.0, 0.0, 0.0], [3.0, 0.0, 0.0], [3, 0, 0]),     # N s_mid = (2.5, 0, 0)
        ([-3.0, 0.0, 0.0], [-2.0, 0.0, 0.0], [5, 0, 0]),   # N s_mid = (-2.5, 0, 0)
        ([0.0, 2.0, -3.0], [0.0, 3.0, -2.0], [0, 3, 5]),   # both signs on other axes
    ]
    for ci, cj, g in cases:
        rows = oracle.pair_list(lat, n, np.array([ci, cj]), 3.0)
        r = [list(x) for x in rows if x[0] == 0 and x[1] == 1]
        assert len(r) == 1
        assert r[0][2:5] == [0, 0, 0]
        assert r[0][5:8] == g, (ci, cj, r[0])
