"""Cell strain for re-assembling frozen proto-subdomains (Sec. III B 2):
exx_cell_strain is host arithmetic, so it runs here without a GPU.  Pinned to
closed forms of the Green-Lagrange strain E = (F^T F - I)/2, F = h h0^-1."""
import math

import numpy as np
import pytest

from paper_2011_07209_gb300 import build, exx


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    exx.lib()


def _rot(axis, angle):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    k = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * k + (1 - math.cos(angle)) * k @ k


L0 = 14.0 * np.array([[1.0, 0.0, 0.0], [0.1, 1.0, 0.0], [0.05, -0.08, 1.0]])   # rows: lattice vectors


def _deform(lattice0, F):
    # h = F h0 with h = lattice^T, so lattice = lattice0 F^T
    return lattice0 @ F.T


def test_identity_and_rotation_carry_no_strain():
    eps, dvol = exx.cell_strain(L0, L0)                # F = h h0^-1 = I up to rounding
    assert eps < 1e-15 and dvol == 0.0
    eps, dvol = exx.cell_strain(L0, _deform(L0, _rot([1, 2, 3], 0.7)))
    assert eps < 1e-14 and abs(dvol) < 1e-14


def test_uniaxial_stretch():
    for e in (1e-3, 0.05, -0.08):
        F = np.diag([1.0, 1.0, 1.0 + e])
        eps, dvol = exx.cell_strain(L0, _deform(L0, F))
        assert eps == pytest.approx(abs(e + 0.5 * e * e), rel=1e-12)
        assert dvol == pytest.approx(e, rel=1e-12)


def test_simple_shear_closed_form():
    g = 0.2
    F = np.eye(3)
    F[0, 1] = g
    eps, dvol = exx.cell_strain(L0, _deform(L0, F))
    # E = [[0, g/2], [g/2, g^2/2]]: eigenvalues g^2/4 +- sqrt(g^4/16 + g^2/4)
    lam = g * g / 4 + math.sqrt(g ** 4 / 16 + g * g / 4)
    assert eps == pytest.approx(lam, rel=1e-12)
    assert abs(dvol) < 1e-14


def test_random_deformation_against_symmetric_eigensolver():
    rng = np.random.default_rng(7209)
    for _ in range(20):
        F = np.eye(3) + 0.15 * rng.standard_normal((3, 3))
        if np.linalg.det(F) <= 0.2:
            continue
        E = 0.5 * (F.T @ F - np.eye(3))
        eps, dvol = exx.cell_strain(L0, _deform(L0, F))
        assert eps == pytest.approx(np.abs(np.linalg.eigvalsh(E)).max(), rel=1e-10, abs=1e-14)
        assert dvol == pytest.approx(np.linalg.det(F) - 1.0, rel=1e-10, abs=1e-14)


def test_bad_cells_and_null_pointers():
    lib = exx.lib()
    flip = L0.copy()
    flip[0] *= -1.0                                   # left-handed
    with pytest.raises(exx.ExxError) as e:
        exx.cell_strain(L0, flip)
    assert e.value.code == exx.ERR_CELL
    with pytest.raises(exx.ExxError):
        exx.cell_strain(np.zeros((3, 3)), L0)         # singular reference
    assert lib.exx_cell_strain(None, None, None) == exx.ERR_ARG


def test_reassembly_policy():
    stretched = _deform(L0, np.diag([1.0, 1.0, 1.06]))
    p = exx.Reassembly(eps_max=0.05)
    assert not p.due(L0, _deform(L0, np.diag([1.0, 1.0, 1.04])), steps_since=10 ** 6)
    assert p.due(L0, stretched, steps_since=1)        # 0.06 + 0.0018 > 0.05
    q = exx.Reassembly(stride=1000)
    assert not q.due(L0, stretched, steps_since=999)
    assert q.due(L0, L0, steps_since=1000)
    with pytest.raises(ValueError):
        exx.Reassembly(eps_max=0.0)
    with pytest.raises(ValueError):
        exx.Reassembly(stride=-1)
