"""Seeded synthetic inputs: water-like sets of localized orbitals on boxed grids.

This module only *prepares inputs*.  It holds none of the exact-exchange
arithmetic (no pair list, no Poisson solve, no multipoles, no stress), so the
CPU oracle and the CUDA path can both be fed from it without sharing any of
the method's code.

Recipe (stand-in for the liquid-water / ice MLWF snapshots of the paper, which
come from converged Quantum ESPRESSO runs and are not available here):

* oxygen sites uniform in fractional coordinates, accepted by rejection when
  their minimum-image distance to every earlier site is >= ``min_sep`` bohr;
* four orbital centres per oxygen, ``d_oc`` bohr from it along the vertices of
  a regular tetrahedron under a uniformly random rotation (random unit
  quaternion);
* each orbital is ``exp(-|r-c|^2 / (2 s^2)) * (1 + a.(r-c))`` with
  ``a ~ N(0, a_sigma^2)`` per component, sampled on a periodic index box
  around its centre and normalized on the grid (sum phi^2 dV = 1); orbitals
  are not orthogonalized.

Conventions: ``lattice`` rows are the lattice vectors L_alpha (bohr), so the
cell tensor is ``h = lattice.T`` (columns are L_alpha); grid point ``g`` sits at
``r = h @ (g / n)``.  An orbital box is ``phi[i][b0][b1][b2]`` whose element
``(u, v, w)`` is the grid point ``(box_lo[i] + (u, v, w)) mod n``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BOHR_S = 0.7          # Gaussian width s of every orbital (bohr)
A_SIGMA = 0.3         # std of the linear-distortion vector a
D_OC = 0.6            # centre-to-oxygen distance (bohr)
MIN_SEP = 4.7         # minimum O-O separation (bohr)
R_PHI = 6.0           # radius of the orbital support box (bohr)
SEED_BASE = 7209


@dataclasses.dataclass
class MLWFSet:
    """One cell's orbitals in the boxed layout (all arrays numpy, C order)."""
    lattice: np.ndarray      # (3, 3) float64, rows = lattice vectors
    n: np.ndarray            # (3,) int32 grid points along L_alpha
    centres: np.ndarray      # (n_orb, 3) float64 Cartesian bohr
    a: np.ndarray            # (n_orb, 3) float64 distortion vectors
    box: np.ndarray          # (3,) int32 box extent
    box_lo: np.ndarray       # (n_orb, 3) int32 first grid index (wraps mod n)
    phi: np.ndarray          # (n_orb, b0, b1, b2) float64
    s: float = BOHR_S

    @property
    def n_orb(self) -> int:
        return int(self.centres.shape[0])

    def padded(self, box) -> "MLWFSet":
        """The same orbitals on larger boxes (zeros appended after each box's last point)."""
        box = np.asarray(box, np.int32)
        assert np.all(box >= self.box)
        phi = np.zeros((self.n_orb,) + tuple(int(b) for b in box))
        b0, b1, b2 = (int(b) for b in self.box)
        phi[:, :b0, :b1, :b2] = self.phi
        return MLWFSet(lattice=self.lattice, n=self.n, centres=self.centres, a=self.a, box=box,
                       box_lo=self.box_lo, phi=phi, s=self.s)

    def subset(self, k: int) -> "MLWFSet":
        """The first k orbitals of the cell (same grid and boxes)."""
        return MLWFSet(lattice=self.lattice, n=self.n, centres=self.centres[:k].copy(), a=self.a[:k].copy(),
                       box=self.box, box_lo=self.box_lo[:k].copy(), phi=self.phi[:k].copy(), s=self.s)

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))

    @property
    def dv(self) -> float:
        return self.volume / float(np.prod(self.n))


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a normalized Gaussian quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


_TETRA = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) / math.sqrt(3.0)


def oxygen_sites(lattice: np.ndarray, n_mol: int, rng: np.random.Generator,
                 min_sep: float = MIN_SEP, max_tries: int = 2_000_000) -> np.ndarray:
    """Random sequential addition of ``n_mol`` sites with minimum-image separation."""
    h = np.asarray(lattice, float).T
    frac = np.empty((0, 3))
    tries = 0
    while frac.shape[0] < n_mol:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place oxygen sites at this density")
        s = rng.random(3)
        if frac.shape[0]:
            ds = frac - s
            ds -= np.round(ds)
            # check the 27 neighbouring images to be safe in skewed cells
            best = np.full(ds.shape[0], np.inf)
            for k in np.ndindex(3, 3, 3):
                d = (ds + (np.array(k) - 1)) @ h.T
                best = np.minimum(best, np.einsum("ij,ij->i", d, d))
            if best.min() < min_sep * min_sep:
                continue
        frac = np.vstack([frac, s])
    return frac @ h.T


def box_halfwidth(lattice: np.ndarray, n, radius: float) -> np.ndarray:
    """Index half-widths of the box that covers a sphere of ``radius`` bohr."""
    h = np.asarray(lattice, float).T
    hinv = np.linalg.inv(h)
    n = np.asarray(n, int)
    return np.ceil(radius * n * np.linalg.norm(hinv, axis=1)).astype(np.int64)


def orbital_boxes(lattice: np.ndarray, n, centres: np.ndarray, radius: float):
    """Box extent and per-orbital first index for boxes centred on ``centres``."""
    n = np.asarray(n, np.int64)
    h = np.asarray(lattice, float).T
    hw = box_halfwidth(lattice, n, radius)
    box = np.minimum(2 * hw + 1, n)
    frac = np.asarray(centres, float) @ np.linalg.inv(h).T
    frac -= np.floor(frac)
    gc = np.floor(frac * n + 0.5).astype(np.int64)
    box_lo = gc - box // 2
    return box.astype(np.int32), box_lo.astype(np.int32)


def eval_orbitals(lattice: np.ndarray, n, centres: np.ndarray, a: np.ndarray,
                  s: float = BOHR_S, r_phi: float = R_PHI):
    """Sample every orbital on its box and normalize it on the grid."""
    lattice = np.asarray(lattice, float)
    n = np.asarray(n, np.int64)
    h = lattice.T
    box, box_lo = orbital_boxes(lattice, n, centres, r_phi)
    dv = abs(np.linalg.det(h)) / float(np.prod(n))
    u = [np.arange(int(b)) for b in box]
    loc = np.stack(np.meshgrid(*u, indexing="ij"), axis=-1).reshape(-1, 3).astype(float)
    r_loc = (loc / n) @ h.T                       # h @ (local / n), (P, 3)
    phi = np.empty((centres.shape[0],) + tuple(int(b) for b in box))
    inv2s2 = 1.0 / (2.0 * s * s)
    # centres wrapped into the cell: the box sits around the wrapped centre
    frac = np.asarray(centres, float) @ np.linalg.inv(h).T
    cw = (frac - np.floor(frac)) @ h.T
    for i in range(centres.shape[0]):
        shift = h @ (box_lo[i] / n) - cw[i]
        d = r_loc + shift
        d2 = np.einsum("ij,ij->i", d, d)
        f = np.exp(-d2 * inv2s2) * (1.0 + d @ a[i])
        f /= math.sqrt(float(np.dot(f, f)) * dv)
        phi[i] = f.reshape(phi.shape[1:])
    return box, box_lo, phi


def water_cell(lattice, n, n_mol: int, seed: int, *, s: float = BOHR_S,
               a_sigma: float = A_SIGMA, d_oc: float = D_OC, min_sep: float = MIN_SEP,
               r_phi: float = R_PHI, rng: np.random.Generator | None = None) -> MLWFSet:
    """Water-like orbital set: 4 orbitals per oxygen on a tetrahedron."""
    lattice = np.asarray(lattice, float)
    rng = _rng(seed) if rng is None else rng
    oxy = oxygen_sites(lattice, n_mol, rng, min_sep)
    cen = []
    for o in oxy:
        rot = _random_rotation(rng)
        cen.append(o + d_oc * (_TETRA @ rot.T))
    centres = np.vstack(cen) if cen else np.empty((0, 3))
    a = rng.normal(scale=a_sigma, size=centres.shape) if a_sigma > 0 else np.zeros_like(centres)
    box, box_lo, phi = eval_orbitals(lattice, n, centres, a, s, r_phi)
    return MLWFSet(lattice=lattice, n=np.asarray(n, np.int32), centres=centres, a=a,
                   box=box, box_lo=box_lo, phi=phi, s=s)


def gaussian_set(lattice, n, centres, *, s: float = BOHR_S, r_phi: float = R_PHI) -> MLWFSet:
    """Pure Gaussians (a = 0) at given centres: the closed-form test case."""
    lattice = np.asarray(lattice, float)
    centres = np.asarray(centres, float).reshape(-1, 3)
    a = np.zeros_like(centres)
    box, box_lo, phi = eval_orbitals(lattice, n, centres, a, s, r_phi)
    return MLWFSet(lattice=lattice, n=np.asarray(n, np.int32), centres=centres, a=a,
                   box=box, box_lo=box_lo, phi=phi, s=s)


def strained(ws: MLWFSet, eps: np.ndarray) -> MLWFSet:
    """Apply h <- (I + eps) h holding the orbitals fixed in crystal coordinates.

    Grid values are kept (same boxes, same indices) and rescaled by
    sqrt(V / V') so each orbital stays normalized; centres move affinely.
    """
    eps = np.asarray(eps, float)
    f = np.eye(3) + eps
    lat2 = (f @ ws.lattice.T).T
    scale = math.sqrt(abs(np.linalg.det(ws.lattice)) / abs(np.linalg.det(lat2)))
    return MLWFSet(lattice=lat2, n=ws.n.copy(), centres=ws.centres @ f.T, a=ws.a.copy(),
                   box=ws.box.copy(), box_lo=ws.box_lo.copy(), phi=ws.phi * scale, s=ws.s)


# --------------------------------------------------------------------------
# The five workloads (sizes of the paper's liquid-water / ice cases).
# --------------------------------------------------------------------------

def lattice_cubic(L: float) -> np.ndarray:
    return np.diag([L, L, L]).astype(float)


CONFIGS = {
    1: dict(name="water4_cubic14.7_n48", lattice=lattice_cubic(14.7), n=(48, 48, 48), n_mol=4,
            r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-10, precision="fp64"),
    2: dict(name="water64_cubic23.5_n120", lattice=lattice_cubic(23.5), n=(120, 120, 120), n_mol=64,
            r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-9, precision="mixed"),
    3: dict(name="water128_triclinic29.6_n150",
            lattice=29.6 * np.array([[1.0, 0.0, 0.0], [0.1, 1.0, 0.0], [0.05, -0.08, 1.0]]),
            n=(150, 150, 150), n_mol=128, r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-9, precision="mixed"),
    5: dict(name="water256_triclinic37.3_n190",
            lattice=37.3 * np.array([[1.0, 0.0, 0.0], [0.08, 1.0, 0.0], [0.04, 0.06, 1.0]]),
            n=(190, 190, 190), n_mol=256, r_pair=8.0, r_pe=6.0, r_me=8.0, tol=1e-9, precision="mixed"),
}

# Three uneven cells launched together (32 / 96 / 192 molecules); R_PE per cell
# is drawn from {5, 6, 7} with the config's seed.
BATCH_CELLS = [
    dict(name="water32_cubic18.6", lattice=lattice_cubic(18.6), n_mol=32),
    dict(name="water96_ortho26.8x26.8x28.0", lattice=np.diag([26.8, 26.8, 28.0]), n_mol=96),
    dict(name="water192_mono33.9_shear0.12",
         lattice=33.9 * np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.12, 0.0, 1.0]]), n_mol=192),
]


def grid_for_spacing(lattice: np.ndarray, spacing: float = 0.2) -> tuple:
    return tuple(int(round(float(np.linalg.norm(v)) / spacing)) for v in np.asarray(lattice, float))


def make_config(k: int) -> MLWFSet:
    c = CONFIGS[k]
    return water_cell(c["lattice"], c["n"], c["n_mol"], SEED_BASE + k)


def make_batch(k: int = 4):
    """Cells of the batched workload, each with its own R_PE from {5, 6, 7}."""
    rng = _rng(SEED_BASE + k)
    out = []
    for c in BATCH_CELLS:
        r_pe = float(rng.choice([5.0, 6.0, 7.0]))
        n = grid_for_spacing(c["lattice"], 0.2)
        ws = water_cell(c["lattice"], n, c["n_mol"], 0, rng=rng)
        out.append((c["name"], ws, r_pe))
    return out


def trajectory(ws0: MLWFSet, n_steps: int, seed: int, strain_sigma: float = 1e-3,
               centre_sigma: float = 0.05):
    """Cells of a short trajectory: per step a symmetric strain and centre jitter.

    Orbitals are re-sampled at every step from the moved centres in the new cell.
    """
    rng = _rng(seed)
    lat = ws0.lattice.copy()
    cen = ws0.centres.copy()
    steps = [ws0]
    for _ in range(n_steps - 1):
        e = rng.normal(scale=strain_sigma, size=(3, 3))
        e = 0.5 * (e + e.T)
        f = np.eye(3) + e
        lat = (f @ lat.T).T
        cen = cen @ f.T + rng.normal(scale=centre_sigma, size=cen.shape)
        box, box_lo, phi = eval_orbitals(lat, ws0.n, cen, ws0.a, ws0.s)
        steps.append(MLWFSet(lattice=lat.copy(), n=ws0.n.copy(), centres=cen.copy(), a=ws0.a.copy(),
                             box=box, box_lo=box_lo, phi=phi, s=ws0.s))
    return steps
