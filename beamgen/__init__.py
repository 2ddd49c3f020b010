"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module only *draws* inputs: particle phase-space coordinates, particle ids,
reference-particle presets and lattice element lists.  It holds none of the
tracking arithmetic (maps, deposition, field solve, kicks); both the oracle and
the CUDA path receive the same bytes from here.

Random numbers come from numpy's Philox4x32-10 counter-based bit generator
(Salmon et al., SC'11) keyed by the seed, so every array is reproducible on any
host.

Phase-space coordinates follow the ImpactX convention used throughout the
package (paper §ImpactX, Listing 1): x, y [m]; px, py = transverse momentum over
the reference momentum; t = c * (arrival-time lag) [m]; pt = -(energy deviation)
/ (reference momentum * c).  Arrays are returned as a (6, n) float64 C-contiguous
block in the order (x, px, y, py, t, pt), plus int64 ids 0..n-1.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np

# element type codes (shared with the C-ABI header's BX_DRIFT / BX_QUAD / BX_SBEND /
# BX_DIPEDGE / BX_CONSTF / BX_MULTIPOLE)
DRIFT, QUAD, SBEND, DIPEDGE, CONSTF, MULTIPOLE = 0, 1, 2, 3, 4, 5

# rest energies, CODATA 2018 [MeV]
MASS_PROTON_MEV = 938.27208816
MASS_ELECTRON_MEV = 0.51099895000


@dataclass(frozen=True)
class Element:
    """One lattice element: type code, length [m], focusing strength k [1/m^2]
    (quadrupole only; k > 0 focuses x), total bend angle [rad] (sector bend only)
    and the number of slices (space-charge kicks) through it."""
    kind: int
    length: float
    k: float = 0.0
    angle: float = 0.0
    nslice: int = 1
    k2: float = 0.0
    order: int = 0


def drift(length, nslice=1):
    return Element(DRIFT, float(length), 0.0, 0.0, int(nslice))


def quad(length, k, nslice=1):
    return Element(QUAD, float(length), float(k), 0.0, int(nslice))


def sbend(length, angle, nslice=1):
    return Element(SBEND, float(length), 0.0, float(angle), int(nslice))


def dipedge(psi, curvature):
    """Thin dipole edge: edge angle psi [rad], bend curvature 1/rho [1/m]."""
    return Element(DIPEDGE, 0.0, float(curvature), float(psi), 0)


def constf(length, kx, ky, nslice=1):
    """Constant transverse focusing channel piece (k_x, k_y in 1/m^2)."""
    return Element(CONSTF, float(length), float(kx), 0.0, int(nslice), float(ky))


def multipole(order, kn, ks=0.0):
    """Thin multipole of order m (1 dipole, 2 quadrupole, 3 sextupole, ...):
    integrated normal and skew strengths kn, ks [1/m^(m-1)] (k holds kn, k2
    holds ks)."""
    return Element(MULTIPOLE, 0.0, float(kn), 0.0, 0, float(ks), int(order))


def fodo_cell(nslice, kf=1.0, kd=-1.0):
    """The FODO cell of the paper's Listing 1: drift 0.25 m, QF (1 m, k=kf),
    drift 0.5 m, QD (1 m, k=kd), drift 0.25 m."""
    return [drift(0.25, nslice), quad(1.0, kf, nslice), drift(0.5, nslice),
            quad(1.0, kd, nslice), drift(0.25, nslice)]


def fodo_lattice(periods, nslice, kf=1.0, kd=-1.0):
    return fodo_cell(nslice, kf, kd) * int(periods)


def fodo8_lattice(ks, periods=5, nslice=2):
    """Super-period of four Listing-1 FODO cells whose eight quadrupoles each
    have their own strength, ks = (QF1, QD1, QF2, QD2, QF3, QD3, QF4, QD4),
    repeated `periods` times (5 periods = 20 cells)."""
    ks = [float(v) for v in ks]
    if len(ks) != 8:
        raise ValueError("eight quadrupole strengths")
    sp = []
    for c in range(4):
        sp += fodo_cell(nslice, ks[2 * c], ks[2 * c + 1])
    return sp * int(periods)


def fodo8_families(lattice: Sequence[Element]) -> np.ndarray:
    """Index (0..7) of the quadrupole strength of each element of a
    fodo8_lattice, -1 for drifts."""
    fam = np.full(len(lattice), -1, dtype=np.int64)
    for i, e in enumerate(lattice):
        if e.kind == QUAD:
            cell, pos = (i % 20) // 5, i % 5
            fam[i] = 2 * cell + (0 if pos == 1 else 1)
    return fam


KS_FODO8 = (1.0, -1.0, 1.0, -1.0, 1.0, -1.0, 1.0, -1.0)
# Matched Courant-Snyder parameters of the Listing-1 FODO cell at its start
# (phase advance 67.8 deg, beta 2.8216 m, alpha -+1.5905), eps for ~1 mm rms,
# then sigma_t, sigma_pt: (alpha_x, beta_x, eps_x, alpha_y, beta_y, eps_y, st, spt).
TWISS_FODO = (-1.5905004, 2.8216194, 3.5e-7, 1.5905004, 2.8216194, 3.5e-7, 1e-3, 1e-4)


def standard_normal6(n: int, seed: int = 0) -> np.ndarray:
    """(6, n) independent standard normal draws (the xi of a Twiss bunch)."""
    return np.ascontiguousarray(_rng(seed).standard_normal((6, int(n))))


def chicane_rect_lattice(nslice=50):
    """chicane_lattice with rectangular bends: a thin edge of half the bend
    angle on both faces of every sector bend."""
    out = []
    for e in chicane_lattice(nslice):
        if e.kind == SBEND:
            h = e.angle / e.length
            out += [dipedge(0.5 * e.angle, h), e, dipedge(0.5 * e.angle, h)]
        else:
            out.append(e)
    return out


def fodo_multipole_lattice(nslice=2, periods=1):
    """FODO cells of Listing 1 with thin nonlinear multipoles between the
    elements (the paper lists a chain of thin multipoles among its examples;
    orders and strengths here are a reading, sized so that no multipole kicks
    a particle at 2 cm by more than ~1e-3, which keeps a bunch of 1 mm rms
    bounded over many cells):
    a skew quadrupole at the start, normal sextupoles at both faces of QF, an
    octupole and a decapole together at the cell centre, a skew-normal
    sextupole after QD and a skew dodecapole at the end."""
    out = []
    for _ in range(int(periods)):
        out += [multipole(2, 0.0, 0.01),
                drift(0.25, nslice), multipole(3, 2.0), quad(1.0, 1.0, nslice),
                multipole(3, 2.0), drift(0.5, nslice),
                multipole(4, -600.0, 100.0), multipole(5, 1e5),
                quad(1.0, -1.0, nslice), multipole(3, -1.5, 0.8),
                drift(0.25, nslice), multipole(6, 0.0, 2e7)]
    return out


# Listing 1 (FODO.py): Waterbag parameters (sigmaX, sigmaY, sigmaT, sigmaPx,
# sigmaPy, sigmaPt, muxpx, muypy, mutpt) of the rms-matched 2 GeV electron beam
# with 2 nm unnormalised emittance, 1e4 particles, 1 nC, 25 slices per element.
LISTING1_WATERBAG = (3.9984884770e-5, 3.9984884770e-5, 1.0e-3, 2.6623538760e-5,
                     2.6623538760e-5, 2.0e-3, -0.846574929020762, 0.846574929020762, 0.0)


def uniform01(n: int, seed: int = 0) -> np.ndarray:
    """n uniform draws in [0, 1) (the radii of a Waterbag bunch)."""
    return _rng(seed + 7919).random(int(n))


def chicane_lattice(nslice=50):
    """Four sector bends (L=0.5 m, +-0.1 rad) separated by 1 m drifts, preceded
    by two matching quadrupoles (L=0.5 m, k=+-0.5 /m^2)."""
    return [quad(0.5, 0.5, nslice), quad(0.5, -0.5, nslice),
            sbend(0.5, 0.1, nslice), drift(1.0, nslice),
            sbend(0.5, -0.1, nslice), drift(1.0, nslice),
            sbend(0.5, -0.1, nslice), drift(1.0, nslice),
            sbend(0.5, 0.1, nslice), drift(1.0, nslice)]


def count_kicks(lattice: Sequence[Element]) -> int:
    return int(sum(e.nslice for e in lattice))


def lattice_array(lattice: Sequence[Element]) -> np.ndarray:
    """Lattice as a (m, 5) float64 table: kind, length, k, angle, nslice."""
    return np.array([[e.kind, e.length, e.k, e.angle, e.nslice] for e in lattice],
                    dtype=np.float64).reshape(-1, 5)


@dataclass(frozen=True)
class Species:
    """Reference particle: rest energy and kinetic energy [MeV], charge sign."""
    mass_MeV: float
    kinetic_MeV: float
    charge_sign: float


PROTON_2GEV = Species(MASS_PROTON_MEV, 2000.0, +1.0)
PROTON_1GEV = Species(MASS_PROTON_MEV, 1000.0, +1.0)
ELECTRON_500MEV = Species(MASS_ELECTRON_MEV, 500.0, -1.0)
ELECTRON_2GEV = Species(MASS_ELECTRON_MEV, 2000.0, -1.0)

SIGMAS_DEFAULT = (1e-3, 1e-4, 1e-3, 1e-4, 1e-3, 1e-4)  # x, px, y, py, t, pt


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def gaussian6d(n: int, sigmas=SIGMAS_DEFAULT, seed: int = 0) -> np.ndarray:
    """Uncorrelated 6D Gaussian bunch, zero mean, given rms per coordinate."""
    g = _rng(seed).standard_normal((6, int(n)))
    return np.ascontiguousarray(g * np.asarray(sigmas, dtype=np.float64)[:, None])


def gaussian_with_halo(n: int, sigmas=SIGMAS_DEFAULT, halo_fraction=0.2,
                       halo_semi_axes_in_sigma=3.0, seed: int = 0) -> np.ndarray:
    """Gaussian core plus a halo whose positions (x, y, t) are uniform in the
    ellipsoid with semi-axes `halo_semi_axes_in_sigma` * sigma and whose momenta
    are Gaussian.  The last round(halo_fraction * n) particles are the halo."""
    n = int(n)
    nh = int(round(halo_fraction * n))
    rng = _rng(seed)
    out = rng.standard_normal((6, n)) * np.asarray(sigmas, dtype=np.float64)[:, None]
    if nh > 0:
        d = rng.standard_normal((3, nh))
        d /= np.sqrt((d * d).sum(axis=0))
        r = rng.random(nh) ** (1.0 / 3.0)
        for row, ax in zip((0, 2, 4), range(3)):
            out[row, n - nh:] = halo_semi_axes_in_sigma * sigmas[row] * r * d[ax]
    return np.ascontiguousarray(out)


def uniform_lattice_points(n_side: int, semi_axes=(1e-3, 1e-3, 1e-3)):
    """Deterministic points of a cubic lattice clipped to the ellipsoid with the
    given semi-axes (x, y, t); momenta zero.  Used for closed-form field checks."""
    s = (np.arange(n_side) + 0.5) / n_side * 2.0 - 1.0
    gx, gy, gz = np.meshgrid(s, s, s, indexing="ij")
    m = gx * gx + gy * gy + gz * gz <= 1.0
    out = np.zeros((6, int(m.sum())))
    out[0] = gx[m] * semi_axes[0]
    out[2] = gy[m] * semi_axes[1]
    out[4] = gz[m] * semi_axes[2]
    return out


def ids(n: int) -> np.ndarray:
    return np.arange(int(n), dtype=np.int64)


@dataclass
class Workload:
    """A named tracking workload: bunch, reference particle, lattice, grid."""
    name: str
    n_particles: int
    species: Species
    bunch_charge_C: float
    lattice: List[Element]
    n_grid: int
    seed: int = 0
    halo: bool = False
    sigmas: tuple = field(default=SIGMAS_DEFAULT)

    @property
    def kicks(self) -> int:
        return count_kicks(self.lattice)

    def particles(self, n: int | None = None) -> np.ndarray:
        n = self.n_particles if n is None else int(n)
        if self.halo:
            return gaussian_with_halo(n, self.sigmas, seed=self.seed)
        return gaussian6d(n, self.sigmas, seed=self.seed)


@dataclass(frozen=True)
class Variant:
    """One problem of a batch: bunch size and seed, grid, FODO strengths."""
    n_particles: int
    n_grid: int
    kf: float
    kd: float
    seed: int

    def lattice(self, periods=10, nslice=4):
        return fodo_lattice(periods, nslice, self.kf, self.kd)

    def particles(self) -> np.ndarray:
        return gaussian6d(self.n_particles, seed=self.seed)


def batch_variants(count: int = 256, seed: int = 0, n_min: float = 1e4, n_max: float = 5e5,
                   spread: float = 0.2, grids=(32, 64)) -> List[Variant]:
    """Lattice variants of the Listing-1 FODO: k_QF, k_QD drawn uniformly within
    +-spread of +1 and -1 (per quadrupole family), particle counts
    floor(10^U(log10 n_min, log10 n_max)), grid 32^3 or 64^3 with equal odds,
    bunch seeds 1000 + index."""
    g = _rng(seed)
    out = []
    lo, hi = np.log10(n_min), np.log10(n_max)
    for i in range(int(count)):
        u = g.random(4)
        n = int(np.floor(10.0 ** (lo + (hi - lo) * u[0])))
        grid = grids[0] if u[1] < 0.5 else grids[1]
        kf = 1.0 * (1.0 + spread * (2.0 * u[2] - 1.0))
        kd = -1.0 * (1.0 + spread * (2.0 * u[3] - 1.0))
        out.append(Variant(n, grid, kf, kd, 1000 + i))
    return out


def workload(name: str) -> Workload:
    """The three tracking workloads:

    fodo_1e4_32  : 1e4 particles, 2 GeV p, FODO x10, 5 kicks/element (250), 32^3, 1 nC
    fodo_1e6_64  : 1e6 particles (20% halo), 1 GeV p, FODO x50, 4 kicks/element
                   (1000), 64^3, 10 nC
    chicane_25e6_128 : 2.5e7 particles, 500 MeV e-, quads + 4-bend chicane,
                   50 kicks/element (500), 128^3
    fodo8_grad_1e6_64 : 1e6 particles (Twiss bunch), 1 GeV p, 8-strength FODO
                   super-period x5 (20 cells), 2 kicks/element (200), 64^3, 10 nC
    """
    if name == "fodo_1e4_32":
        return Workload(name, 10_000, PROTON_2GEV, 1e-9, fodo_lattice(10, 5), 32)
    if name == "fodo_1e6_64":
        return Workload(name, 1_000_000, PROTON_1GEV, 10e-9, fodo_lattice(50, 4), 64,
                        halo=True)
    if name == "chicane_25e6_128":
        return Workload(name, 25_000_000, ELECTRON_500MEV, 1e-9, chicane_lattice(50), 128)
    if name == "fodo8_grad_1e6_64":
        return Workload(name, 1_000_000, PROTON_1GEV, 10e-9, fodo8_lattice(KS_FODO8, 5, 2), 64)
    raise KeyError(name)
