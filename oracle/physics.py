"""Constants, reference particle, linear element maps and the slice schedule.

Oracle (test infrastructure only; see oracle/__init__.py).

Paper anchors (arXiv:2208.02382):
  * §Model Assumptions: particles are pushed in s by symplectic maps accurate
    through linear order about the reference orbit.
  * Listing 1: elements Drift(ds, nslice), Quad(ds, k, nslice); reference
    particle set by set_energy_MeV(energy, mass); `ns` slices per element.
  * §Benchmark: Berlin-Zeuthen chicane: sector bends (element list is a reading).

Coordinates (reading; the paper names none): x, y [m]; px, py = p_x/p_ref,
p_y/p_ref; t = c*(t - t_ref) [m]; pt = -(E - E_ref)/(p_ref c).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# CODATA 2018
C_LIGHT = 299792458.0                # m/s
Q_E = 1.602176634e-19                # C
EPS0 = 8.8541878128e-12              # F/m

DRIFT, QUAD, SBEND, DIPEDGE, CONSTF, MULTIPOLE = 0, 1, 2, 3, 4, 5
X, PX, Y, PY, T, PT = range(6)


@dataclass(frozen=True)
class RefPart:
    """Reference particle from kinetic energy W and rest energy mc^2 [MeV].

    Reading of Listing 1 `set_energy_MeV(energy_MeV, mass_MeV)`: the energy is
    kinetic.  gamma = 1 + W/mc^2, beta*gamma = sqrt(gamma^2 - 1),
    beta = beta*gamma / gamma.
    """
    mass_MeV: float
    kinetic_MeV: float
    charge_sign: float = 1.0

    @property
    def gamma(self) -> float:
        return 1.0 + self.kinetic_MeV / self.mass_MeV

    @property
    def betagamma(self) -> float:
        g = self.gamma
        return math.sqrt(g * g - 1.0)

    @property
    def beta(self) -> float:
        return self.betagamma / self.gamma

    @property
    def mass_eV(self) -> float:
        return self.mass_MeV * 1e6


def drift_matrix(ds: float, ref: RefPart) -> np.ndarray:
    """Linear drift of length ds: x += ds*px, y += ds*py, t += ds/(beta gamma)^2 * pt.

    The t-row is the first-order time of flight: d(1/beta)/d(gamma) =
    -1/(beta gamma)^3 and pt = -dgamma/(beta gamma).
    """
    m = np.eye(6)
    m[X, PX] = ds
    m[Y, PY] = ds
    m[T, PT] = ds / ref.betagamma ** 2
    return m


def _focus_block(ds: float, k: float) -> np.ndarray:
    """2x2 transfer block of the linear equation u'' = -k u over ds."""
    if k > 0.0:
        w = math.sqrt(k)
        c, s = math.cos(w * ds), math.sin(w * ds)
        return np.array([[c, s / w], [-w * s, c]])
    if k < 0.0:
        w = math.sqrt(-k)
        c, s = math.cosh(w * ds), math.sinh(w * ds)
        return np.array([[c, s / w], [w * s, c]])
    return np.array([[1.0, ds], [0.0, 1.0]])


def quad_matrix(ds: float, k: float, ref: RefPart) -> np.ndarray:
    """Thick quadrupole of length ds and strength k [1/m^2]; k > 0 focuses x.

    x'' = -k x, y'' = +k y; t-row as the drift (reading: linear order, the
    quadrupole field does not change the energy).
    """
    m = np.eye(6)
    m[X:X + 2, X:X + 2] = _focus_block(ds, k)
    m[Y:Y + 2, Y:Y + 2] = _focus_block(ds, -k)
    m[T, PT] = ds / ref.betagamma ** 2
    return m


def sbend_matrix(ds: float, rho: float, ref: RefPart) -> np.ndarray:
    """Sector bend slice of arc length ds and signed bend radius rho [m].

    theta = ds/rho; y-plane is a drift.  With delta = dp/p = -pt/beta (first
    order), the x-plane carries dispersion rho(1-cos) delta and the t-row the
    path-length change plus the velocity term (reading; derived, checked to be
    symplectic by the oracle tests):
      x'  = cos x + rho sin px - rho (1-cos)/beta pt
      px' = -sin/rho x + cos px - sin/beta pt
      t'  = t + sin/beta x + rho (1-cos)/beta px + rho (sin/beta^2 - theta) pt
    """
    th = ds / rho
    c, s = math.cos(th), math.sin(th)
    b = ref.beta
    m = np.eye(6)
    m[X, X], m[X, PX], m[X, PT] = c, rho * s, -rho * (1.0 - c) / b
    m[PX, X], m[PX, PX], m[PX, PT] = -s / rho, c, -s / b
    m[Y, PY] = ds
    m[T, X], m[T, PX], m[T, PT] = s / b, rho * (1.0 - c) / b, rho * (s / b ** 2 - th)
    return m


def dipedge_matrix(psi: float, curvature: float) -> np.ndarray:
    """Thin hard-edge dipole fringe field (K. L. Brown, SLAC-75, 1972): edge
    angle psi, bend curvature h = 1/rho;  px += h tan(psi) x,
    py -= h tan(psi) y.  A rectangular bend of angle theta has psi = theta/2
    at both faces.  (Paper §Benchmark: chicane; reading: edge elements make
    the chicane achromatic.)"""
    m = np.eye(6)
    m[PX, X] = curvature * math.tan(psi)
    m[PY, Y] = -curvature * math.tan(psi)
    return m


def constf_matrix(ds: float, kx: float, ky: float, ref: RefPart) -> np.ndarray:
    """Constant linear focusing over ds (paper §Numerical Experiments: "a
    stationary beam in a constant focusing channel"): u'' = -k_u u per
    transverse plane, t-row as the drift (reading: no longitudinal focusing)."""
    m = np.eye(6)
    m[X:X + 2, X:X + 2] = _focus_block(ds, kx)
    m[Y:Y + 2, Y:Y + 2] = _focus_block(ds, ky)
    m[T, PT] = ds / ref.betagamma ** 2
    return m


def multipole_kick(coords: np.ndarray, order: int, kn: float, ks: float) -> np.ndarray:
    """Thin multipole of order m (1 dipole, 2 quadrupole, 3 sextupole, ...) with
    integrated normal and skew strengths kn, ks [1/m^(m-1)] (paper §Numerical
    Experiments: a chain of thin multipoles; the paper prints no formula).

    Reading: the field of a straight 2D multipole magnet of length L is
    B_y + i B_x = (B rho / L) (kn + i ks) (x + i y)^(m-1) / (m-1)!, and the
    Lorentz force on a reference-rigidity particle over L changes the scaled
    momenta by dpx = -L B_y / (B rho), dpy = +L B_x / (B rho), so that
        dpx - i dpy = -(kn + i ks) (x + i y)^(m-1) / (m-1)!
    (m = 2, kn > 0: px -= kn x, py += kn y, focusing in x like a quadrupole
    with k > 0; m = 3: px -= kn (x^2 - y^2)/2, py += kn x y).  x, y, t and pt
    are unchanged (a thin kick)."""
    if order < 1:
        raise ValueError("multipole order must be >= 1")
    out = np.array(coords, dtype=np.float64, copy=True)
    z = out[X] + 1j * out[Y]
    zp = np.ones_like(z)
    for _ in range(order - 1):     # z^(m-1) by repeated multiplication
        zp = zp * z
    w = (kn + 1j * ks) * zp / math.factorial(order - 1)
    out[PX] = out[PX] - w.real
    out[PY] = out[PY] + w.imag
    return out


def is_thin(e) -> bool:
    """Thin elements (dipole edges, multipoles) act between slices and take
    no kick."""
    return e.kind in (DIPEDGE, MULTIPOLE)


def is_linear_thin(e) -> bool:
    return e.kind == DIPEDGE


def thin_apply(coords: np.ndarray, lattice, ie: int, ref: "RefPart") -> np.ndarray:
    """Apply the thin element `ie` to (6, n) coordinates."""
    e = lattice[ie]
    if e.kind == MULTIPOLE:
        return multipole_kick(coords, int(e.order), e.k, getattr(e, "k2", 0.0))
    return push(coords, thin_matrix(lattice, [ie], ref))


def element_matrix(kind: int, length: float, k: float, angle: float, ds: float,
                   ref: RefPart, k2: float = 0.0) -> np.ndarray:
    """Map of a piece of arc length ds of the given element (the whole of a
    thin element: ds is ignored)."""
    if kind == DRIFT:
        return drift_matrix(ds, ref)
    if kind == QUAD:
        return quad_matrix(ds, k, ref)
    if kind == DIPEDGE:
        return dipedge_matrix(angle, k)
    if kind == CONSTF:
        return constf_matrix(ds, k, k2, ref)
    if kind == SBEND:
        if angle == 0.0:
            return drift_matrix(ds, ref)
        return sbend_matrix(ds, length / angle, ref)
    raise ValueError(f"unknown element type {kind}")


def slice_schedule(lattice) -> list:
    """Split-operator schedule (paper §Model Assumptions; Listing 1 `nslice`).

    Each element of length L with `nslice` slices contributes nslice slices of
    length ds = L/nslice.  Each slice is one space-charge kick.  Returns a list
    of (element index, ds) per slice, in beamline order.
    """
    out = []
    for ie, e in enumerate(lattice):
        if is_thin(e):
            continue
        if e.nslice <= 0 or e.length <= 0.0:
            raise ValueError("element needs nslice > 0 and length > 0")
        ds = e.length / e.nslice
        out.extend((ie, ds) for _ in range(e.nslice))
    return out


def thin_schedule(lattice) -> tuple:
    """Thin elements in beamline order around the slices: (before, after)
    with before[j] the indices of the thin elements between slice j-1 and
    slice j (before slice 0 for j = 0) and `after` those past the last slice.
    A call tracking slices [a, b) applies before[j] ahead of slice j, and
    `after` when b is the end of the lattice."""
    n = len(slice_schedule(lattice))
    before = [[] for _ in range(n)]
    after = []
    j = 0
    for ie, e in enumerate(lattice):
        if is_thin(e):
            (before[j] if j < n else after).append(ie)
        else:
            j += e.nslice
    return before, after


def thin_matrix(lattice, indices, ref: RefPart) -> np.ndarray:
    """Product of the (linear) thin elements `indices` in beamline order."""
    m = np.eye(6)
    for ie in indices:
        e = lattice[ie]
        if not is_linear_thin(e):
            raise ValueError("thin_matrix: element %d is not linear" % ie)
        m = element_matrix(e.kind, e.length, e.k, e.angle, 0.0, ref, getattr(e, "k2", 0.0)) @ m
    return m


def symplectic_form() -> np.ndarray:
    """J for canonical pairs (x, px), (y, py), (t, pt)."""
    j = np.zeros((6, 6))
    for a in (0, 2, 4):
        j[a, a + 1] = 1.0
        j[a + 1, a] = -1.0
    return j


def push(coords: np.ndarray, m: np.ndarray) -> np.ndarray:
    """Apply a 6x6 linear map to (6, n) coordinates: each output row is the sum
    over the six input rows in order (no blocking)."""
    out = np.zeros_like(coords)
    for r in range(6):
        acc = np.zeros(coords.shape[1])
        for c in range(6):
            if m[r, c] != 0.0:
                acc = acc + m[r, c] * coords[c]
        out[r] = acc
    return out
