"""Space-charge kick of the split-operator step: box rule, CIC deposit,
integrated Green's function, Hockney doubled-grid solve, field, gather + kick.

Oracle (test infrastructure only; see oracle/__init__.py).

Paper anchors (arXiv:2208.02382):
  * §Model Assumptions: fields are electrostatic in the bunch rest frame; the
    Poisson equation is solved there; linearisation assumes a negligible
    velocity spread, so the rest frame is reached by the reference Lorentz
    boost; space charge enters through a map-based split-operator step.
  * §ImpactX: charge deposition and Poisson solve are the reused PIC routines.
  * Listing 1: set_particle_shape (B-spline order; order 1 = CIC here),
    init_grids (mesh covering the beam).
The formulas are readings (the paper prints none); each function names its own.

Array layout: grids are numpy arrays indexed [z, y, x] (x fastest in memory),
i.e. node (i, j, l) of an n^3 grid sits at flat index i + n*(j + n*l).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from . import build as _build
from .physics import EPS0, PT, PX, PY, RefPart, T, X, Y

# ---------------------------------------------------------------- rest frame

def rest_frame(coords: np.ndarray, ref: RefPart) -> np.ndarray:
    """Rest-frame positions (3, n): X = x, Y = y, Z = -beta*gamma*t.

    Reading of §Model Assumptions: the lab longitudinal offset at fixed time is
    z = -beta t (t is c times the time lag), boosted by gamma into the rest frame.
    """
    return np.stack([coords[X], coords[Y], -ref.betagamma * coords[T]])


# ----------------------------------------------------------------- box rule

@dataclass(frozen=True)
class Box:
    lo: tuple
    hi: tuple

    def h(self, n: int) -> tuple:
        """Node spacing per dimension: (hi - lo)/(n - 1)."""
        return tuple((self.hi[d] - self.lo[d]) / (n - 1) for d in range(3))


def box_rule(pos: np.ndarray, box: Box | None) -> tuple:
    """Grid box with hysteresis (reading of Listing 1 `init_grids`; the paper
    states no rule).  Returns (box, regridded).

    With exact per-dimension min/max of the rest-frame positions and
    ext = max - min (floored at 1e-6 * the largest extent, or 1e-6 m if every
    extent is zero), a new box is made when there is no box yet, when a
    particle lies outside [lo, hi), or when ext < 0.5 * (hi - lo) in some
    dimension.  The new box is centred on (min + max)/2 with half-width
    0.55 * ext (a 5% margin on each side).
    """
    mn = pos.min(axis=1)
    mx = pos.max(axis=1)
    ext = mx - mn
    big = float(ext.max())
    floor = 1e-6 * big if big > 0.0 else 1e-6
    ext = np.maximum(ext, floor)
    need = box is None
    if not need:
        for d in range(3):
            if mn[d] < box.lo[d] or mx[d] >= box.hi[d] or ext[d] < 0.5 * (box.hi[d] - box.lo[d]):
                need = True
    if not need:
        return box, False
    c = 0.5 * (mn + mx)
    w = 0.55 * ext
    return Box(tuple(float(v) for v in c - w), tuple(float(v) for v in c + w)), True


# ------------------------------------------------------------ CIC weights

def cic_cells(pos: np.ndarray, box: Box, n: int):
    """Cell index and fractional offset per dimension (shape order 1, CIC).

    u = (X - lo)/h, i = floor(u) clamped to [0, n-2], f = u - i; the node
    weights are (1 - f) on node i and f on node i + 1.
    """
    h = box.h(n)
    idx, frac = [], []
    for d in range(3):
        u = (pos[d] - box.lo[d]) / h[d]
        i = np.clip(np.floor(u), 0, n - 2).astype(np.int64)
        idx.append(i)
        frac.append(u - i)
    return idx, frac


def tsc_nodes(pos: np.ndarray, box: Box, n: int):
    """Nearest node and quadratic B-spline weights per dimension (shape order
    2, TSC; Listing 1 set_particle_shape(2)).

    Reading: u = (X - lo)/h is first limited to [1/2, n - 3/2] (so the three
    nodes i-1, i, i+1 exist; inside the box rule's 5% margin this only acts on
    grids of fewer than ~20 nodes), i = floor(u + 1/2) limited to [1, n-2],
    f = u - i, and the weights of nodes i-1, i, i+1 are
    (1/2 - f)^2 / 2, 3/4 - f^2, (1/2 + f)^2 / 2.
    """
    h = box.h(n)
    idx, wts = [], []
    for d in range(3):
        u = np.clip((pos[d] - box.lo[d]) / h[d], 0.5, n - 1.5)
        i = np.clip(np.floor(u + 0.5), 1, n - 2).astype(np.int64)
        f = u - i
        idx.append(i)
        wts.append((0.5 * (0.5 - f) ** 2, 0.75 - f * f, 0.5 * (0.5 + f) ** 2))
    return idx, wts


def deposit(pos: np.ndarray, q_macro: float, box: Box, n: int, shape: int = 1) -> np.ndarray:
    """Charge density on the n^3 node grid (C/m^3), CIC (shape 1) or TSC
    (shape 2).

    Each particle adds q * wx * wy * wz to the 8 nodes of its cell (CIC) or the
    27 nodes around its nearest node (TSC), in particle order, node by node;
    the grid is divided by the cell volume at the end.
    """
    if shape == 2:
        (i, j, l), (wx, wy, wz) = tsc_nodes(pos, box, n)
        rho = np.zeros((n, n, n))
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    np.add.at(rho, (l + dz, j + dy, i + dx),
                              q_macro * (wx[dx + 1] * wy[dy + 1] * wz[dz + 1]))
        h = box.h(n)
        return rho / (h[0] * h[1] * h[2])
    (i, j, l), (fx, fy, fz) = cic_cells(pos, box, n)
    wx, wy, wz = (1.0 - fx, fx), (1.0 - fy, fy), (1.0 - fz, fz)
    rho = np.zeros((n, n, n))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                np.add.at(rho, (l + dz, j + dy, i + dx), q_macro * (wx[dx] * wy[dy] * wz[dz]))
    h = box.h(n)
    return rho / (h[0] * h[1] * h[2])


# ------------------------------------------------- integrated Green's function

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(_build.build())
        lib.oracle_igf_octant.restype = ctypes.c_int
        lib.oracle_igf_octant.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_void_p]
        for f in (lib.oracle_igf_point, lib.oracle_igf_point_double):
            f.restype = ctypes.c_double
            f.argtypes = [ctypes.c_double] * 6
        _LIB = lib
    return _LIB


def igf_point(a, b, c, h) -> float:
    """G at offset (a, b, c) cells (see igf_quad.c) [V m^3 / C]: the potential
    at the origin from unit charge density filling the cell at that offset."""
    return _lib().oracle_igf_point(float(a), float(b), float(c), *map(float, h))


def igf_point_double(a, b, c, h) -> float:
    return _lib().oracle_igf_point_double(float(a), float(b), float(c), *map(float, h))


def igf_octant(n: int, h) -> np.ndarray:
    """(n+1)^3 table G[c, b, a] for offsets a, b, c = 0..n (float128 inside)."""
    out = np.empty((n + 1, n + 1, n + 1))
    rc = _lib().oracle_igf_octant(int(n), float(h[0]), float(h[1]), float(h[2]),
                                  out.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle_igf_octant")
    return out


def green_doubled(n: int, h) -> np.ndarray:
    """Green's function on the (2n)^3 doubled grid (Hockney).

    Index m in [0, 2n) per dimension holds offset m for m <= n and m - 2n for
    m > n; G is even, so entry m holds G(min(m, 2n - m)).  Offset +-n carries
    the true IGF value (reading), which makes the potential exact on nodes
    -1..n, the ghost ring used by the centred-difference field.
    """
    oct_ = igf_octant(n, h)
    m = np.arange(2 * n)
    fold = np.minimum(m, 2 * n - m)
    return oct_[np.ix_(fold, fold, fold)]


def green_hat(n: int, h) -> np.ndarray:
    """Real spectrum of the doubled Green's function, rfftn layout
    (2n, 2n, n+1).  G is real and even, so its DFT is real; the imaginary
    part (rounding noise) is dropped."""
    return np.fft.rfftn(green_doubled(n, h)).real.copy()


# -------------------------------------------------------------------- solve

def solve(rho: np.ndarray, h, ghat: np.ndarray | None = None) -> np.ndarray:
    """Open-boundary potential phi = G (*) rho (aperiodic convolution), via the
    zero-padded (2n)^3 FFT (Hockney).  numpy's FFT is the library primitive;
    the inverse carries the 1/(2n)^3 normalisation.

    Returns phi on nodes -1..n per dimension, shape (n+2)^3, where array index
    k holds node k - 1.
    """
    n = rho.shape[0]
    if ghat is None:
        ghat = green_hat(n, h)
    pad = np.zeros((2 * n,) * 3)
    pad[:n, :n, :n] = rho
    full = np.fft.irfftn(np.fft.rfftn(pad) * ghat, s=(2 * n,) * 3, axes=(0, 1, 2))
    k = np.arange(-1, n + 1) % (2 * n)
    return full[np.ix_(k, k, k)]


def solve_direct(rho: np.ndarray, h) -> np.ndarray:
    """Brute-force phi_i = sum_j rho_j G(i - j) on nodes -1..n (tiny n only)."""
    n = rho.shape[0]
    oct_ = igf_octant(n, h)
    out = np.zeros((n + 2,) * 3)
    src = np.argwhere(rho != 0.0)
    nodes = np.arange(-1, n + 1)
    for (l, j, i) in src:
        dz = np.abs(nodes - l)
        dy = np.abs(nodes - j)
        dx = np.abs(nodes - i)
        out += rho[l, j, i] * oct_[np.ix_(dz, dy, dx)]
    return out


# -------------------------------------------------------------------- field

def field(phi: np.ndarray, h) -> np.ndarray:
    """Rest-frame field E = -grad phi on nodes 0..n-1 by centred differences,
    using the ghost nodes -1 and n (reading; the paper names no scheme).
    Returns (3, n, n, n) for (Ex, Ey, Ez), each indexed [z, y, x]."""
    c = phi[1:-1, 1:-1, 1:-1]
    ex = -(phi[1:-1, 1:-1, 2:] - phi[1:-1, 1:-1, :-2]) / (2.0 * h[0])
    ey = -(phi[1:-1, 2:, 1:-1] - phi[1:-1, :-2, 1:-1]) / (2.0 * h[1])
    ez = -(phi[2:, 1:-1, 1:-1] - phi[:-2, 1:-1, 1:-1]) / (2.0 * h[2])
    assert ex.shape == c.shape
    return np.stack([ex, ey, ez])


# ------------------------------------------------------------ gather + kick

def gather(pos: np.ndarray, efield: np.ndarray, box: Box, shape: int = 1) -> np.ndarray:
    """Field at each particle with the same weights as the deposit (CIC or
    TSC)."""
    n = efield.shape[1]
    if shape == 2:
        (i, j, l), (wx, wy, wz) = tsc_nodes(pos, box, n)
        out = np.zeros((3, pos.shape[1]))
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    w = wx[dx + 1] * wy[dy + 1] * wz[dz + 1]
                    for c in range(3):
                        out[c] += w * efield[c, l + dz, j + dy, i + dx]
        return out
    (i, j, l), (fx, fy, fz) = cic_cells(pos, box, n)
    wx, wy, wz = (1.0 - fx, fx), (1.0 - fy, fy), (1.0 - fz, fz)
    out = np.zeros((3, pos.shape[1]))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = wx[dx] * wy[dy] * wz[dz]
                for c in range(3):
                    out[c] += w * efield[c, l + dz, j + dy, i + dx]
    return out


def kick(coords: np.ndarray, e_at: np.ndarray, ds: float, ref: RefPart) -> np.ndarray:
    """Momentum kick over a slice ds from the rest-frame field (reading of
    §Model Assumptions; derived, the paper gives no formula).

    Lab transverse force q E'/gamma for a time ds/(beta c), over p_ref:
        dpx = sign * E'x * ds / (mc^2[eV] * (beta gamma)^2)   (and y)
    Work q E'z ds (E_z is boost-invariant), over p_ref c:
        dpt = -sign * E'z * ds / (mc^2[eV] * beta gamma)
    """
    out = coords.copy()
    s = ref.charge_sign
    kt = s * ds / (ref.mass_eV * ref.betagamma ** 2)
    kz = -s * ds / (ref.mass_eV * ref.betagamma)
    out[PX] = coords[PX] + kt * e_at[0]
    out[PY] = coords[PY] + kt * e_at[1]
    out[PT] = coords[PT] + kz * e_at[2]
    return out


def macro_charge(bunch_charge_C: float, n: int, ref: RefPart) -> float:
    """q per macroparticle = sign * |Q| / N (Listing 1 add_particles(qm, Q, ...))."""
    return ref.charge_sign * abs(bunch_charge_C) / n if n > 0 else 0.0


def coulomb_direct(pos: np.ndarray, q_macro: float) -> np.ndarray:
    """Rest-frame field at each particle from all others (no self term), by the
    direct Coulomb sum.  Brute force, O(n^2): small n only."""
    d = pos[:, :, None] - pos[:, None, :]
    r2 = (d * d).sum(axis=0)
    np.fill_diagonal(r2, np.inf)
    inv3 = r2 ** -1.5
    return q_macro / (4.0 * math.pi * EPS0) * (d * inv3[None]).sum(axis=2)
