"""Split-operator tracking loop and beam moments.

Oracle (test infrastructure only; see oracle/__init__.py).

Paper anchors (arXiv:2208.02382):
  * §Model Assumptions: space charge through a map-based split-operator
    approach.  Reading: second-order Strang splitting per slice,
    map(ds/2) -> space-charge kick over ds -> map(ds/2).
  * Listing 1: `sim.evolve()` walks the lattice element by element and slice by
    slice; `set_space_charge(False)` switches the kick off.
  * §ImpactX (beam statistics) and §Benchmark FODO / IOTA (second moments and
    emittances are the checked observables).
"""
from __future__ import annotations

import numpy as np

from . import physics as ph
from . import spacecharge as sc


class Tracker:
    """Holds what persists between slices: the grid box, the Green's function
    spectrum for the box's cell size, the kick counter and the regrid log."""

    def __init__(self, ref: ph.RefPart, bunch_charge_C: float, n_grid: int,
                 space_charge: bool = True, shape: int = 1):
        if n_grid < 2:
            raise ValueError("n_grid >= 2")
        if shape not in (1, 2):
            raise ValueError("shape 1 (CIC) or 2 (TSC)")
        self.shape = int(shape)
        self.ref = ref
        self.bunch_charge_C = bunch_charge_C
        self.n = int(n_grid)
        self.space_charge = bool(space_charge)
        self.box = None
        self.ghat = None
        self.ghat_h = None
        self.kick_index = 0
        self.regrid_log = []

    def space_charge_kick(self, coords: np.ndarray, ds: float) -> np.ndarray:
        """One space-charge kick over ds at the current positions."""
        npart = coords.shape[1]
        if npart == 0:
            return coords
        if not np.all(np.isfinite(coords)):
            raise FloatingPointError("non-finite particle coordinates")
        pos = sc.rest_frame(coords, self.ref)
        self.box, regridded = sc.box_rule(pos, self.box)
        if regridded:
            self.regrid_log.append(self.kick_index)
        h = self.box.h(self.n)
        if self.ghat is None or self.ghat_h != h:
            self.ghat = sc.green_hat(self.n, h)
            self.ghat_h = h
        q = sc.macro_charge(self.bunch_charge_C, npart, self.ref)
        rho = sc.deposit(pos, q, self.box, self.n, self.shape)
        phi = sc.solve(rho, h, self.ghat)
        e = sc.field(phi, h)
        e_at = sc.gather(pos, e, self.box, self.shape)
        return sc.kick(coords, e_at, ds, self.ref)

    def track(self, coords: np.ndarray, lattice, first_kick: int = 0,
              nkicks: int | None = None, diagnostics: list | None = None) -> np.ndarray:
        """Track (6, n) coordinates through slices [first_kick, first_kick+nkicks)
        of the lattice's slice schedule.  Each slice: map(ds/2), kick(ds) when
        space charge is on, map(ds/2).  With `diagnostics`, the moments_vector
        of the bunch at the end of every slice is appended to it (Listing 1
        set_slice_step_diagnostics)."""
        sched = ph.slice_schedule(lattice)
        before, after = ph.thin_schedule(lattice)
        stop = len(sched) if nkicks is None else min(len(sched), first_kick + nkicks)
        c = np.array(coords, dtype=np.float64, copy=True)
        for j in range(first_kick, stop):
            ie, ds = sched[j]
            for it in before[j]:
                c = ph.thin_apply(c, lattice, it, self.ref)
            e = lattice[ie]
            half = ph.element_matrix(e.kind, e.length, e.k, e.angle, 0.5 * ds, self.ref,
                                     getattr(e, "k2", 0.0))
            c = ph.push(c, half)
            if self.space_charge:
                c = self.space_charge_kick(c, ds)
            c = ph.push(c, half)
            self.kick_index += 1
            if diagnostics is not None:
                diagnostics.append(moments_vector(c))
        if stop == len(sched) and stop > first_kick:
            for it in after:
                c = ph.thin_apply(c, lattice, it, self.ref)
        return c


def moments(coords: np.ndarray) -> dict:
    """Beam statistics: means, centred second moments (two passes), rms sizes
    and unnormalised rms emittances per plane,
    eps = sqrt(<du^2><dpu^2> - <du dpu>^2)."""
    n = coords.shape[1]
    mean = coords.sum(axis=1) / n
    d = coords - mean[:, None]
    cov = (d @ d.T) / n
    out = {"mean": mean, "cov": cov, "sigma": np.sqrt(np.diag(cov))}
    for name, a in (("x", 0), ("y", 2), ("t", 4)):
        out["eps_" + name] = float(np.sqrt(cov[a, a] * cov[a + 1, a + 1] - cov[a, a + 1] ** 2))
    return out


def moments_vector(coords: np.ndarray) -> np.ndarray:
    """27 numbers: the 6 means then the 21 upper-triangle centred second
    moments in row-major order (00, 01, .., 05, 11, .., 55)."""
    m = moments(coords)
    iu = np.triu_indices(6)
    return np.concatenate([m["mean"], m["cov"][iu]])


def moments_vector_exact(coords: np.ndarray) -> np.ndarray:
    """moments_vector in exact rational arithmetic (every double is a
    rational), rounded once to the nearest double per output: the definition
    mean_a = sum x_a / N, C_ab = sum (x_a - mean_a)(x_b - mean_b) / N written
    out without rounding.  Slow: small bunches only."""
    from fractions import Fraction
    n = coords.shape[1]
    if n == 0:
        raise ValueError("moments of an empty bunch")
    cols = [[Fraction(float(v)) for v in coords[a]] for a in range(6)]
    mean = [sum(c, Fraction(0)) / n for c in cols]
    dev = [[v - mean[a] for v in cols[a]] for a in range(6)]
    out = [float(m) for m in mean]
    for a in range(6):
        for b in range(a, 6):
            out.append(float(sum((u * w for u, w in zip(dev[a], dev[b])), Fraction(0)) / n))
    return np.array(out)
