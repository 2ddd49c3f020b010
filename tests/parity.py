"""Helpers shared by the GPU parity tests: the comparison metric and the
conversion between oracle arrays and the CUDA path's tensors."""
from __future__ import annotations

import numpy as np

import beamgen as bg
from oracle import physics as ph

# Tolerance stated by the task for FP64 phase-space coordinates and grid potentials.
REL_TOL = 1e-11


def coord_rel_err(a: np.ndarray, b: np.ndarray) -> float:
    """max_p |a_p - b_p| / max(|b_p|, rms(b)) per coordinate row, max over rows."""
    worst = 0.0
    for r in range(a.shape[0]):
        rms = float(np.sqrt(np.mean(b[r] ** 2))) if b.shape[1] else 0.0
        den = np.maximum(np.abs(b[r]), rms)
        den = np.where(den > 0, den, 1.0)
        if b.shape[1]:
            worst = max(worst, float(np.max(np.abs(a[r] - b[r]) / den)))
    return worst


def grid_rel_err(a: np.ndarray, b: np.ndarray) -> float:
    """max |a - b| / max |b|."""
    m = float(np.abs(b).max())
    return float(np.abs(a - b).max()) / (m if m > 0 else 1.0)


def oracle_ref(species: bg.Species) -> ph.RefPart:
    return ph.RefPart(species.mass_MeV, species.kinetic_MeV, species.charge_sign)
