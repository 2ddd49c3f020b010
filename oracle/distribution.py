"""Initial bunches in the parametrisation of Listing 1 (`distribution.Waterbag`
and its Gaussian counterpart).

Oracle (test infrastructure only; see oracle/__init__.py).

Paper anchor (arXiv:2208.02382, Listing 1): a Waterbag distribution given by
sigmaX, sigmaY, sigmaT, sigmaPx, sigmaPy, sigmaPt and the correlations muxpx,
muypy, mutpt.  Reading (the paper prints no formula; pinned by the worked
example, whose printed values follow from the matched FODO optics only under
it): per plane, with lam = sigmaX, lamp = sigmaPx, mu = muxpx,

    u  = lam / sqrt(1 - mu^2) * a
    pu = lamp * (b - mu / sqrt(1 - mu^2) * a)

for unit-rms, uncorrelated a, b: rms u = lam/sqrt(1-mu^2), rms pu =
lamp/sqrt(1-mu^2), correlation coefficient -mu.

Waterbag: uniform inside a 6D ball; the unit-rms ball has radius sqrt(8)
(for a uniform n-ball of radius R, <x_i^2> = R^2/(n+2)).  Its points are the
direction of six standard normals times sqrt(8) u^(1/6), u uniform in [0, 1).
The random draws are inputs, so the oracle and the CUDA path transform the
same numbers.
"""
from __future__ import annotations

import math

import numpy as np

from .physics import PT, PX, PY, T, X, Y

PLANES = ((X, PX), (Y, PY), (T, PT))


def correlate(unit: np.ndarray, params) -> np.ndarray:
    """Apply the per-plane parametrisation to unit-rms coordinates (6, n).
    params = (sigmaX, sigmaY, sigmaT, sigmaPx, sigmaPy, sigmaPt, muxpx, muypy,
    mutpt) as in Listing 1."""
    p = [float(v) for v in params]
    lam, lamp, mu = p[0:3], p[3:6], p[6:9]
    out = np.empty_like(unit, dtype=np.float64)
    for i, (u, pu) in enumerate(PLANES):
        root = math.sqrt(1.0 - mu[i] * mu[i])
        a, b = unit[u], unit[pu]
        out[u] = lam[i] / root * a
        out[pu] = lamp[i] * (b - mu[i] / root * a)
    return out


def waterbag(normals: np.ndarray, uniforms: np.ndarray, params) -> np.ndarray:
    """Waterbag bunch from six standard normals and one uniform per particle."""
    r = np.sqrt(np.sum(normals * normals, axis=0))
    radius = math.sqrt(8.0) * uniforms ** (1.0 / 6.0)
    return correlate(normals / r * radius, params)


def gaussian(normals: np.ndarray, params) -> np.ndarray:
    """Gaussian bunch with the same parametrisation (unit normals in)."""
    return correlate(normals, params)


def covariance(params) -> np.ndarray:
    """Population covariance of either distribution (unit-rms, uncorrelated
    inputs), written out per plane: var u = lam^2/(1-mu^2),
    var pu = lamp^2/(1-mu^2), cov(u, pu) = -mu lam lamp/(1-mu^2)."""
    p = [float(v) for v in params]
    lam, lamp, mu = p[0:3], p[3:6], p[6:9]
    c = np.zeros((6, 6))
    for i, (u, pu) in enumerate(PLANES):
        d = 1.0 - mu[i] * mu[i]
        c[u, u] = lam[i] ** 2 / d
        c[pu, pu] = lamp[i] ** 2 / d
        c[u, pu] = c[pu, u] = -mu[i] * lam[i] * lamp[i] / d
    return c
