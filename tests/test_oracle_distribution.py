"""Pins of the Listing-1 bunch parametrisation (oracle/distribution.py) and of
the per-slice diagnostics: the population covariance against the worked
example's Twiss optics, the Waterbag's geometry (radius bound, radial law,
unit rms), sample moments at the statistical level, and the paper's FODO
benchmark (a matched beam keeps its emittances slice by slice)."""
import math

import numpy as np
import pytest

import beamgen as bg
from oracle import distribution as ds
from oracle import physics as ph
from oracle import track as tr

P = bg.LISTING1_WATERBAG
REF_E = ph.RefPart(bg.MASS_ELECTRON_MEV, 2000.0, -1.0)


def _fodo_matrix(ref):
    m = np.eye(6)
    for e in bg.fodo_cell(1):
        m = ph.element_matrix(e.kind, e.length, e.k, e.angle, e.length, ref) @ m
    return m


def test_population_covariance_is_the_matched_optics():
    # the worked example's parameters describe the periodic Twiss ellipse of
    # the FODO cell with eps = 2 nm: Sigma = M Sigma M^T for the cell map, to
    # the precision of the printed values (11 significant digits, amplified by
    # the cell map to a few 1e-9)
    c = ds.covariance(P)
    m = _fodo_matrix(REF_E)
    out = m @ c @ m.T
    assert np.abs(out[:4, :4] - c[:4, :4]).max() <= 2e-8 * np.abs(c[:4, :4]).max()
    for u, pu in ((0, 1), (2, 3)):
        eps = math.sqrt(c[u, u] * c[pu, pu] - c[u, pu] ** 2)
        assert eps == pytest.approx(2e-9, rel=1e-9)


def test_correlate_maps_unit_covariance_to_the_population_covariance():
    # correlate is linear: applied to the identity basis it gives columns T
    # with T T^T = covariance (closed form, per plane)
    eye = np.eye(6)
    T = ds.correlate(eye, P)
    assert np.allclose(T @ T.T, ds.covariance(P), rtol=1e-14, atol=1e-30)


def test_waterbag_geometry():
    n = 200_000
    z = bg.standard_normal6(n, seed=5)
    u = bg.uniform01(n, seed=5)
    unit = ds.waterbag(z, u, (1, 1, 1, 1, 1, 1, 0, 0, 0))
    r = np.sqrt(np.sum(unit * unit, axis=0))
    assert r.max() <= math.sqrt(8.0) * (1 + 1e-15)
    # radial law: P(r <= R) = (R / sqrt 8)^6
    for q in (0.3, 0.6, 0.9):
        frac = np.mean(r <= q * math.sqrt(8.0))
        assert frac == pytest.approx(q ** 6, abs=4.0 / math.sqrt(n))
    # unit rms, uncorrelated (statistical level)
    cov = np.cov(unit, bias=True)
    assert np.abs(cov - np.eye(6)).max() < 6.0 / math.sqrt(n)


@pytest.mark.parametrize("kind", ["waterbag", "gaussian"])
def test_sample_moments_reach_the_parameters(kind):
    n = 400_000
    z = bg.standard_normal6(n, seed=11)
    c = ds.waterbag(z, bg.uniform01(n, seed=11), P) if kind == "waterbag" else ds.gaussian(z, P)
    got = np.cov(c, bias=True)
    want = ds.covariance(P)
    scale = np.sqrt(np.outer(np.diag(want), np.diag(want)))
    assert np.abs(got - want).max() / scale.max() < 8.0 / math.sqrt(n) * 10


def test_fodo_benchmark_matched_beam_keeps_its_emittance_per_slice():
    # Benchmark FODO cell (Listing 1): 1e4 Waterbag particles, 2 GeV e-,
    # ns = 25, space charge off: the unnormalised emittances stay constant at
    # every slice end (linear symplectic maps) and the rms sizes oscillate
    n = 10_000
    c0 = ds.waterbag(bg.standard_normal6(n, seed=0), bg.uniform01(n, seed=0), P)
    t = tr.Tracker(REF_E, 1e-9, 16, space_charge=False)
    diag = []
    t.track(c0, bg.fodo_cell(25), diagnostics=diag)
    assert len(diag) == 125
    m0 = tr.moments(c0)
    for d in diag:
        cov = np.zeros((6, 6))
        cov[np.triu_indices(6)] = d[6:]
        for u in (0, 2):
            eps = math.sqrt(cov[u, u] * cov[u + 1, u + 1] - cov[u, u + 1] ** 2)
            assert eps == pytest.approx(m0["eps_" + "xy"[u // 2]], rel=1e-12)
    sx = [math.sqrt(d[6]) for d in diag]
    assert max(sx) / min(sx) > 1.5
