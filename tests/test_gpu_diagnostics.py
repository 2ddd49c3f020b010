"""Listing-1 bunches and per-slice diagnostics on the GPU (through the C ABI)
against the oracle, and the paper's FODO benchmark end to end: a 2 GeV
electron Waterbag bunch matched to the FODO cell (2 nm), 25 slices per
element, space charge off and on."""
import math

import numpy as np
import pytest
import torch

import beamgen as bg
from oracle import distribution as ds
from oracle import physics as ph
from oracle import track as tr
from tests.parity import REL_TOL, coord_rel_err

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
P = bg.LISTING1_WATERBAG
E2GEV = bg.ELECTRON_2GEV


@pytest.fixture(scope="module")
def bt():
    import paper_2208_02382_b300 as p
    from paper_2208_02382_b300 import build
    build.build()
    return p


def _inputs(n, seed):
    z = bg.standard_normal6(n, seed=seed)
    u = bg.uniform01(n, seed=seed)
    return z, u, torch.tensor(z, device=DEV), torch.tensor(u, device=DEV)


@pytest.mark.parametrize("kind,n", [("waterbag", 10_000), ("gaussian", 3_001), ("waterbag", 1)])
def test_distribution_matches_oracle(bt, kind, n):
    z, u, zt, ut = _inputs(n, seed=n)
    got = bt.distribution_beam(kind, P, zt, ut if kind == "waterbag" else None).cpu().numpy()
    want = ds.waterbag(z, u, P) if kind == "waterbag" else ds.gaussian(z, P)
    assert coord_rel_err(got, want) < 1e-14


def _diag_err(got, want):
    # per-slice moments: relative to the slice's rms scale per coordinate
    worst = 0.0
    for g, w in zip(got, want):
        cov = np.zeros((6, 6))
        cov[np.triu_indices(6)] = w[6:]
        sig = np.sqrt(np.diag(cov))
        scale = np.concatenate([sig, np.outer(sig, sig)[np.triu_indices(6)]])
        worst = max(worst, float(np.max(np.abs(g - w) / scale)))
    return worst


@pytest.mark.parametrize("space_charge", [False, True])
def test_fodo_benchmark_per_slice_moments_match_oracle(bt, space_charge):
    n = 10_000
    z, u, zt, ut = _inputs(n, seed=0)
    c0 = ds.waterbag(z, u, P)
    lat = bg.fodo_cell(25)
    sp = bt.Species(E2GEV.mass_MeV, E2GEV.kinetic_MeV, E2GEV.charge_sign)
    beam = bt.Beam(bt.distribution_beam("waterbag", P, zt, ut), sp, 1e-9)
    trk = bt.Tracker(32)
    diag = trk.track(beam, lat, space_charge=space_charge, diagnostics=True).cpu().numpy()
    trk.sync()
    ref = ph.RefPart(E2GEV.mass_MeV, E2GEV.kinetic_MeV, E2GEV.charge_sign)
    t = tr.Tracker(ref, 1e-9, 32, space_charge=space_charge)
    want_diag = []
    final = t.track(c0, lat, diagnostics=want_diag)
    assert diag.shape == (125, 27)
    assert _diag_err(diag, np.array(want_diag)) < 1e-11
    order = np.argsort(beam.ids.cpu().numpy())
    assert coord_rel_err(beam.coords.cpu().numpy()[:, order], final) < REL_TOL
    if not space_charge:
        # the benchmark's check: emittances constant at every slice end
        e0 = tr.moments(c0)
        for d in diag:
            cov = np.zeros((6, 6))
            cov[np.triu_indices(6)] = d[6:]
            for uu, name in ((0, "eps_x"), (2, "eps_y")):
                eps = math.sqrt(cov[uu, uu] * cov[uu + 1, uu + 1] - cov[uu, uu + 1] ** 2)
                assert eps == pytest.approx(e0[name], rel=1e-11)


def test_diagnostics_do_not_change_tracking(bt):
    n = 5000
    z, u, zt, ut = _inputs(n, seed=3)
    sp = bt.Species(E2GEV.mass_MeV, E2GEV.kinetic_MeV, E2GEV.charge_sign)
    lat = bg.fodo_cell(5)
    b1 = bt.Beam(bt.distribution_beam("waterbag", P, zt, ut), sp, 1e-9)
    b2 = bt.Beam(bt.distribution_beam("waterbag", P, zt, ut), sp, 1e-9)
    t1, t2 = bt.Tracker(16), bt.Tracker(16)
    t1.track(b1, lat)
    t2.track(b2, lat, diagnostics=True)
    torch.cuda.synchronize()
    assert torch.equal(b1.coords, b2.coords) and torch.equal(b1.ids, b2.ids)
