"""Thin dipole edges and constant focusing on the GPU (through the C ABI)
against the oracle: tracking with space charge (a chicane of rectangular
bends), calls split between slices with edges in between, per-slice
diagnostics, constant focusing, and the reverse mode through thin maps."""
import numpy as np
import pytest
import torch

import beamgen as bg
from oracle import adjoint as adj
from oracle import physics as ph
from oracle import track as tr
from tests.parity import REL_TOL, coord_rel_err, oracle_ref

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def bt():
    import paper_2208_02382_b300 as p
    from paper_2208_02382_b300 import build
    build.build()
    return p


def _els(bt, lat):
    return [bt.Element(e.kind, e.length, e.k, e.angle, e.nslice, e.k2) for e in lat]


def _beam(bt, c, species, charge):
    sp = bt.Species(species.mass_MeV, species.kinetic_MeV, species.charge_sign)
    return bt.Beam(torch.tensor(c, dtype=torch.float64, device=DEV), sp, charge)


def _np(beam):
    order = np.argsort(beam.ids.cpu().numpy())
    return beam.coords.cpu().numpy()[:, order]


@pytest.mark.parametrize("space_charge", [True, False])
def test_rectangular_chicane_matches_oracle(bt, space_charge):
    sp = bg.ELECTRON_500MEV
    lat = bg.chicane_rect_lattice(4)
    c0 = bg.gaussian6d(20_001, seed=21)
    trk = bt.Tracker(32)
    beam = _beam(bt, c0, sp, 1e-9)
    trk.track(beam, _els(bt, lat), space_charge=space_charge)
    trk.sync()
    t = tr.Tracker(oracle_ref(sp), 1e-9, 32, space_charge=space_charge)
    want = t.track(c0, lat)
    assert coord_rel_err(_np(beam), want) < REL_TOL
    if space_charge:
        assert trk.regrid_log() == t.regrid_log


def test_split_calls_apply_edges_once(bt):
    sp = bg.ELECTRON_500MEV
    lat = bg.chicane_rect_lattice(3)
    K = len(ph.slice_schedule(lat))
    c0 = bg.gaussian6d(5000, seed=22)
    trk = bt.Tracker(16)
    beam = _beam(bt, c0, sp, 1e-9)
    els = _els(bt, lat)
    for a, b in ((0, 7), (7, 8), (8, K)):        # splits land next to edges
        trk.track(beam, els, a, b - a)
    trk.sync()
    t = tr.Tracker(oracle_ref(sp), 1e-9, 16)
    want = t.track(c0, lat)
    assert coord_rel_err(_np(beam), want) < REL_TOL


def test_diagnostics_with_edges_and_constant_focusing(bt):
    sp = bg.PROTON_1GEV
    lat = [bg.constf(0.5, 1.2, 0.7, 3), bg.dipedge(0.05, 0.4), bg.drift(0.3, 2),
           bg.dipedge(-0.05, 0.4), bg.constf(0.4, 0.9, 1.4, 2), bg.dipedge(0.1, 0.2)]
    c0 = bg.gaussian6d(4000, seed=23)
    trk = bt.Tracker(16)
    beam = _beam(bt, c0, sp, 5e-9)
    diag = trk.track(beam, _els(bt, lat), diagnostics=True).cpu().numpy()
    trk.sync()
    t = tr.Tracker(oracle_ref(sp), 5e-9, 16)
    want_d = []
    want = t.track(c0, lat, diagnostics=want_d)
    assert coord_rel_err(_np(beam), want) < REL_TOL
    want_d = np.array(want_d)
    scale = np.maximum(np.abs(want_d), np.abs(want_d).max(axis=0) * 1e-6)
    assert np.max(np.abs(diag - want_d) / scale) < 1e-10


def test_gradient_through_edges_matches_oracle(bt):
    sp = bg.PROTON_1GEV
    xi = bg.standard_normal6(3000, seed=24)
    lat = []
    for e in bg.fodo8_lattice(bg.KS_FODO8, periods=1, nslice=1):
        lat += [e, bg.dipedge(0.03, 0.25)]
    w = np.array([1.0, 0.5, -0.3, 0.2])
    trk = bt.Tracker(16)
    spc = bt.Species(sp.mass_MeV, sp.kinetic_MeV, sp.charge_sign)
    beam = bt.Beam(bt.twiss_beam(bg.TWISS_FODO, torch.tensor(xi, device=DEV)), spc, 10e-9)
    trk.grad_forward(beam, _els(bt, lat), 6)
    dk, S, _ = trk.grad_backward(beam, w)
    o = adj.gradients(xi, bg.TWISS_FODO, lat, oracle_ref(sp), 10e-9, 16, w)
    dk, odk = np.array(dk), o["dk"]
    assert np.max(np.abs(dk - odk)) / np.max(np.abs(odk)) < 1e-9
    dtw = np.array(bt.twiss_grad(bg.TWISS_FODO, S))
    assert np.max(np.abs(dtw - o["dtwiss"])) / np.max(np.abs(o["dtwiss"])) < 1e-9
