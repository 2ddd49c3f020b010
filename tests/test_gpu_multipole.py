"""Thin multipoles on the GPU (through the C ABI) against the oracle:
tracking with and without space charge through FODO cells with thin
multipoles between the elements (at the start, between slices of different
elements, two at one point, at the end), calls split at those boundaries, a
batch problem, the refusals (per-slice diagnostics, reverse mode, bad
orders), and a bunch driven to non-finite coordinates ending with a clean
status."""
import numpy as np
import pytest
import torch

import beamgen as bg
from oracle import physics as ph
from oracle import track as tr
from tests.parity import REL_TOL, coord_rel_err, oracle_ref

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SP = bg.PROTON_1GEV
CHARGE = 2e-9


@pytest.fixture(scope="module")
def bt():
    import paper_2208_02382_b300 as p
    from paper_2208_02382_b300 import build
    build.build()
    return p


def _els(bt, lat):
    return [bt.Element(e.kind, e.length, e.k, e.angle, e.nslice, e.k2, e.order) for e in lat]


def _beam(bt, c, charge=CHARGE):
    sp = bt.Species(SP.mass_MeV, SP.kinetic_MeV, SP.charge_sign)
    return bt.Beam(torch.tensor(c, dtype=torch.float64, device=DEV), sp, charge)


def _np(beam):
    order = np.argsort(beam.ids.cpu().numpy())
    return beam.coords.cpu().numpy()[:, order]


@pytest.mark.parametrize("space_charge", [True, False])
def test_multipole_fodo_matches_oracle(bt, space_charge):
    lat = bg.fodo_multipole_lattice(3, periods=2)
    c0 = bg.gaussian6d(12_345, seed=31)
    trk = bt.Tracker(32)
    beam = _beam(bt, c0)
    trk.track(beam, _els(bt, lat), space_charge=space_charge)
    trk.sync()
    t = tr.Tracker(oracle_ref(SP), CHARGE, 32, space_charge=space_charge)
    want = t.track(c0, lat)
    assert coord_rel_err(_np(beam), want) < REL_TOL
    # the multipoles act: tracking without them differs
    lin = [e for e in lat if e.kind != ph.MULTIPOLE]
    t2 = tr.Tracker(oracle_ref(SP), CHARGE, 32, space_charge=space_charge)
    assert coord_rel_err(t2.track(c0, lin), want) > 1e-6
    if space_charge:
        assert trk.regrid_log() == t.regrid_log


def test_split_calls_at_multipole_boundaries(bt):
    lat = bg.fodo_multipole_lattice(2)
    K = len(ph.slice_schedule(lat))
    c0 = bg.gaussian6d(3000, seed=32)
    trk = bt.Tracker(16)
    beam = _beam(bt, c0)
    els = _els(bt, lat)
    # splits at the boundaries before QF (slice 2), at the cell centre (slice
    # 6) and inside QD (slice 7)
    for a, b in ((0, 2), (2, 6), (6, 7), (7, K)):
        trk.track(beam, els, a, b - a)
    trk.sync()
    t = tr.Tracker(oracle_ref(SP), CHARGE, 16)
    want = t.track(c0, lat)
    assert coord_rel_err(_np(beam), want) < REL_TOL


def test_multipole_only_lattice_ends(bt):
    # a single thick element with multipoles on both sides and several at one
    # point, space charge off (the maps-only kernel) and on
    lat = [bg.multipole(3, 30.0, -10.0), bg.multipole(2, 0.02), bg.drift(0.6, 3),
           bg.multipole(4, 5e4), bg.multipole(1, 1e-5, -2e-5), bg.multipole(7, 0.0, 3e15)]
    c0 = bg.gaussian6d(2000, seed=33)
    for sc in (False, True):
        trk = bt.Tracker(16)
        beam = _beam(bt, c0)
        trk.track(beam, _els(bt, lat), space_charge=sc)
        trk.sync()
        want = tr.Tracker(oracle_ref(SP), CHARGE, 16, space_charge=sc).track(c0, lat)
        assert coord_rel_err(_np(beam), want) < REL_TOL


def test_batch_problem_with_multipoles(bt):
    lat = bg.fodo_multipole_lattice(2)
    c0 = bg.gaussian6d(4000, seed=34)
    c1 = bg.gaussian6d(2500, seed=35)
    trks = [bt.Tracker(16), bt.Tracker(32)]
    beams = [_beam(bt, c0), _beam(bt, c1)]
    b = bt.Batch(trks, beams, [_els(bt, lat), _els(bt, bg.fodo_lattice(1, 2))])
    b.launch()
    torch.cuda.synchronize()
    want = tr.Tracker(oracle_ref(SP), CHARGE, 16).track(c0, lat)
    assert coord_rel_err(_np(beams[0]), want) < REL_TOL
    want1 = tr.Tracker(oracle_ref(SP), CHARGE, 32).track(c1, bg.fodo_lattice(1, 2))
    assert coord_rel_err(_np(beams[1]), want1) < REL_TOL
    b.close()


def test_multipole_refusals(bt):
    from paper_2208_02382_b300 import _lib as L
    lat = bg.fodo_multipole_lattice(1)
    c0 = bg.gaussian6d(500, seed=36)
    trk = bt.Tracker(16)
    with pytest.raises(L.BeamtrackError):
        trk.track(_beam(bt, c0), _els(bt, lat), diagnostics=True)
    with pytest.raises(L.BeamtrackError):
        trk.grad_forward(_beam(bt, c0), _els(bt, lat))
    for order in (0, 13):
        bad = [bg.drift(0.5, 1), bt.Element(L.BX_MULTIPOLE, 0.0, 1.0, 0.0, 0, 0.0, order)]
        with pytest.raises(L.BeamtrackError):
            trk.track(_beam(bt, c0), bad)
    with pytest.raises(L.BeamtrackError):   # thin: nslice must be 0
        trk.track(_beam(bt, c0), [bg.drift(0.5, 1), bt.Element(L.BX_MULTIPOLE, 0.0, 1.0, 0.0, 1, 0.0, 3)])


def test_blown_up_bunch_reports_nonfinite(bt):
    # strong high-order multipoles drive the tails of the bunch to 1e150 and
    # then to Inf/NaN (the oracle does the same): the call ends with
    # BX_NONFINITE, the degenerate boxes on the way build no Green's function
    # from non-finite cell sizes, and the context tracks normally afterwards
    from paper_2208_02382_b300 import _lib as L
    m = bg.multipole
    lat = []
    for _ in range(2):
        lat += [m(2, 0.0, 0.01), bg.drift(0.25, 3), m(3, 20.0), bg.quad(1.0, 1.0, 3), m(3, 20.0),
                bg.drift(0.5, 3), m(4, -6e4, 1e4), m(5, 2.4e8), bg.quad(1.0, -1.0, 3),
                m(3, -15.0, 8.0), bg.drift(0.25, 3), m(6, 0.0, 1.2e12)]
    c0 = bg.gaussian6d(12_345, seed=31)
    for sc in (True, False):
        trk = bt.Tracker(32)
        beam = _beam(bt, c0)
        with pytest.raises(L.BeamtrackError) as err:
            trk.track(beam, _els(bt, lat), space_charge=sc)
            trk.sync()
        assert err.value.code == L.BX_NONFINITE
        trk.reset()
        tame = bg.fodo_multipole_lattice(2)
        beam = _beam(bt, c0)
        trk.track(beam, _els(bt, tame), space_charge=sc)
        trk.sync()
        want = tr.Tracker(oracle_ref(SP), CHARGE, 32, space_charge=sc).track(c0, tame)
        assert coord_rel_err(_np(beam), want) < REL_TOL
