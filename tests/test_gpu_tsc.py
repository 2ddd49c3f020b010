"""TSC particle shape (Listing 1 set_particle_shape(2)) on the GPU through the
C ABI against the oracle: deposit (including grids small enough for the edge
limit to act), gather + kick, whole-lattice tracking with regrids, batches;
the reverse mode refuses shape 2."""
import numpy as np
import pytest
import torch

import beamgen as bg
from oracle import spacecharge as sc
from oracle import track as tr
from tests.parity import REL_TOL, coord_rel_err, grid_rel_err, oracle_ref

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def bt():
    import paper_2208_02382_b300 as p
    from paper_2208_02382_b300 import build
    build.build()
    return p


def _beam(bt, c, species, charge):
    sp = bt.Species(species.mass_MeV, species.kinetic_MeV, species.charge_sign)
    return bt.Beam(torch.tensor(np.ascontiguousarray(c), dtype=torch.float64, device=DEV), sp,
                   charge)


def _np(beam):
    torch.cuda.synchronize()
    order = np.argsort(beam.ids.cpu().numpy())
    return beam.coords.cpu().numpy()[:, order]


@pytest.mark.parametrize("npart,n", [(1, 8), (777, 8), (20_001, 32), (100_003, 64)])
def test_tsc_deposit_matches_oracle(bt, npart, n):
    c = bg.gaussian6d(npart, seed=npart + 1)
    sp = bg.PROTON_2GEV
    trk = bt.Tracker(n, shape_order=2)
    grid = trk.deposit(_beam(bt, c, sp, 1e-9), bt.Grid(n, DEV))
    trk.sync()
    ref = oracle_ref(sp)
    pos = sc.rest_frame(c, ref)
    box, _ = sc.box_rule(pos, None)
    want = sc.deposit(pos, sc.macro_charge(1e-9, npart, ref), box, n, shape=2)
    got = grid.rho.cpu().numpy().reshape(n, n, n)
    assert grid_rel_err(got, want) <= 1e-13
    h = box.h(n)
    assert got.sum() * h[0] * h[1] * h[2] == pytest.approx(1e-9, rel=1e-13)


def test_tsc_gather_kick_matches_oracle(bt):
    n, npart = 32, 20_000
    sp = bg.PROTON_1GEV
    ref = oracle_ref(sp)
    c = bg.gaussian6d(npart, seed=4)
    pos = sc.rest_frame(c, ref)
    box, _ = sc.box_rule(pos, None)
    h = box.h(n)
    phi = sc.solve(sc.deposit(pos, sc.macro_charge(1e-9, npart, ref), box, n, 2), h)
    ds = 0.05
    want = sc.kick(c, sc.gather(pos, sc.field(phi, h), box, 2), ds, ref)
    beam = _beam(bt, c, sp, 1e-9)
    trk = bt.Tracker(n, shape_order=2)
    grid = bt.Grid(n, DEV, lo=box.lo, hi=box.hi)
    grid.h = list(h)
    grid.phi.copy_(torch.tensor(phi.ravel(), device=DEV))
    trk.gather_kick(beam, grid, ds)
    got = _np(beam)
    assert coord_rel_err(got, want) <= 1e-14
    for r in (1, 3, 5):
        assert grid_rel_err(got[r] - c[r], want[r] - c[r]) <= 1e-12


@pytest.mark.parametrize("n", [8, 32])
def test_tsc_tracking_matches_oracle(bt, n):
    w = bg.workload("fodo_1e4_32")
    lat = bg.fodo_lattice(4, 5)
    c0 = w.particles()
    beam = _beam(bt, c0, w.species, w.bunch_charge_C)
    trk = bt.Tracker(n, shape_order=2)
    trk.track(beam, lat)
    trk.sync()
    t = tr.Tracker(oracle_ref(w.species), w.bunch_charge_C, n, shape=2)
    want = t.track(c0, lat)
    assert trk.regrid_log() == t.regrid_log
    assert coord_rel_err(_np(beam), want) < REL_TOL
    # the shape matters: CIC gives a different result
    t1 = tr.Tracker(oracle_ref(w.species), w.bunch_charge_C, n, shape=1)
    assert coord_rel_err(t1.track(c0, lat), want) > 1e-6


def test_tsc_batch_equals_sequential_and_grad_refuses(bt):
    w = bg.workload("fodo_1e4_32")
    lat = bg.fodo_lattice(2, 4)
    c0 = w.particles(5000)
    ref_t = bt.Tracker(16, shape_order=2)
    b_ref = _beam(bt, c0, w.species, 1e-9)
    ref_t.track(b_ref, lat)
    trk = bt.Tracker(16, shape_order=2)
    b = _beam(bt, c0, w.species, 1e-9)
    batch = bt.Batch([trk], [b], [lat])
    batch.launch()
    assert np.array_equal(_np(b), _np(b_ref))
    batch.close()
    with pytest.raises(Exception):
        trk.grad_forward(_beam(bt, c0, w.species, 1e-9), lat, 4)
