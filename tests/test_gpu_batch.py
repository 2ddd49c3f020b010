"""Batches of independent tracking problems (bx_batch_* through the C ABI):
one graph launch must give, bit for bit, what reset + bx_track gives for each
problem on its own, for ragged particle counts, mixed grid sizes, lattice
variants and a problem without space charge; one problem is also checked
against the oracle (relative 1e-11)."""
import numpy as np
import pytest
import torch

import beamgen as bg
from oracle import track as tr
from tests.parity import REL_TOL, coord_rel_err, oracle_ref

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SPECIES = bg.PROTON_1GEV
CHARGE = 10e-9


@pytest.fixture(scope="module")
def bt():
    import paper_2208_02382_b300 as p
    from paper_2208_02382_b300 import build
    build.build()
    return p


def _problems(bt):
    specs = [(1000, 16, 1.1, -0.9), (3001, 32, 0.85, -1.15), (777, 16, 1.0, -1.0),
             (20_000, 32, 1.2, -0.8), (1, 16, 1.0, -1.0), (5000, 16, 0.95, -1.05)]
    sp = bt.Species(SPECIES.mass_MeV, SPECIES.kinetic_MeV, SPECIES.charge_sign)
    out = []
    for i, (n, grid, kf, kd) in enumerate(specs):
        lat = bg.fodo_lattice(2, 2, kf, kd)
        c = bg.gaussian6d(n, seed=50 + i)
        out.append((n, grid, lat, c, i == 5))
    return sp, out


def _beam(bt, sp, c):
    return bt.Beam(torch.tensor(c, dtype=torch.float64, device=DEV), sp, CHARGE)


def _in_id_order(beam):
    ids = beam.ids.cpu().numpy()
    return beam.coords.cpu().numpy()[:, np.argsort(ids)]


def test_batch_equals_sequential_tracking_bitwise(bt):
    sp, probs = _problems(bt)
    # sequential reference: reset + track per problem, twice (two lattice passes)
    seq = []
    for n, grid, lat, c, no_sc in probs:
        trk = bt.Tracker(grid)
        beam = _beam(bt, sp, c)
        logs = []
        for rep in range(2):
            trk.reset()
            trk.track(beam, lat, 0, -1, space_charge=not no_sc)
            trk.sync()
            logs.append(trk.regrid_log())
        seq.append((_in_id_order(beam), logs))
        trk.close()
    # batch: one graph launch per lattice pass
    trks = [bt.Tracker(g) for _, g, _, _, _ in probs]
    beams = [_beam(bt, sp, c) for _, _, _, c, _ in probs]
    lats = [lat for _, _, lat, _, _ in probs]
    # the problem without space charge goes into a batch of its own (the space-
    # charge switch is per lattice list)
    idx_sc = [i for i, p in enumerate(probs) if not p[4]]
    idx_ns = [i for i, p in enumerate(probs) if p[4]]
    b1 = bt.Batch([trks[i] for i in idx_sc], [beams[i] for i in idx_sc], [lats[i] for i in idx_sc])
    b2 = bt.Batch([trks[i] for i in idx_ns], [beams[i] for i in idx_ns], [lats[i] for i in idx_ns],
                  space_charge=False)
    for rep in range(2):
        b1.launch()
        b2.launch()
        torch.cuda.synchronize()
        for i in idx_sc:
            trks[i].sync()
    for i, (ref, logs) in enumerate(seq):
        got = _in_id_order(beams[i])
        assert np.array_equal(got, ref), i
        if i in idx_sc:
            assert trks[i].regrid_log() == logs[1], i
    b1.close()
    b2.close()


def test_batch_problem_matches_oracle(bt):
    sp, probs = _problems(bt)
    n, grid, lat, c, _ = probs[1]
    trks = [bt.Tracker(probs[k][1]) for k in (0, 1)]
    beams = [_beam(bt, sp, probs[k][3]) for k in (0, 1)]
    b = bt.Batch(trks, beams, [probs[0][2], lat])
    b.launch()
    torch.cuda.synchronize()
    got = _in_id_order(beams[1])
    t = tr.Tracker(oracle_ref(SPECIES), CHARGE, grid)
    want = t.track(c, lat)
    assert coord_rel_err(got, want) < REL_TOL
    assert trks[1].regrid_log() == t.regrid_log
    b.close()


def test_batch_rejects_bad_arguments(bt):
    sp, probs = _problems(bt)
    trk = bt.Tracker(16)
    beam = _beam(bt, sp, probs[0][3])
    with pytest.raises(Exception):
        bt.Batch([trk, trk], [beam, beam], [probs[0][2], probs[0][2]])
    with pytest.raises(Exception):
        bt.Batch([], [], [])


def test_binning_autotuner_keeps_results_and_beam(bt):
    sp, probs = _problems(bt)
    n, grid, lat, c, _ = probs[3]            # 20000 particles, 32^3
    trk = bt.Tracker(grid)
    beam = _beam(bt, sp, c)
    before = beam.coords.clone()
    ids_before = beam.ids.clone()
    (iv, be, co), ms = trk.autotune_binning(beam, lat, kicks=12)
    assert torch.equal(beam.coords, before) and torch.equal(beam.ids, ids_before)
    assert len(ms) >= 2 and all(v > 0 for v in ms)
    assert iv in (-1, 8, 32) and (iv == -1 or be in (4, 8, 16)) and co in (0, 1)
    trk.track(beam, lat)
    trk.sync()
    ref = bt.Tracker(grid)
    b2 = _beam(bt, sp, c)
    ref.track(b2, lat)
    ref.sync()
    # binning changes particle order, never the physics
    assert np.array_equal(_in_id_order(beam), _in_id_order(b2))
    assert trk.regrid_log() == ref.regrid_log()


def test_binning_options_validated(bt):
    with pytest.raises(Exception):
        bt.Tracker(32, bin_edge=3)
    with pytest.raises(Exception):
        bt.Tracker(32, rebin_interval=-2)
    with pytest.raises(Exception):
        bt.Tracker(32, cell_order=2)
    t = bt.Tracker(64, rebin_interval=-1, bin_edge=4)
    with pytest.raises(Exception):
        t.set_binning(8, 64)
    with pytest.raises(Exception):
        t.set_binning(8, 8, -1)
