"""GPU parity at the configuration the throughput is quoted on: the chicane
workload chicane_25e6_128 (500 MeV electrons, gamma ~ 979.5, so rest-frame
cells of aspect ~1:1000; 1 nC; quadrupoles then four sector bends) on its full
128^3 grid (256^3 doubled), against the FP64 oracle.

* Particle subsamples tracked from a fresh state: from the lattice start (the
  first box and Green's function build included), across the
  quadrupole -> sector-bend and sector-bend -> drift boundaries (merged maps
  with dispersion and path-length terms) and through the end of the lattice,
  with re-binning inside the window.  Coordinates to
  1e-11 relative, identical regrid logs.
* The Green's function table at N = 128 for the cell sizes of this workload's
  boxes against the float128 oracle, every one of the 129^3 entries.
* The full 2.5e7-particle bunch in the launch configuration the benchmark
  times (re-binning every 64 kicks with 8-cell bins, the autotuner's choice
  there): one kick from a fresh state through the CUDA-graph path, checked on
  a sample of particles that the oracle follows one by one through the same
  kick (the oracle deposits the whole bunch, solves, and gathers and kicks the
  sample); then properties that hold at any size over further kicks (bitwise
  reproducibility, identical particle order)."""
import numpy as np
import pytest
import torch

import beamgen as bg
from oracle import physics as ph
from oracle import spacecharge as sc
from oracle import track as tr
from tests.parity import REL_TOL, coord_rel_err, oracle_ref

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
W = bg.workload("chicane_25e6_128")


@pytest.fixture(scope="module")
def bt():
    import paper_2208_02382_b300 as p
    from paper_2208_02382_b300 import build
    build.build()
    return p


def gpu_beam(bt, coords):
    sp = W.species
    t = torch.tensor(np.ascontiguousarray(coords), dtype=torch.float64, device=DEV)
    return bt.Beam(t, bt.Species(sp.mass_MeV, sp.kinetic_MeV, sp.charge_sign), W.bunch_charge_C)


def by_id(beam):
    torch.cuda.synchronize()
    ids = beam.ids.cpu().numpy()
    assert np.array_equal(np.sort(ids), np.arange(len(ids)))
    return beam.coords.cpu().numpy()[:, np.argsort(ids)]


@pytest.mark.parametrize("npart,first,nk,rebin", [
    (300_001, 0, 8, 16),     # lattice start: first box, Green's function at 128^3
    (200_003, 97, 6, 4),     # kicks 97..102: Q2 -> B1 boundary at kick 100
    (150_001, 145, 10, 4),   # kicks 145..154: end of B1, into the drift after it
    (100_003, 490, 10, 4),   # the last ten kicks: the final half map ends the lattice
])
def test_chicane_128_subsample_tracking_matches_oracle(bt, npart, first, nk, rebin):
    c = W.particles(npart)
    ref = oracle_ref(W.species)
    otr = tr.Tracker(ref, W.bunch_charge_C, W.n_grid)
    want = otr.track(c, W.lattice, first, nk)
    beam = gpu_beam(bt, c)
    trk = bt.Tracker(W.n_grid)
    trk.set_binning(rebin, 8)
    trk.track(beam, W.lattice, first, nk)
    trk.sync()
    got = by_id(beam)
    assert trk.regrid_log() == otr.regrid_log    # kick counts since creation, both sides
    assert coord_rel_err(got, want) <= REL_TOL
    # the rest-frame cells really are the extreme aspect of this workload
    h = otr.box.h(W.n_grid)
    assert h[2] / h[0] > 500.0


def _box_h(npart):
    pos = sc.rest_frame(W.particles(npart), oracle_ref(W.species))
    box, _ = sc.box_rule(pos, None)
    return box.h(W.n_grid)


@pytest.mark.parametrize("npart", [300_001, 25_000_000])
def test_green_table_128_at_chicane_cells_matches_float128_oracle(bt, npart):
    """129^3 offsets up to 128 cells at the first box's cell size of the
    300 001-particle subsample and of the full bunch (aspect ~1:1000): every
    far-field series order and the near-cell double-double corners."""
    h = _box_h(npart)
    n = W.n_grid
    trk = bt.Tracker(n)
    g = trk.green_table(h, DEV).cpu().numpy().reshape(n + 1, n + 1, n + 1)
    want = sc.igf_octant(n, h)
    rel = np.abs(g - want) / np.abs(want)
    assert rel.max() <= 4e-16, (h, float(rel.max()), np.unravel_index(rel.argmax(), rel.shape))


def _oracle_one_kick_sample(c, sample):
    """The oracle's first kick of the chicane on the whole bunch c, followed
    for the particles `sample` only: half map of the first slice (all
    particles, cheap), box rule and deposit of the whole bunch, solve and
    field, then gather + kick + half map for the sample."""
    ref = oracle_ref(W.species)
    sched = ph.slice_schedule(W.lattice)
    ie, ds = sched[0]
    e = W.lattice[ie]
    half = ph.element_matrix(e.kind, e.length, e.k, e.angle, 0.5 * ds, ref)
    c1 = ph.push(c, half)
    pos = sc.rest_frame(c1, ref)
    box, _ = sc.box_rule(pos, None)
    h = box.h(W.n_grid)
    rho = sc.deposit(pos, sc.macro_charge(W.bunch_charge_C, c.shape[1], ref), box, W.n_grid)
    del pos
    phi = sc.solve(rho, h)
    ef = sc.field(phi, h)
    cs = c1[:, sample]
    e_at = sc.gather(sc.rest_frame(cs, ref), ef, box)
    return ph.push(sc.kick(cs, e_at, ds, ref), half)


def test_chicane_full_bunch_first_kick_matches_oracle_on_a_sample(bt):
    c = W.particles()
    rng = np.random.default_rng(12345)
    sample = np.sort(rng.choice(c.shape[1], size=20_000, replace=False))
    want = _oracle_one_kick_sample(c, sample)
    beam = gpu_beam(bt, c)
    del c
    trk = bt.Tracker(W.n_grid)
    trk.set_binning(64, 8)       # kick 0 re-bins: the sort is inside this kick
    trk.track(beam, W.lattice, 0, 1)
    trk.sync()
    ids = beam.ids.cpu().numpy()
    inv = np.empty_like(ids)
    inv[ids] = np.arange(len(ids))
    got = beam.coords[:, torch.tensor(inv[sample], device=DEV)].cpu().numpy()
    assert trk.regrid_log() == [0]
    # relative to max(|value|, rms of the sample's row)
    assert coord_rel_err(got, want) <= REL_TOL


def test_chicane_full_bunch_is_bitwise_reproducible_over_kicks(bt):
    """Twelve kicks of the 2.5e7-particle bunch in two calls (the second call
    starts from the box kept by the first), twice: identical particle order and
    identical bits."""
    c = torch.tensor(W.particles(), dtype=torch.float64, device=DEV)
    sp = bt.Species(W.species.mass_MeV, W.species.kinetic_MeV, W.species.charge_sign)
    outs = []
    for _ in range(2):
        beam = bt.Beam(c.clone(), sp, W.bunch_charge_C)
        trk = bt.Tracker(W.n_grid)
        trk.set_binning(64, 8)
        trk.track(beam, W.lattice, 0, 5)
        trk.track(beam, W.lattice, 5, 7)
        trk.sync()
        torch.cuda.synchronize()
        outs.append((beam.coords.clone(), beam.ids.clone(), trk.regrid_log()))
        trk.close()
        del beam
    assert torch.equal(outs[0][1], outs[1][1])
    assert torch.equal(outs[0][0], outs[1][0])
    assert outs[0][2] == outs[1][2]
