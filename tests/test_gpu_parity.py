"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: relative 1e-11 on phase-space coordinates (metric of
tests/parity.py: per particle, relative to max(|value|, rms of the row)) and
on grids (relative to the grid's max).  Inputs are the seeded synthetic bunches
of beamgen; sizes span several FFT/cell tiles with ragged particle counts."""
import numpy as np
import pytest
import torch

import beamgen as bg
from oracle import physics as ph
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


def gpu_beam(bt, coords, species, charge):
    t = torch.tensor(np.ascontiguousarray(coords), dtype=torch.float64, device=DEV)
    return bt.Beam(t, bt.Species(species.mass_MeV, species.kinetic_MeV, species.charge_sign),
                   charge)


def to_np(beam):
    """Coordinates in id order (the tracking may re-bin particles)."""
    torch.cuda.synchronize()
    ids = beam.ids.cpu().numpy()
    assert np.array_equal(np.sort(ids), np.arange(len(ids)))
    return beam.coords.cpu().numpy()[:, np.argsort(ids)]


# ------------------------------------------------------------- Green's function

@pytest.mark.parametrize("n,h", [(8, (1e-3, 1e-3, 1e-3)), (16, (1e-3, 2.5e-3, 7e-3)),
                                 (32, (2e-4, 2e-4, 0.2))])
def test_green_table_matches_float128_oracle(bt, n, h):
    trk = bt.Tracker(n)
    g = trk.green_table(h, DEV).cpu().numpy().reshape(n + 1, n + 1, n + 1)
    ref = sc.igf_octant(n, h)
    rel = np.abs(g - ref) / np.abs(ref)
    assert rel.max() <= 4e-16


# ------------------------------------------------------------------- deposit

@pytest.mark.parametrize("npart,n", [(1, 8), (333, 8), (10_000, 32), (100_003, 64)])
def test_deposit_matches_oracle(bt, npart, n):
    c = bg.gaussian6d(npart, seed=npart)
    sp = bg.PROTON_2GEV
    beam = gpu_beam(bt, c, sp, 1e-9)
    trk = bt.Tracker(n)
    grid = trk.deposit(beam, bt.Grid(n, DEV))
    trk.sync()
    ref = oracle_ref(sp)
    pos = sc.rest_frame(c, ref)
    box, _ = sc.box_rule(pos, None)
    assert tuple(grid.lo) == box.lo and tuple(grid.hi) == box.hi
    rho_ref = sc.deposit(pos, sc.macro_charge(1e-9, npart, ref), box, n)
    rho = grid.rho.cpu().numpy().reshape(n, n, n)
    assert grid_rel_err(rho, rho_ref) <= 1e-13


def test_deposit_is_bitwise_reproducible(bt):
    c = bg.gaussian6d(200_000, seed=5)
    beam = gpu_beam(bt, c, bg.PROTON_1GEV, 1e-9)
    trk = bt.Tracker(32)
    a = trk.deposit(beam, bt.Grid(32, DEV)).rho.clone()
    b = trk.deposit(beam, bt.Grid(32, DEV, lo=trk.box()[0], hi=trk.box()[1])).rho.clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)


# --------------------------------------------------------------------- solve

@pytest.mark.parametrize("n,h", [(8, (1e-3, 1.5e-3, 2.5e-3)), (32, (1e-4, 1e-4, 3e-4)),
                                 (64, (5e-5, 6e-5, 2e-3))])
def test_solve_matches_oracle(bt, n, h):
    rng = np.random.default_rng(n)
    rho = rng.random((n, n, n)) * 1e-3
    trk = bt.Tracker(n)
    grid = bt.Grid(n, DEV)
    grid.rho.copy_(torch.tensor(rho.ravel(), device=DEV))
    grid.h = list(h)
    trk.solve(grid)
    phi = grid.phi.cpu().numpy().reshape(n + 2, n + 2, n + 2)
    ref = sc.solve(rho, h)
    assert grid_rel_err(phi, ref) <= REL_TOL


@pytest.mark.parametrize("n", [128, 256])
def test_solve_of_point_charge_is_the_green_function(bt, n):
    """On the grids the oracle tests do not reach (256- and 512-point lines):
    the solve of a unit charge density at one node j gives phi(i) = G(i - j)
    at every node -1..n (offsets up to n, the doubled grid's +-n entries
    included), G the context's own integrated Green's function table; this
    checks the FFT passes' staging, pruning and crop independently of the
    tracking solve, which is compared with this one below."""
    h = (1.0e-4, 1.3e-4, 2.1e-3)
    trk = bt.Tracker(n)
    g = trk.green_table(h, DEV).cpu().numpy().reshape(n + 1, n + 1, n + 1)   # [c][b][a]
    grid = bt.Grid(n, DEV)
    grid.h = list(h)
    j = (n // 3, n // 2 + 1, (2 * n) // 3)       # (x, y, z) node
    rho = torch.zeros(n ** 3, dtype=torch.float64, device=DEV)
    rho[(j[2] * n + j[1]) * n + j[0]] = 1.0
    grid.rho.copy_(rho)
    trk.solve(grid)
    phi = grid.phi.cpu().numpy().reshape(n + 2, n + 2, n + 2)                # [z][y][x], nodes -1..n
    idx = np.arange(-1, n + 1)
    ax = np.abs(idx - j[0])
    by = np.abs(idx - j[1])
    cz = np.abs(idx - j[2])
    want = g[cz[:, None, None], by[None, :, None], ax[None, None, :]]
    assert grid_rel_err(phi, want) <= 1e-12


@pytest.mark.parametrize("n", [32, 128, 256])
def test_tracking_solve_matches_fp64_solve(bt, n):
    """Tracking solves in block floating point (int64 values, one exponent per
    line transform); the explicit deposit -> solve -> gather+kick calls use
    the FP64 FFT.  One slice of a drift both ways (half map, kick, half map),
    also on the largest grids (256- and 512-point lines) that the oracle tests
    do not reach: the kicks agree to 1e-13 of their size (measured 4e-15 at
    32^3 to 3.5e-14 at 256^3)."""
    c = bg.gaussian6d(400_000, seed=n)
    sp = bg.PROTON_1GEV
    L_ = 0.2
    beam = gpu_beam(bt, c, sp, 1e-9)
    trk = bt.Tracker(n)
    trk.track(beam, [bg.drift(L_, 1)], 0, 1, True)
    trk.sync()
    got = to_np(beam)
    half = [bg.drift(0.5 * L_, 1)]
    beam2 = gpu_beam(bt, c, sp, 1e-9)
    t2 = bt.Tracker(n)
    t2.track(beam2, half, 0, 1, False)
    grid = t2.deposit(beam2, bt.Grid(n, DEV))
    t2.solve(grid)
    t2.gather_kick(beam2, grid, L_)
    t3 = bt.Tracker(n)
    t3.track(beam2, half, 0, 1, False)
    t3.sync()
    want = to_np(beam2)
    kick_err = max(grid_rel_err(got[r] - c[r], want[r] - c[r]) for r in (1, 3, 5))
    err = coord_rel_err(got, want)
    assert kick_err <= 1e-13, (kick_err, err)
    assert err <= 1e-13, (kick_err, err)


# ------------------------------------------------------------- gather + kick

def test_gather_kick_matches_oracle(bt):
    n, npart = 32, 20_000
    sp = bg.PROTON_1GEV
    ref = oracle_ref(sp)
    c = bg.gaussian6d(npart, seed=3)
    pos = sc.rest_frame(c, ref)
    box, _ = sc.box_rule(pos, None)
    h = box.h(n)
    rho = sc.deposit(pos, sc.macro_charge(1e-9, npart, ref), box, n)
    phi = sc.solve(rho, h)
    ds = 0.05
    want = sc.kick(c, sc.gather(pos, sc.field(phi, h), box), ds, ref)
    beam = gpu_beam(bt, c, sp, 1e-9)
    trk = bt.Tracker(n)
    grid = bt.Grid(n, DEV, lo=box.lo, hi=box.hi)
    grid.h = list(h)
    grid.phi.copy_(torch.tensor(phi.ravel(), device=DEV))
    trk.gather_kick(beam, grid, ds)
    got = to_np(beam)
    assert coord_rel_err(got, want) <= 1e-14
    # the kick itself (the change of momenta) to the same tolerance as the grids
    for r in (1, 3, 5):
        assert grid_rel_err(got[r] - c[r], want[r] - c[r]) <= 1e-12


# ------------------------------------------------------------------- moments

def test_moments_match_oracle(bt):
    c = bg.gaussian_with_halo(123_457, seed=2)
    beam = gpu_beam(bt, c, bg.PROTON_1GEV, 1e-9)
    trk = bt.Tracker(8)
    m = trk.moments(beam).cpu().numpy()
    ref = tr.moments_vector(c)
    assert np.abs(m - ref).max() <= 1e-12 * np.abs(ref).max()
    m2 = trk.moments(beam).cpu().numpy()
    assert np.array_equal(m, m2)


# ------------------------------------------------------------------ tracking

def _track_both(bt, coords, species, charge, lattice, n, space_charge=True, first=0, nk=None):
    ref = oracle_ref(species)
    otr = tr.Tracker(ref, charge, n, space_charge=space_charge)
    want = otr.track(coords, lattice, first, nk)
    beam = gpu_beam(bt, coords, species, charge)
    trk = bt.Tracker(n)
    trk.track(beam, lattice, first, -1 if nk is None else nk, space_charge)
    trk.sync()
    return to_np(beam), want, trk, otr


@pytest.mark.parametrize("lat", ["fodo", "chicane"])
def test_track_without_space_charge(bt, lat):
    lattice = bg.fodo_lattice(3, 4) if lat == "fodo" else bg.chicane_lattice(5)
    sp = bg.PROTON_2GEV if lat == "fodo" else bg.ELECTRON_500MEV
    c = bg.gaussian6d(5_001, seed=7)
    got, want, _, _ = _track_both(bt, c, sp, 1e-9, lattice, 8, space_charge=False)
    assert coord_rel_err(got, want) <= 1e-13


def test_track_small_workload_full_run(bt):
    """fodo_1e4_32: 1e4 particles, 2 GeV p, FODO x10, 250 kicks, 32^3, 1 nC."""
    w = bg.workload("fodo_1e4_32")
    c = w.particles()
    got, want, trk, otr = _track_both(bt, c, w.species, w.bunch_charge_C, w.lattice, w.n_grid)
    assert trk.regrid_log() == otr.regrid_log
    assert coord_rel_err(got, want) <= REL_TOL


def test_track_chicane_electrons_ragged(bt):
    c = bg.gaussian6d(7_777, seed=11)
    lattice = bg.chicane_lattice(3)
    got, want, trk, otr = _track_both(bt, c, bg.ELECTRON_500MEV, 1e-9, lattice, 16)
    assert trk.regrid_log() == otr.regrid_log
    assert coord_rel_err(got, want) <= REL_TOL


def test_track_in_pieces_equals_one_call(bt):
    w = bg.workload("fodo_1e4_32")
    c = w.particles(4_000)
    sp = bt.Species(w.species.mass_MeV, w.species.kinetic_MeV, w.species.charge_sign)
    a = bt.Beam(torch.tensor(c, device=DEV), sp, 1e-9)
    b = bt.Beam(torch.tensor(c, device=DEV), sp, 1e-9)
    t1, t2 = bt.Tracker(16), bt.Tracker(16)
    t1.track(a, w.lattice, 0, 30)
    t2.track(b, w.lattice, 0, 12)
    t2.track(b, w.lattice, 12, 18)
    torch.cuda.synchronize()
    # merged half-maps across the call boundary round differently: compare to 1e-13
    assert coord_rel_err(to_np(a), to_np(b)) <= 1e-13
    assert t1.regrid_log() == t2.regrid_log()


def test_track_one_kick_per_call_matches_oracle(bt):
    # every call after the first deposits its first kick in the prologue, into
    # the box kept from the call before (the box rule re-deposits on a regrid);
    # re-binning runs on the context's kick count across the calls
    w = bg.workload("fodo_1e4_32")
    c = w.particles(3_000)
    sp = bt.Species(w.species.mass_MeV, w.species.kinetic_MeV, w.species.charge_sign)
    beam = bt.Beam(torch.tensor(c, device=DEV), sp, w.bunch_charge_C)
    trk = bt.Tracker(16)
    trk.set_binning(4, 0)
    nk = 24
    for k in range(nk):
        trk.track(beam, w.lattice, k, 1)
    trk.sync()
    ref = oracle_ref(w.species)
    otr = tr.Tracker(ref, w.bunch_charge_C, 16)
    want = otr.track(c, w.lattice, 0, nk)
    assert coord_rel_err(to_np(beam), want) <= REL_TOL
    assert trk.regrid_log() == otr.regrid_log


@pytest.mark.parametrize("npart", [0, 1, 2, 3])
def test_track_degenerate_bunches(bt, npart):
    """Empty bunch, a single particle (all extents zero, floored box) and
    two/three particles.  A lone macroparticle sits at the centre of its box,
    so its CIC self-field vanishes in exact arithmetic; at 1 nC in a 1e-6 m
    box the rounding-level asymmetry is amplified by fields of ~1e14 V/m, so
    the bitwise-sensitive comparison uses a femtocoulomb bunch and the 1 nC
    run checks finiteness and the regrid log."""
    c = bg.gaussian6d(npart, seed=1)
    lattice = bg.fodo_lattice(1, 2)
    got, want, trk, otr = _track_both(bt, c, bg.PROTON_2GEV, 1e-15, lattice, 8)
    assert got.shape == want.shape
    if npart:
        assert np.all(np.isfinite(got))
        assert coord_rel_err(got, want) <= REL_TOL
        assert trk.regrid_log() == otr.regrid_log
        got, want, trk, otr = _track_both(bt, c, bg.PROTON_2GEV, 1e-9, lattice, 8)
        assert np.all(np.isfinite(got))
        assert trk.regrid_log() == otr.regrid_log


def test_one_context_tracks_beams_of_different_sizes(bt):
    """A context keeps per-particle scratch (the deposit's cell codes, the
    binning buffers) and a captured kick graph; a smaller and then a larger
    bunch through the same context reuse or reallocate them, and each call
    matches the oracle."""
    w = bg.workload("fodo_1e4_32")
    trk = bt.Tracker(16)
    for npart, seed in ((6_000, 11), (2_500, 12), (9_001, 13)):
        c = bg.gaussian6d(npart, seed=seed)
        beam = gpu_beam(bt, c, w.species, w.bunch_charge_C)
        trk.reset()
        trk.track(beam, w.lattice, 0, 30)
        trk.sync()
        otr = tr.Tracker(oracle_ref(w.species), w.bunch_charge_C, 16)
        want = otr.track(c, w.lattice, 0, 30)
        assert coord_rel_err(to_np(beam), want) <= REL_TOL
        assert trk.regrid_log() == otr.regrid_log


def test_track_is_bitwise_reproducible(bt):
    w = bg.workload("fodo_1e4_32")
    c = w.particles()
    outs = []
    for _ in range(3):
        beam = gpu_beam(bt, c, w.species, w.bunch_charge_C)
        trk = bt.Tracker(w.n_grid)
        trk.track(beam, w.lattice, 0, 40)
        torch.cuda.synchronize()
        outs.append((beam.coords.cpu().numpy(), beam.ids.cpu().numpy()))
    for k in (1, 2):  # same particle order and bitwise the same coordinates
        assert np.array_equal(outs[0][1], outs[k][1])
        assert np.array_equal(outs[0][0], outs[k][0])


def test_track_reports_nonfinite(bt):
    c = bg.gaussian6d(1000, seed=1)
    c[3, 17] = np.inf
    beam = gpu_beam(bt, c, bg.PROTON_2GEV, 1e-9)
    trk = bt.Tracker(8)
    from paper_2208_02382_b300 import _lib as L
    with pytest.raises(L.BeamtrackError) as e:
        trk.track(beam, bg.fodo_lattice(1, 1), 0, 2)
        trk.sync()
    assert e.value.code == L.BX_NONFINITE


def test_track_medium_workload_first_kicks(bt):
    """fodo_1e6_64 at full size (1e6 particles with halo, 64^3), first 6 kicks."""
    w = bg.workload("fodo_1e6_64")
    c = w.particles()
    got, want, trk, otr = _track_both(bt, c, w.species, w.bunch_charge_C, w.lattice, w.n_grid,
                                      nk=6)
    assert trk.regrid_log() == otr.regrid_log
    assert coord_rel_err(got, want) <= REL_TOL


def test_graph_and_plain_launch_paths_agree_bitwise(bt):
    """bx_track replays one CUDA graph per kick (conditional nodes for the
    Green's function rebuild, re-binning and re-deposit); with kernel timing
    on it launches the same kernels one by one.  Both give identical bits."""
    w = bg.workload("fodo_1e4_32")
    c = w.particles(6_000)
    outs = []
    for timing in (False, True):
        beam = gpu_beam(bt, c, w.species, w.bunch_charge_C)
        trk = bt.Tracker(16)
        if timing:
            trk.profile(True)
        trk.track(beam, w.lattice, 0, 45)
        trk.track(beam, w.lattice, 45, 20)
        trk.sync()
        torch.cuda.synchronize()
        outs.append((beam.coords.cpu().numpy(), beam.ids.cpu().numpy(), trk.regrid_log()))
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][2] == outs[1][2] and len(outs[0][2]) > 3


@pytest.mark.parametrize("workload,npart,n,nk,be", [("fodo_1e4_32", 9_001, 16, 40, 4),
                                                    ("fodo_1e6_64", 200_003, 64, 12, 8),
                                                    ("chicane_25e6_128", 150_001, 128, 10, 8)])
def test_cell_order_binning_is_bitwise_the_bin_order_one(bt, workload, npart, n, nk, be):
    """Re-binning by cell within bin (a second counting-sort pass; the tile
    deposit spreads its atomics over the block's particles) against re-binning
    by bin: the same integer charge, so bitwise the same coordinates and regrid
    log, re-binning every 4 kicks (each sort inside the window)."""
    w = bg.workload(workload)
    c = w.particles(npart)
    outs = []
    for co in (0, 1):
        beam = gpu_beam(bt, c, w.species, w.bunch_charge_C)
        trk = bt.Tracker(n, rebin_interval=4, bin_edge=be, cell_order=co)
        trk.track(beam, w.lattice, 0, nk)
        trk.sync()
        outs.append((to_np(beam), trk.regrid_log()))
        trk.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]
    otr = tr.Tracker(oracle_ref(w.species), w.bunch_charge_C, n)
    assert coord_rel_err(outs[1][0], otr.track(c, w.lattice, 0, nk)) <= REL_TOL


def test_track_medium_workload_long_run_subsample(bt):
    """fodo_1e6_64's bunch shape (80% Gaussian, 20% uniform-ellipsoid halo), 1 GeV
    protons, 10 nC, 64^3 grid: a 20 000-particle subsample through the first
    200 of its 1000 kicks from a fresh state (the box rule regrids on about half
    of them), against the oracle: identical regrid logs and coordinates to 1e-11
    after the growth of any rounding difference over 200 space-charge kicks."""
    w = bg.workload("fodo_1e6_64")
    c = w.particles(20_000)
    got, want, trk, otr = _track_both(bt, c, w.species, w.bunch_charge_C, w.lattice, w.n_grid,
                                      nk=200)
    assert trk.regrid_log() == otr.regrid_log and len(otr.regrid_log) > 50
    assert coord_rel_err(got, want) <= REL_TOL
