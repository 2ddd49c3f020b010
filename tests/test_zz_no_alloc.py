"""GPU test of bx_deposit_noalloc, the deposition entry point for callers that
may not allocate device memory while running (fixed-footprint control-loop
models, hosts that own all device memory).  It shares the context deposit's
per-particle arithmetic, so it must give bitwise the same charge density as
bx_deposit with the same explicit box, call after call, although its
accumulators live in a static array that every call reuses; and both must
match the oracle's deposit.  Grids of 8^3, 32^3 and 64^3 nodes (64^3 fills the
whole static array); boxes that are the bunch's exact extent (extreme
particles on the box faces), and boxes that leave particles outside (skipped
and flagged, as the context deposit skips them).

This file sorts last so that a run stopping at the first failure has already
run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import beamgen as bg
from oracle import spacecharge as sc
from tests.parity import grid_rel_err, oracle_ref

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SP = bg.PROTON_1GEV


def _beam(bt, coords):
    t = torch.tensor(np.ascontiguousarray(coords), dtype=torch.float64, device=DEV)
    return bt.Beam(t, bt.Species(SP.mass_MeV, SP.kinetic_MeV, SP.charge_sign), 1e-9)


def _noalloc(lib, L, beam, lo, hi, n):
    out = torch.full((n ** 3,), np.nan, dtype=torch.float64, device=DEV)
    flags = torch.zeros(1, dtype=torch.int32, device=DEV)
    b = beam.c_struct()
    rc = lib.bx_deposit_noalloc(ctypes.byref(b), (ctypes.c_double * 3)(*lo),
                                (ctypes.c_double * 3)(*hi), n, ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(flags.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == L.BX_OK, lib.bx_last_error(None)
    torch.cuda.synchronize()
    return out, int(flags.item())


def _exact_box(coords):
    pos = sc.rest_frame(coords, oracle_ref(SP))
    return [float(v) for v in pos.min(axis=1)], [float(v) for v in pos.max(axis=1)]


@pytest.mark.parametrize("n", [8, 32, 64])
def test_noalloc_deposit_matches_context_deposit_and_oracle_on_consecutive_calls(n):
    import paper_2208_02382_b300 as bt
    from paper_2208_02382_b300 import _lib as L
    from paper_2208_02382_b300 import build
    build.build()
    lib = L.load()
    trk = bt.Tracker(n)
    ref = oracle_ref(SP)
    # two calls in a row, different bunches: the box-rule box, then the exact extent
    for seed, npart, exact in ((1, 100_003, False), (2, 54_321, True)):
        c = bg.gaussian6d(npart, seed=seed + n)
        beam = _beam(bt, c)
        if exact:
            lo, hi = _exact_box(c)
        else:
            g = trk.deposit(beam, bt.Grid(n, DEV))       # context path, box rule
            lo, hi = list(g.lo), list(g.hi)
        want = trk.deposit(beam, bt.Grid(n, DEV, lo=lo, hi=hi)).rho.clone()
        trk.sync()
        got, flags = _noalloc(lib, L, beam, lo, hi, n)
        assert flags == 0
        assert torch.equal(got, want)
        rho_ref = sc.deposit(sc.rest_frame(c, ref), sc.macro_charge(1e-9, npart, ref),
                             sc.Box(tuple(lo), tuple(hi)), n)
        assert grid_rel_err(got.cpu().numpy().reshape(n, n, n), rho_ref) <= 1e-13
    trk.close()


def test_noalloc_deposit_skips_and_flags_particles_outside_the_box():
    import paper_2208_02382_b300 as bt
    from paper_2208_02382_b300 import _lib as L
    lib = L.load()
    n = 64
    c = bg.gaussian6d(80_001, seed=9)
    c[0, 5] = np.nan
    beam = _beam(bt, c)
    lo, hi = _exact_box(np.nan_to_num(c))
    lo = [0.5 * v for v in lo]          # half the extent: the tails lie outside
    hi = [0.5 * v for v in hi]
    got, flags = _noalloc(lib, L, beam, lo, hi, n)
    assert flags == L.BX_NOALLOC_OUTSIDE | L.BX_NOALLOC_NONFINITE
    trk = bt.Tracker(n)
    want = trk.deposit(beam, bt.Grid(n, DEV, lo=lo, hi=hi)).rho.clone()
    with pytest.raises(L.BeamtrackError):
        trk.sync()                      # the context path reports the outside particles
    assert torch.equal(got, want)
    # the oracle on the particles well inside the box (none near a face)
    ref = oracle_ref(SP)
    pos = sc.rest_frame(np.nan_to_num(c, nan=1e9), ref)
    h = [(hi[d] - lo[d]) / (n - 1) for d in range(3)]
    u = [(pos[d] - lo[d]) / h[d] for d in range(3)]
    inside = np.all([(ud > 1e-6) & (ud < n - 1 - 1e-6) for ud in u], axis=0)
    near = np.any([((ud > -1e-6) & (ud <= 1e-6)) | ((ud >= n - 1 - 1e-6) & (ud < n - 1 + 1e-5))
                   for ud in u], axis=0)
    assert not near.any()
    rho_ref = sc.deposit(pos[:, inside], sc.macro_charge(1e-9, c.shape[1], ref),
                         sc.Box(tuple(lo), tuple(hi)), n)
    assert grid_rel_err(got.cpu().numpy().reshape(n, n, n), rho_ref) <= 1e-13
    trk.close()


def test_noalloc_deposit_rejects_grids_beyond_its_static_scratch():
    import paper_2208_02382_b300 as bt
    from paper_2208_02382_b300 import _lib as L
    lib = L.load()
    beam = _beam(bt, bg.gaussian6d(100, seed=3))
    out = torch.zeros(128 ** 3, dtype=torch.float64, device=DEV)
    b = beam.c_struct()
    rc = lib.bx_deposit_noalloc(ctypes.byref(b), (ctypes.c_double * 3)(-1, -1, -1),
                                (ctypes.c_double * 3)(1, 1, 1), 128,
                                ctypes.c_void_p(out.data_ptr()), None, None)
    assert rc == L.BX_BAD_ARG
    assert b"64" in lib.bx_last_error(None)
