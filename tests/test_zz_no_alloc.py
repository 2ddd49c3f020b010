"""GPU test of bx_deposit_noalloc, the deposition entry point for callers that
may not allocate device memory while running (fixed-footprint control-loop
models, hosts that own all device memory).  It must give the same charge
density as bx_deposit with an explicit box, call after call, although its
accumulators live in a static array that every call reuses.

This file sorts last so that a run stopping at the first failure has already
run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import beamgen as bg
from tests.parity import grid_rel_err

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _beam(bt, coords):
    sp = bg.PROTON_1GEV
    t = torch.tensor(np.ascontiguousarray(coords), dtype=torch.float64, device=DEV)
    return bt.Beam(t, bt.Species(sp.mass_MeV, sp.kinetic_MeV, sp.charge_sign), 1e-9)


def test_noalloc_deposit_matches_context_deposit_on_consecutive_calls():
    import paper_2208_02382_b300 as bt
    from paper_2208_02382_b300 import _lib as L
    from paper_2208_02382_b300 import build
    build.build()
    lib = L.load()
    n = 32
    trk = bt.Tracker(n)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed, npart in ((1, 100_003), (2, 54_321)):   # two calls in a row, different bunches
        beam = _beam(bt, bg.gaussian6d(npart, seed=seed))
        ref = trk.deposit(beam, bt.Grid(n, DEV))       # context path, box rule
        lo, hi = list(ref.lo), list(ref.hi)
        want = trk.deposit(beam, bt.Grid(n, DEV, lo=lo, hi=hi)).rho.clone()
        out = torch.full((n ** 3,), np.nan, dtype=torch.float64, device=DEV)
        b = beam.c_struct()
        rc = lib.bx_deposit_noalloc(ctypes.byref(b), (ctypes.c_double * 3)(*lo),
                                    (ctypes.c_double * 3)(*hi), n,
                                    ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == L.BX_OK, lib.bx_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert grid_rel_err(got, want.cpu().numpy()) <= 1e-13


def test_noalloc_deposit_rejects_grids_beyond_its_static_scratch():
    import paper_2208_02382_b300 as bt
    from paper_2208_02382_b300 import _lib as L
    lib = L.load()
    beam = _beam(bt, bg.gaussian6d(100, seed=3))
    out = torch.zeros(128 ** 3, dtype=torch.float64, device=DEV)
    b = beam.c_struct()
    rc = lib.bx_deposit_noalloc(ctypes.byref(b), (ctypes.c_double * 3)(-1, -1, -1),
                                (ctypes.c_double * 3)(1, 1, 1), 128,
                                ctypes.c_void_p(out.data_ptr()), None)
    assert rc == L.BX_BAD_ARG
    assert b"64" in lib.bx_last_error(None)
