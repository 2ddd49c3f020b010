"""bx_moments on the GPU: the two ways of reading the particles, the exact-sum
properties, degenerate bunches, and the bounded device wait of the staging.

* Against oracle.track.moments_vector_exact (rational arithmetic, rounded once
  per output): degenerate and far-offset bunches, small and ragged.  The only
  rounding of the GPU path before its final conversion is q = round(x 2^k) at
  2^-43 of a coordinate's half-extent, so each mean is within 2^-42 of its
  half-extent and each second moment within 2^-40 of the product of the two
  half-extents; a coordinate whose particles all share one value has that
  exact mean and zero spread.
* Bulk copies (16-byte aligned arrays) and plain loads (arrays off 16-byte
  boundaries) give bitwise the same moments, and so does any particle order:
  the sums are exact integers.
* The bounded wait: a barrier that nothing completes times out, bx_sync
  reports BX_DEVICE_TIMEOUT, and the context keeps working."""
import ctypes
import time

import numpy as np
import pytest
import torch

import beamgen as bg
from oracle import track as tr

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def bt():
    import paper_2208_02382_b300 as p
    from paper_2208_02382_b300 import build
    build.build()
    return p


def moments_raw(bt, trk, rows):
    """bx_moments on six separately allocated device arrays (each 16-byte
    aligned whatever n is)."""
    from paper_2208_02382_b300 import _lib as L
    b = L.bx_beam()
    for k in range(6):
        b.coord[k] = rows[k].data_ptr()
    b.id = None
    b.n = rows[0].numel()
    b.charge_sign, b.bunch_charge_C, b.mass_MeV, b.kinetic_MeV = 1.0, 1e-9, 938.272, 1000.0
    out = torch.empty(27, dtype=torch.float64, device=DEV)
    rc = trk.lib.bx_moments(trk.ctx, ctypes.byref(b), ctypes.c_void_p(out.data_ptr()),
                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, trk.lib.bx_last_error(trk.ctx)
    return out.cpu().numpy()


def moments_offset(bt, trk, c):
    """bx_moments of the bunch stored 8 bytes past a 16-byte boundary (every
    row misaligned: the plain-load path)."""
    n = c.shape[1]
    buf = torch.empty(6 * n + 1, dtype=torch.float64, device=DEV)
    v = buf[1:].view(6, n)
    v.copy_(torch.tensor(c, dtype=torch.float64))
    assert v.data_ptr() % 16 == 8
    beam = bt.Beam(v, bt.Species(938.272, 1000.0, 1.0), 1e-9)
    assert beam.coords.data_ptr() == v.data_ptr()
    return trk.moments(beam).cpu().numpy()


def rows_of(c):
    return [torch.tensor(np.ascontiguousarray(c[k]), dtype=torch.float64, device=DEV)
            for k in range(6)]


def assert_close_to_exact(m, c):
    ex = tr.moments_vector_exact(c)
    half = (c.max(axis=1) - c.min(axis=1)) / 2
    iu = np.triu_indices(6)
    for a in range(6):
        if half[a] == 0.0:
            assert m[a] == c[a, 0]                   # one shared value: exact
        else:
            assert abs(m[a] - ex[a]) <= 2.0 ** -42 * half[a] + 2.0 ** -52 * abs(ex[a]), a
    for k, (a, b) in enumerate(zip(*iu)):
        if half[a] == 0.0 or half[b] == 0.0:
            assert m[6 + k] == 0.0, (a, b)
        else:
            assert abs(m[6 + k] - ex[6 + k]) <= 2.0 ** -40 * half[a] * half[b] + \
                2.0 ** -50 * abs(ex[6 + k]), (a, b)


def _case(name, n, seed=0):
    rng = np.random.default_rng(seed)
    c = rng.normal(size=(6, n)) * np.array([1e-3, 1e-4, 2e-3, 3e-4, 1e-2, 1e-5])[:, None]
    if name == "constant_rows":
        c[1] = 1e-3                                  # a shared non-integer value
        c[5] = -2.5
    elif name == "far_offset":
        c[4] = 1e6 + rng.normal(size=n) * 1e-9       # spread far below the offset's ulp scale
        c[0] += 7.0
    elif name == "halo":
        c[:, : max(1, n // 100)] *= 50.0
    return c


CASES = [("gauss", 1), ("gauss", 2), ("constant_rows", 1), ("constant_rows", 3),
         ("far_offset", 5), ("gauss", 1_023), ("halo", 1_025), ("constant_rows", 2_049),
         ("far_offset", 3_001), ("halo", 20_001)]


@pytest.mark.parametrize("name,n", CASES)
def test_moments_match_exact_rational_moments(bt, name, n):
    c = _case(name, n, seed=n)
    trk = bt.Tracker(8)
    m = moments_raw(bt, trk, rows_of(c))            # bulk copies, ragged (odd) tails included
    assert_close_to_exact(m, c)
    assert np.array_equal(moments_offset(bt, trk, c), m)    # plain loads: bitwise the same
    trk.sync()
    trk.close()


@pytest.mark.parametrize("n", [148 * 1024 * 2 + 777, 148 * 1024 * 3 + 1_024])
def test_bulk_copy_and_plain_load_paths_agree_bitwise_and_match_oracle(bt, n):
    c = bg.gaussian_with_halo(n, seed=11)
    trk = bt.Tracker(8)
    m = moments_raw(bt, trk, rows_of(c))
    ref = tr.moments_vector(c)
    assert np.abs(m - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.array_equal(moments_offset(bt, trk, c), m)
    trk.sync()
    trk.close()


def test_moments_do_not_depend_on_particle_order(bt):
    c = bg.gaussian_with_halo(500_001, seed=3)
    trk = bt.Tracker(8)
    m = moments_raw(bt, trk, rows_of(c))
    perm = np.random.default_rng(9).permutation(c.shape[1])
    assert np.array_equal(moments_raw(bt, trk, rows_of(c[:, perm])), m)
    trk.close()


def test_headline_bunch_moments_match_oracle(bt):
    """The 2.5e7-particle chicane bunch the end-to-end loop reads every step."""
    w = bg.workload("chicane_25e6_128")
    c = w.particles()
    trk = bt.Tracker(8)
    m = moments_raw(bt, trk, rows_of(c))
    ref = tr.moments_vector(c)
    assert np.abs(m - ref).max() <= 1e-12 * np.abs(ref).max()
    # per entry: means relative to |mean| + rms, second moments to
    # sqrt(C_aa C_bb) (their Cauchy-Schwarz bound)
    iu = np.triu_indices(6)
    var = ref[6:][[k for k, (a, b) in enumerate(zip(*iu)) if a == b]]
    rms = np.sqrt(var)
    scale = np.concatenate([np.abs(ref[:6]) + rms, rms[iu[0]] * rms[iu[1]]])
    assert (np.abs(m - ref) <= 1e-11 * scale).all()
    trk.close()


def test_bounded_wait_times_out_and_the_context_survives(bt):
    from paper_2208_02382_b300 import _lib as L
    trk = bt.Tracker(8)
    c = bg.gaussian_with_halo(10_001, seed=5)
    rows = rows_of(c)
    before = moments_raw(bt, trk, rows)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    trk.selftest_wait_timeout(150.0)
    with pytest.raises(L.BeamtrackError) as err:
        trk.sync()
    dt = time.perf_counter() - t0
    assert err.value.code == L.BX_DEVICE_TIMEOUT
    assert 0.15 <= dt < 10.0
    trk.sync()                                      # the status was cleared
    assert np.array_equal(moments_raw(bt, trk, rows), before)
    trk.sync()
    trk.close()
