"""Pins of the oracle's space-charge kick: IGF against quadrature and closed
forms, deposit invariants, the FFT solve against the direct sum, fields of
a uniform ellipsoid and a spherical Gaussian, a direct Coulomb sum, the
envelope perveance and rest-frame isotropy of the kick."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import beamgen as bg
from oracle import physics as ph
from oracle import spacecharge as sc
from oracle import track as tr

KE = 1.0 / (4 * math.pi * ph.EPS0)


# ------------------------------------------------------------------ IGF

def _box_quad(a, b, c, h):
    f = lambda z, y, x: 1.0 / math.sqrt(x * x + y * y + z * z)
    lo = [(a - 0.5) * h[0], (b - 0.5) * h[1], (c - 0.5) * h[2]]
    v, _ = integrate.tplquad(f, lo[0], lo[0] + h[0], lo[1], lo[1] + h[1], lo[2], lo[2] + h[2],
                             epsabs=0, epsrel=1e-13)
    return KE * v


def test_igf_cube_at_origin_closed_form(oracle_lib):
    # integral of 1/r over the unit cube centred at the origin = 3 ln(2+sqrt3) - pi/2
    h = 2e-3
    want = KE * h * h * (3 * math.log(2 + math.sqrt(3)) - math.pi / 2)
    assert sc.igf_point(0, 0, 0, (h, h, h)) == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("off", [(1, 0, 0), (1, 1, 0), (2, 1, 1), (3, 0, 2), (0, 0, 4)])
@pytest.mark.parametrize("h", [(1e-3, 1e-3, 1e-3), (1e-3, 2e-3, 5e-3), (5e-4, 5e-4, 2e-2)])
def test_igf_matches_triple_quadrature(oracle_lib, off, h):
    assert sc.igf_point(*off, h) == pytest.approx(_box_quad(*off, h), rel=1e-11)


def test_igf_far_cells_match_high_precision_quadrature(oracle_lib):
    import mpmath as mp
    mp.mp.dps = 30
    for off, h in [((40, 30, 20), (1e-3, 1e-3, 1e-3)), ((100, 3, 2), (1e-3, 1e-3, 2e-2)),
                   ((64, 64, 64), (1e-3, 1.5e-3, 1e-3))]:
        lo = [mp.mpf(off[d] - 0.5) * mp.mpf(h[d]) for d in range(3)]
        hi = [mp.mpf(off[d] + 0.5) * mp.mpf(h[d]) for d in range(3)]
        v = mp.quad(lambda x, y, z: 1 / mp.sqrt(x * x + y * y + z * z),
                    [lo[0], hi[0]], [lo[1], hi[1]], [lo[2], hi[2]], method="gauss-legendre")
        want = float(v / (4 * mp.pi * mp.mpf("8.8541878128e-12")))
        got = sc.igf_point(*off, h)
        assert got == pytest.approx(want, rel=2e-15)
        # plain double loses many digits to cancellation here; the oracle must not
        assert abs(sc.igf_point_double(*off, h) - want) > 10 * abs(got - want)


def test_igf_even_symmetry(oracle_lib):
    h = (1e-3, 2e-3, 3e-3)
    for a, b, c in [(1, 2, 3), (5, 0, 1), (0, 7, 2)]:
        g = sc.igf_point(a, b, c, h)
        for s in [(-1, 1, 1), (1, -1, 1), (1, 1, -1), (-1, -1, -1)]:
            assert sc.igf_point(s[0] * a, s[1] * b, s[2] * c, h) == pytest.approx(g, rel=1e-15)


def test_igf_far_field_limit(oracle_lib):
    h = (1e-3, 1e-3, 1e-3)
    for off in [(200, 150, 100), (300, 0, 0)]:
        r = math.sqrt(sum((o * 1e-3) ** 2 for o in off))
        assert sc.igf_point(*off, h) / (KE * 1e-9 / r) == pytest.approx(1.0, abs=1e-9)


def test_igf_octant_table_and_doubled_layout(oracle_lib):
    n, h = 6, (1e-3, 1.3e-3, 0.7e-3)
    oct_ = sc.igf_octant(n, h)
    for (c, b, a) in [(0, 0, 0), (1, 2, 3), (6, 6, 6), (0, 5, 2)]:
        assert oct_[c, b, a] == pytest.approx(sc.igf_point(a, b, c, h), rel=1e-15)
    gd = sc.green_doubled(n, h)
    assert gd.shape == (12, 12, 12)
    assert gd[0, 0, n] == oct_[0, 0, n]            # offset +-n holds the true value
    assert gd[0, 0, n + 1] == oct_[0, 0, n - 1]    # index n+1 is offset -(n-1)
    assert np.array_equal(gd, gd[::-1, ::-1, ::-1][np.ix_(*[np.r_[-1, 0:11]] * 3)])


# ----------------------------------------------------------------- deposit

def _rand_pos(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3, n)) * np.array([[1e-3], [2e-3], [5e-3]])


def test_deposit_conserves_charge_and_centroid():
    pos = _rand_pos(5000, 1)
    box, _ = sc.box_rule(pos, None)
    n = 16
    q = 1e-9 / 5000
    rho = sc.deposit(pos, q, box, n)
    h = box.h(n)
    vol = h[0] * h[1] * h[2]
    assert rho.sum() * vol == pytest.approx(1e-9, rel=1e-13)
    # CIC reproduces linear functions: sum_nodes w_node * x_node = X
    nodes = [box.lo[d] + h[d] * np.arange(n) for d in range(3)]
    for d, axis in ((0, (0, 1)), (1, (0, 2)), (2, (1, 2))):
        prof = rho.sum(axis=axis) * vol
        assert (prof * nodes[d]).sum() == pytest.approx(q * pos[d].sum(), rel=1e-11, abs=1e-24)


def test_deposit_node_and_cell_centre_cases():
    n = 8
    box = sc.Box((0.0, 0.0, 0.0), (7.0, 7.0, 7.0))      # h = 1
    rho = sc.deposit(np.array([[2.0], [3.0], [4.0]]), 1.0, box, n)
    assert rho[4, 3, 2] == 1.0 and rho.sum() == 1.0
    rho = sc.deposit(np.array([[2.5], [3.5], [4.5]]), 1.0, box, n)
    assert np.all(rho[4:6, 3:5, 2:4] == 0.125) and rho.sum() == 1.0
    # a particle on the upper edge lands on the last node (clamped cell n-2)
    rho = sc.deposit(np.array([[7.0], [0.0], [0.0]]), 1.0, box, n)
    assert rho[0, 0, 7] == 1.0


def test_box_rule_contains_particles_and_regrids_on_shrink():
    pos = _rand_pos(1000, 2)
    box, r = sc.box_rule(pos, None)
    assert r
    for d in range(3):
        assert box.lo[d] <= pos[d].min() and pos[d].max() < box.hi[d]
        ext = pos[d].max() - pos[d].min()
        assert box.hi[d] - box.lo[d] == pytest.approx(1.1 * ext, rel=1e-12)
    box2, r2 = sc.box_rule(pos * 0.95, box)
    assert not r2 and box2 == box
    box3, r3 = sc.box_rule(pos * 0.4, box)
    assert r3
    box4, r4 = sc.box_rule(pos * 1.2, box)
    assert r4
    one, _ = sc.box_rule(np.zeros((3, 1)), None)
    assert all(one.hi[d] > one.lo[d] for d in range(3))


# ------------------------------------------------------------------- solve

def test_fft_solve_equals_direct_sum(oracle_lib):
    n, h = 6, (1e-3, 1.5e-3, 2.5e-3)
    rng = np.random.default_rng(5)
    rho = rng.random((n, n, n)) - 0.3
    phi = sc.solve(rho, h)
    ref = sc.solve_direct(rho, h)
    assert np.abs(phi - ref).max() <= 1e-13 * np.abs(ref).max()


def _ellipsoid_factor(a, b, c, i):
    # depolarisation factor; scale-free, evaluated in units of the largest axis
    u = max(a, b, c)
    a, b, c = a / u, b / u, c / u
    ax = (a, b, c)[i]
    f = lambda s: 1.0 / ((ax * ax + s) * math.sqrt((a * a + s) * (b * b + s) * (c * c + s)))
    v, _ = integrate.quad(f, 0, np.inf, epsabs=1e-14, epsrel=1e-12, limit=200)
    return a * b * c / 2 * v


def _field_at_particles(pos, q, n):
    box, _ = sc.box_rule(pos, None)
    h = box.h(n)
    rho = sc.deposit(pos, q, box, n)
    e = sc.field(sc.solve(rho, h), h)
    return sc.gather(pos, e, box)


def test_uniform_ellipsoid_field_converges_to_closed_form(oracle_lib):
    # interior field of a uniformly charged ellipsoid: E_i = rho0/eps0 * N_i * x_i
    semi = (1.0e-3, 1.5e-3, 2.5e-3)
    p6 = bg.uniform_lattice_points(64, semi)
    pos = np.stack([p6[0], p6[2], p6[4]])
    q_tot = 1e-9
    q = q_tot / pos.shape[1]
    rho0 = q_tot / (4.0 / 3.0 * math.pi * semi[0] * semi[1] * semi[2])
    fac = [_ellipsoid_factor(*semi, i) for i in range(3)]
    assert sum(fac) == pytest.approx(1.0, rel=1e-9)
    inner = ((pos / np.array(semi)[:, None]) ** 2).sum(axis=0) < 0.5 ** 2
    for n in (16, 32):
        e = _field_at_particles(pos, q, n)
        for i in range(3):
            want = rho0 / ph.EPS0 * fac[i] * pos[i, inner]
            slope = (e[i, inner] @ want) / (want @ want)
            assert slope == pytest.approx(1.0, rel=0.01)
            assert np.abs(e[i, inner] - want).max() <= 0.03 * np.abs(want).max()


def test_spherical_gaussian_field_closed_form(oracle_lib):
    # E_r = Q/(4 pi eps0 r^2) [erf(r/(sqrt2 s)) - sqrt(2/pi) (r/s) exp(-r^2/2s^2)]
    s = 1e-3
    rng = np.random.default_rng(11)
    pos = rng.standard_normal((3, 200_000)) * s
    q_tot = 1e-9
    r = np.sqrt((pos ** 2).sum(axis=0))
    sel = (r > 0.5 * s) & (r < 2.0 * s)
    rr = r[sel] / s
    want = KE * q_tot / r[sel] ** 2 * (special.erf(rr / math.sqrt(2))
                                       - math.sqrt(2 / math.pi) * rr * np.exp(-rr * rr / 2))
    rel = []
    for n in (32, 64):
        e = _field_at_particles(pos, q_tot / pos.shape[1], n)
        er = (e[:, sel] * pos[:, sel]).sum(axis=0) / r[sel]
        rel.append(np.sqrt(np.mean((er - want) ** 2)) / np.sqrt(np.mean(want ** 2)))
    # the box spans +-4.7 sigma, so h = 0.33 sigma at n = 32: second-order convergence
    assert rel[1] < 0.03 and rel[0] / rel[1] > 3.0


def test_direct_coulomb_sum_small_bunch(oracle_lib):
    """2000 point charges: the grid field converges to the direct Coulomb sum.
    The direct field at a particle carries near-neighbour graininess that the
    grid smooths away, so the statistics are the regression of the direct
    field on the grid field (noise in the regressand does not bias it) and the
    virial sum_p x_p E_x(p)."""
    rng = np.random.default_rng(7)
    npart = 2000
    sig = np.array([[1e-3], [1.2e-3], [2e-3]])
    pos = rng.standard_normal((3, npart)) * sig
    q = 1e-12
    direct = sc.coulomb_direct(pos, q)
    core = ((pos / sig) ** 2).sum(axis=0) < 2.0 ** 2
    dev = []
    for n in (16, 32):
        grid = _field_at_particles(pos, q, n)
        for c in range(3):
            a, b = grid[c, core], direct[c, core]
            slope = (a @ b) / (a @ a)
            virial = (pos[c] * grid[c]).sum() / (pos[c] * direct[c]).sum()
            dev.append((abs(slope - 1), abs(virial - 1)))
            if n == 32:
                assert 0.95 < slope < 1.1 and 0.95 < virial < 1.02
                assert np.corrcoef(a, b)[0, 1] > 0.6
    for c in range(3):
        assert dev[3 + c][0] < dev[c][0] and dev[3 + c][1] < dev[c][1]


# --------------------------------------------------------------------- kick

@pytest.mark.parametrize("species", [bg.PROTON_2GEV, bg.ELECTRON_500MEV])
def test_kick_defocuses_and_matches_envelope_perveance(oracle_lib, species):
    """Long uniform round beam (radius a) in a drift: x'' = K x / a^2 with the
    generalised perveance K = 2 I / (I0 beta^3 gamma^3), I0 = 4 pi eps0 m c^3/e
    (textbook envelope equation).  Built in the rest frame, lab length L/gamma."""
    ref = ph.RefPart(species.mass_MeV, species.kinetic_MeV, species.charge_sign)
    a_r, length = 1e-3, 40e-3
    s = (np.arange(64) + 0.5) / 64 * 2 - 1
    gx, gy, gz = np.meshgrid(s, s, np.linspace(-1, 1, 400), indexing="ij")
    m = gx ** 2 + gy ** 2 <= 1.0
    pos = np.stack([gx[m] * a_r, gy[m] * a_r, gz[m] * length / 2])
    q_tot = 1e-9 * species.charge_sign
    e = _field_at_particles(pos, q_tot / pos.shape[1], 32)
    coords = np.zeros((6, pos.shape[1]))
    coords[0], coords[2], coords[4] = pos[0], pos[1], -pos[2] / ref.betagamma
    ds = 0.01
    out = sc.kick(coords, e, ds, ref)
    sel = (np.abs(pos[2]) < length / 8) & (np.hypot(pos[0], pos[1]) < 0.6 * a_r)
    dpx = out[1, sel] - coords[1, sel]
    slope = (dpx @ pos[0, sel]) / (pos[0, sel] @ pos[0, sel])
    lam_lab = abs(q_tot) / (length / ref.gamma)
    current = lam_lab * ref.beta * ph.C_LIGHT
    i0 = 4 * math.pi * ph.EPS0 * ph.C_LIGHT * ref.mass_eV
    k_perv = 2 * current / (i0 * ref.beta ** 3 * ref.gamma ** 3)
    assert slope > 0      # same-sign charges defocus
    assert slope == pytest.approx(k_perv / a_r ** 2 * ds, rel=0.05)


def test_kick_rest_frame_isotropy(oracle_lib):
    """In a uniformly charged sphere the rest-frame force is isotropic,
    F' = q rho r'/(3 eps0).  The rest-frame impulse over the proper time of a
    slice is carried to the lab by the boost: transverse momentum unchanged,
    energy change beta c gamma dp'_z; so dpt/dpx at equal rest-frame
    displacement is -beta gamma, and dpx/X = q rho/(3 eps0) dtau/p_ref."""
    ref = ph.RefPart(bg.MASS_PROTON_MEV, 1000.0, 1.0)
    rad = 1e-3
    p6 = bg.uniform_lattice_points(56, (rad, rad, rad))
    pos = np.stack([p6[0], p6[2], p6[4]])
    q_tot = 1e-9
    e = _field_at_particles(pos, q_tot / pos.shape[1], 32)
    coords = np.zeros((6, pos.shape[1]))
    coords[0], coords[2], coords[4] = pos[0], pos[1], -pos[2] / ref.betagamma
    ds = 0.02
    out = sc.kick(coords, e, ds, ref)
    inner = (pos ** 2).sum(axis=0) < (0.5 * rad) ** 2
    kx = (out[1, inner] @ pos[0, inner]) / (pos[0, inner] @ pos[0, inner])
    kz = (out[5, inner] @ pos[2, inner]) / (pos[2, inner] @ pos[2, inner])
    rho0 = q_tot / (4.0 / 3.0 * math.pi * rad ** 3)
    dtau = ds / (ref.beta * ph.C_LIGHT * ref.gamma)
    p_ref = ref.betagamma * ref.mass_eV * ph.Q_E / ph.C_LIGHT
    want_kx = ph.Q_E * rho0 / (3 * ph.EPS0) * dtau / p_ref
    assert kx == pytest.approx(want_kx, rel=0.03)
    assert kz / kx == pytest.approx(-ref.betagamma, rel=0.03)


def test_zero_charge_reduces_bitwise_to_no_space_charge(oracle_lib):
    ref = ph.RefPart(bg.MASS_PROTON_MEV, 2000.0, 1.0)
    c0 = bg.gaussian6d(500, seed=9)
    lat = bg.fodo_lattice(1, 2)
    a = tr.Tracker(ref, 0.0, 8, space_charge=True).track(c0, lat)
    b = tr.Tracker(ref, 0.0, 8, space_charge=False).track(c0, lat)
    assert np.array_equal(a, b)


def test_space_charge_grows_emittance_of_dense_bunch(oracle_lib):
    w = bg.workload("fodo_1e4_32")
    ref = ph.RefPart(w.species.mass_MeV, w.species.kinetic_MeV, w.species.charge_sign)
    c0 = w.particles(2000)
    t = tr.Tracker(ref, w.bunch_charge_C, 16)
    c1 = t.track(c0, w.lattice, 0, 10)
    assert tr.moments(c1)["sigma"][1] > tr.moments(c0)["sigma"][1]
    assert t.regrid_log[0] == 0 and t.kick_index == 10


def test_nonfinite_input_is_rejected(oracle_lib):
    ref = ph.RefPart(bg.MASS_PROTON_MEV, 2000.0, 1.0)
    c0 = bg.gaussian6d(10, seed=1)
    c0[0, 3] = np.nan
    with pytest.raises(FloatingPointError):
        tr.Tracker(ref, 1e-9, 8).track(c0, bg.fodo_lattice(1, 1))


# ------------------------------------------------------------------- TSC

def test_tsc_weights_moments():
    # quadratic B-spline: weights sum to 1, their first moment is the offset
    # f (linear interpolation exact), their second moment about f is 1/4
    box = sc.Box((0.0, 0.0, 0.0), (7.0, 7.0, 7.0))
    rng = np.random.default_rng(3)
    pos = rng.uniform(0.6, 6.4, size=(3, 500))
    (i, j, l), w = sc.tsc_nodes(pos, box, 8)
    for d, idx in enumerate((i, j, l)):
        f = pos[d] - idx
        s0 = w[d][0] + w[d][1] + w[d][2]
        s1 = w[d][2] - w[d][0]
        s2 = w[d][0] * (-1 - f) ** 2 + w[d][1] * f ** 2 + w[d][2] * (1 - f) ** 2
        assert np.allclose(s0, 1.0, rtol=0, atol=1e-15)
        assert np.allclose(s1, f, rtol=0, atol=1e-15)
        assert np.allclose(s2, 0.25, rtol=0, atol=1e-15)


def test_tsc_deposit_conserves_charge_and_centroid_and_gathers_linear_fields():
    n = 16
    c = bg.gaussian6d(3000, seed=31)
    ref = ph.RefPart(bg.MASS_PROTON_MEV, 1000.0, 1.0)
    pos = sc.rest_frame(c, ref)
    box, _ = sc.box_rule(pos, None)
    h = box.h(n)
    q = 1e-12
    rho = sc.deposit(pos, q, box, n, shape=2)
    V = h[0] * h[1] * h[2]
    assert rho.sum() * V == pytest.approx(q * pos.shape[1], rel=1e-13)
    grid = [box.lo[d] + h[d] * np.arange(n) for d in range(3)]
    for d, ax in ((0, (0, 1)), (1, (0, 2)), (2, (1, 2))):
        mom = (rho.sum(axis=ax) * grid[d]).sum() * V
        assert mom == pytest.approx(q * pos[d].sum(), rel=1e-12)
    # a linear field is interpolated exactly
    zz, yy, xx = np.meshgrid(*grid[::-1], indexing="ij")
    ef = np.stack([2.0 * xx - yy, 3.0 * zz + 1.0, -xx + yy + zz])
    got = sc.gather(pos, ef, box, shape=2)
    X, Y, Z = pos
    want = np.stack([2 * X - Y, 3 * Z + 1, -X + Y + Z])
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


def test_tsc_field_converges_to_cic_and_to_the_coulomb_sum():
    # the same bunch with both shapes: the TSC grid field approaches the direct
    # Coulomb field as the CIC one does (regression slope and virial in the
    # core, as for CIC above), and the two grid fields agree closely
    rng = np.random.default_rng(7)
    npart = 2000
    sig = np.array([[1e-3], [1.2e-3], [2e-3]])
    pos = rng.standard_normal((3, npart)) * sig
    q = 1e-12
    direct = sc.coulomb_direct(pos, q)
    core = ((pos / sig) ** 2).sum(axis=0) < 2.0 ** 2
    n = 32
    box, _ = sc.box_rule(pos, None)
    h = box.h(n)
    ghat = sc.green_hat(n, h)
    fields = {}
    for shape in (1, 2):
        phi = sc.solve(sc.deposit(pos, q, box, n, shape), h, ghat)
        fields[shape] = sc.gather(pos, sc.field(phi, h), box, shape)
    for c in range(3):
        a, b = fields[2][c, core], direct[c, core]
        slope = (a @ b) / (a @ a)
        virial = (pos[c] * fields[2][c]).sum() / (pos[c] * direct[c]).sum()
        assert 0.95 < slope < 1.1 and 0.95 < virial < 1.02
    scale = np.sqrt(np.mean(fields[1] ** 2))
    assert np.sqrt(np.mean((fields[2] - fields[1]) ** 2)) / scale < 0.1
