"""Pins of the oracle's reference particle, element maps and schedule
against closed forms, the equations of motion and the paper's worked example
(Listing 1 / §Benchmark FODO Cell of arXiv:2208.02382)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import beamgen as bg
from oracle import physics as ph
from oracle import track as tr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
REFS = [ph.RefPart(bg.MASS_PROTON_MEV, 2000.0, 1.0), ph.RefPart(bg.MASS_PROTON_MEV, 1000.0, 1.0),
        ph.RefPart(bg.MASS_ELECTRON_MEV, 500.0, -1.0), ph.RefPart(bg.MASS_ELECTRON_MEV, 2000.0, -1.0)]


def test_refpart_kinetic_energy_reading():
    # 2 GeV kinetic proton: gamma = 1 + 2000/938.272...
    r = REFS[0]
    assert r.gamma == pytest.approx(3.131575, rel=1e-6)
    assert r.beta * r.gamma == pytest.approx(r.betagamma, rel=1e-15)
    assert r.gamma ** 2 * (1 - r.beta ** 2) == pytest.approx(1.0, rel=1e-13)


@pytest.mark.parametrize("ref", REFS)
@pytest.mark.parametrize("kind,k,angle", [(ph.DRIFT, 0, 0), (ph.QUAD, 1.3, 0), (ph.QUAD, -0.7, 0),
                                          (ph.QUAD, 0.0, 0), (ph.SBEND, 0, 0.1), (ph.SBEND, 0, -0.1)])
def test_maps_symplectic(ref, kind, k, angle):
    j = ph.symplectic_form()
    for ds in (0.01, 0.125, 0.5, 1.0):
        m = ph.element_matrix(kind, 0.5, k, angle, ds, ref)
        assert np.abs(m.T @ j @ m - j).max() <= 1e-12


@pytest.mark.parametrize("ref", REFS)
@pytest.mark.parametrize("kind,k,angle", [(ph.DRIFT, 0, 0), (ph.QUAD, 1.3, 0), (ph.QUAD, -0.7, 0),
                                          (ph.SBEND, 0, 0.1), (ph.SBEND, 0, -0.2)])
def test_maps_compose_as_a_flow(ref, kind, k, angle):
    # M(a) M(b) = M(a + b): holds only for the exact solution of a linear ODE
    a, b = 0.13, 0.29
    ma = ph.element_matrix(kind, 0.5, k, angle, a, ref)
    mb = ph.element_matrix(kind, 0.5, k, angle, b, ref)
    mab = ph.element_matrix(kind, 0.5, k, angle, a + b, ref)
    assert np.abs(ma @ mb - mab).max() <= 1e-13 * max(1.0, np.abs(mab).max())


def _ode_matrix(rhs, length):
    cols = []
    for c in range(6):
        y0 = np.zeros(6)
        y0[c] = 1.0
        sol = solve_ivp(lambda s, y: rhs(y), (0.0, length), y0, method="DOP853",
                        rtol=1e-13, atol=1e-15)
        cols.append(sol.y[:, -1])
    return np.array(cols).T


@pytest.mark.parametrize("ref", REFS[:3])
@pytest.mark.parametrize("k", [1.0, -1.0, 0.37])
def test_quad_solves_equations_of_motion(ref, k):
    # x'' = -k x, y'' = +k y, t' = pt/(beta gamma)^2 (linearised time of flight)
    bg2 = ref.betagamma ** 2

    def rhs(u):
        x, px, y, py, t, pt = u
        return np.array([px, -k * x, py, k * y, pt / bg2, 0.0])
    m = _ode_matrix(rhs, 0.8)
    assert np.abs(m - ph.quad_matrix(0.8, k, ref)).max() <= 1e-10


@pytest.mark.parametrize("ref", REFS[:3])
@pytest.mark.parametrize("angle", [0.1, -0.1, 0.3])
def test_sbend_solves_equations_of_motion(ref, angle):
    # linearised motion in a sector dipole of radius rho, with delta = -pt/beta:
    #   x'' = -x/rho^2 + delta/rho,  c dt/ds - 1/beta = x/(rho beta) + pt/(beta gamma)^2
    length = 0.5
    rho = length / angle
    b, bg2 = ref.beta, ref.betagamma ** 2

    def rhs(u):
        x, px, y, py, t, pt = u
        return np.array([px, -x / rho ** 2 - pt / (b * rho), py, 0.0, x / (rho * b) + pt / bg2, 0.0])
    m = _ode_matrix(rhs, length)
    assert np.abs(m - ph.sbend_matrix(length, rho, ref)).max() <= 1e-10


def test_sbend_small_angle_tends_to_drift():
    ref = REFS[1]
    # entries that differ from the drift are O(theta): sin/beta, rho(1-cos)/beta, ...
    m = ph.sbend_matrix(0.5, 0.5 / 1e-9, ref)
    assert np.abs(m - ph.drift_matrix(0.5, ref)).max() <= 2e-9 / ref.beta


def _fodo_matrix(lattice, ref):
    m = np.eye(6)
    for e in lattice:
        m = ph.element_matrix(e.kind, e.length, e.k, e.angle, e.length, ref) @ m
    return m


def test_worked_example_listing1():
    """The matched Waterbag parameters printed in Listing 1 follow from the FODO
    maps and the 2 nm emittance; the phase advance is the 67.8 deg of the FODO
    benchmark.  Parametrisation reading: lambda = sigma*sqrt(1 - r^2) and
    mu = -r with r the x-px correlation coefficient."""
    g = json.load(open(os.path.join(GOLDEN, "fodo_listing1.json")))
    ref = ph.RefPart(g["mass_MeV"], g["energy_MeV"], -1.0)
    lat = bg.fodo_cell(1)
    m = _fodo_matrix(lat, ref)
    eps = g["emittance_m"]
    got = {}
    for plane, a in (("x", 0), ("y", 2)):
        r2 = m[a:a + 2, a:a + 2]
        cmu = 0.5 * (r2[0, 0] + r2[1, 1])
        smu = math.copysign(math.sqrt(1 - cmu * cmu), r2[0, 1])
        beta = r2[0, 1] / smu
        alpha = (r2[0, 0] - r2[1, 1]) / (2 * smu)
        gam = (1 + alpha * alpha) / beta
        got[plane] = dict(mu=math.degrees(math.acos(cmu)), lam=math.sqrt(eps / gam),
                          lamp=math.sqrt(eps / beta), corr=-alpha / math.sqrt(1 + alpha * alpha))
    assert round(got["x"]["mu"], g["phase_advance_printed_decimals"]) == g["phase_advance_deg"]
    assert round(got["y"]["mu"], g["phase_advance_printed_decimals"]) == g["phase_advance_deg"]
    assert got["x"]["lam"] == pytest.approx(g["sigmaX"], rel=1e-9)
    assert got["y"]["lam"] == pytest.approx(g["sigmaY"], rel=1e-9)
    assert got["x"]["lamp"] == pytest.approx(g["sigmaPx"], rel=1e-9)
    assert got["y"]["lamp"] == pytest.approx(g["sigmaPy"], rel=1e-9)
    assert -got["x"]["corr"] == pytest.approx(g["muxpx"], rel=1e-9)
    assert -got["y"]["corr"] == pytest.approx(g["muypy"], rel=1e-9)


def test_matched_beam_returns_its_moments_after_one_cell():
    # §Benchmark FODO: second moments stay matched (no space charge)
    ref = ph.RefPart(bg.MASS_ELECTRON_MEV, 2000.0, -1.0)
    m = _fodo_matrix(bg.fodo_cell(1), ref)
    sig = np.zeros((6, 6))
    for a in (0, 2):
        r2 = m[a:a + 2, a:a + 2]
        cmu = 0.5 * (r2[0, 0] + r2[1, 1])
        smu = math.copysign(math.sqrt(1 - cmu * cmu), r2[0, 1])
        beta, alpha = r2[0, 1] / smu, (r2[0, 0] - r2[1, 1]) / (2 * smu)
        sig[a:a + 2, a:a + 2] = 2e-9 * np.array([[beta, -alpha], [-alpha, (1 + alpha ** 2) / beta]])
    sig[4, 4], sig[5, 5] = 1e-6, 4e-6
    out = m @ sig @ m.T
    assert np.abs(out[:4, :4] - sig[:4, :4]).max() <= 1e-12 * np.abs(sig[:4, :4]).max()


def test_emittance_invariant_without_space_charge():
    ref = ph.RefPart(bg.MASS_PROTON_MEV, 2000.0, 1.0)
    c0 = bg.gaussian6d(4000, seed=3)
    t = tr.Tracker(ref, 1e-9, 16, space_charge=False)
    c1 = t.track(c0, bg.fodo_lattice(10, 5))
    m0, m1 = tr.moments(c0), tr.moments(c1)
    for p in ("eps_x", "eps_y"):
        assert abs(m1[p] - m0[p]) <= 1e-12 * m0[p]
    assert not np.allclose(c0, c1)


def test_chicane_preserves_6d_covariance_determinant():
    ref = ph.RefPart(bg.MASS_ELECTRON_MEV, 500.0, -1.0)
    c0 = bg.gaussian6d(3000, seed=4)
    t = tr.Tracker(ref, 1e-9, 16, space_charge=False)
    c1 = t.track(c0, bg.chicane_lattice(3))
    d0 = np.linalg.det(tr.moments(c0)["cov"])
    d1 = np.linalg.det(tr.moments(c1)["cov"])
    assert d1 == pytest.approx(d0, rel=1e-9)


def test_slice_schedule_counts():
    lat = bg.fodo_lattice(10, 5)
    s = ph.slice_schedule(lat)
    assert len(s) == 250 == bg.count_kicks(lat)
    assert s[0] == (0, 0.05) and s[5] == (1, 0.2)
    with pytest.raises(ValueError):
        ph.slice_schedule([bg.drift(1.0, 0)])


def test_moments_brute_force_small():
    rng = np.random.default_rng(1)
    c = rng.standard_normal((6, 7))
    m = tr.moments(c)
    n = c.shape[1]
    for a in range(6):
        mean = sum(c[a, p] for p in range(n)) / n
        assert m["mean"][a] == pytest.approx(mean, rel=1e-14, abs=1e-15)
        for b in range(6):
            mb = sum(c[b, p] for p in range(n)) / n
            v = sum((c[a, p] - mean) * (c[b, p] - mb) for p in range(n)) / n
            assert m["cov"][a, b] == pytest.approx(v, rel=1e-12, abs=1e-15)
    ex = math.sqrt(m["cov"][0, 0] * m["cov"][1, 1] - m["cov"][0, 1] ** 2)
    assert m["eps_x"] == pytest.approx(ex, rel=1e-14)
    assert len(tr.moments_vector(c)) == 27


def test_rectangular_bend_chicane_is_achromatic():
    # four rectangular bends (sector bend + thin edges of half the bend angle
    # on both faces) close the dispersion: R16 = R26 = 0; sector bends alone
    # do not
    ref = ph.RefPart(bg.MASS_ELECTRON_MEV, 500.0, -1.0)

    def total(lat):
        m = np.eye(6)
        for e in lat:
            m = ph.element_matrix(e.kind, e.length, e.k, e.angle, e.length, ref, e.k2) @ m
        return m

    rect = total(bg.chicane_rect_lattice(1)[2:])
    sect = total(bg.chicane_lattice(1)[2:])
    assert abs(rect[0, 5]) < 1e-15 and abs(rect[1, 5]) < 1e-15
    assert abs(sect[0, 5]) > 1e-2
    # the edges only act on px, py (thin): det 1, symplectic
    j = ph.symplectic_form()
    for psi, h in ((0.05, 0.2), (-0.3, 1.7)):
        m = ph.dipedge_matrix(psi, h)
        assert np.abs(m.T @ j @ m - j).max() < 1e-15


def test_constant_focusing_solves_its_equation_of_motion():
    # u'' = -k_u u per plane: compare with direct integration, and k_x = k,
    # k_y = -k reproduces the quadrupole
    from scipy.integrate import solve_ivp
    ref = ph.RefPart(bg.MASS_PROTON_MEV, 1000.0, 1.0)
    kx, ky, L = 0.8, 2.5, 0.7
    m = ph.constf_matrix(L, kx, ky, ref)
    for (a, k) in ((0, kx), (2, ky)):
        sol = solve_ivp(lambda s, y: [y[1], -k * y[0]], (0, L), [1e-3, 2e-4], rtol=1e-12,
                        atol=1e-16)
        assert np.allclose(m[a:a + 2, a:a + 2] @ [1e-3, 2e-4], sol.y[:, -1], rtol=1e-9)
    assert np.allclose(ph.constf_matrix(L, 1.3, -1.3, ref), ph.quad_matrix(L, 1.3, ref))
    j = ph.symplectic_form()
    assert np.abs(m.T @ j @ m - j).max() < 1e-14


def test_thin_elements_between_slices_in_tracking():
    # a lattice with edges tracked slice by slice (no space charge) equals the
    # product of the element maps, whatever the slicing
    ref = ph.RefPart(bg.MASS_ELECTRON_MEV, 500.0, -1.0)
    lat = bg.chicane_rect_lattice(3)
    c0 = bg.gaussian6d(200, seed=8)
    t = tr.Tracker(ref, 1e-9, 8, space_charge=False)
    got = t.track(c0, lat)
    m = np.eye(6)
    for e in lat:
        m = ph.element_matrix(e.kind, e.length, e.k, e.angle, e.length, ref, e.k2) @ m
    assert np.allclose(got, m @ c0, rtol=1e-12, atol=1e-16)
    # split calls: thin elements between two calls are applied once
    t2 = tr.Tracker(ref, 1e-9, 8, space_charge=False)
    half = len(ph.slice_schedule(lat)) // 2
    c1 = t2.track(c0, lat, 0, half)
    c2 = t2.track(c1, lat, half, None)
    assert np.allclose(c2, got, rtol=1e-12, atol=1e-16)
