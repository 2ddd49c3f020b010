"""Pins of the oracle's thin multipole kick (paper §Numerical Experiments: a
chain of thin multipoles; no formula in the paper).  The kick is pinned by
what fixes it independently of its own formula: the thick quadrupole map in
its thin limit (overall sign), Maxwell's equations in the magnet gap (the
kick's Jacobian in x, y is symmetric and traceless; a wrong sign of py or a
wrong power fails this), the rotation that turns a normal multipole into a
skew one (the relative phase of kn and ks), the textbook sextupole kick,
and symplecticity of tracking through a lattice of thick elements and thin
multipoles."""
import math

import numpy as np
import pytest

import beamgen as bg
from oracle import physics as ph
from oracle import track as tr

REF = ph.RefPart(bg.MASS_PROTON_MEV, 1000.0, 1.0)


def _points(n=64, seed=3, scale=1e-3):
    rng = np.random.default_rng(seed)
    c = np.zeros((6, n))
    c[ph.X] = rng.normal(0.0, scale, n)
    c[ph.Y] = rng.normal(0.0, scale, n)
    c[ph.PX] = rng.normal(0.0, 1e-4, n)
    c[ph.PY] = rng.normal(0.0, 1e-4, n)
    c[ph.T] = rng.normal(0.0, 1e-3, n)
    c[ph.PT] = rng.normal(0.0, 1e-4, n)
    return c


def _kicks(c, order, kn, ks):
    out = ph.multipole_kick(c, order, kn, ks)
    return out[ph.PX] - c[ph.PX], out[ph.PY] - c[ph.PY]


def test_multipole_changes_momenta_only():
    c = _points()
    out = ph.multipole_kick(c, 4, 3e4, -2e4)
    for d in (ph.X, ph.Y, ph.T, ph.PT):
        assert np.array_equal(out[d], c[d])
    assert not np.array_equal(out[ph.PX], c[ph.PX])


def test_order_two_is_the_thin_limit_of_the_thick_quadrupole():
    # quad(ds, k = K/ds) tends to px -= K x, py += K y as ds -> 0 (error O(K ds))
    c = _points()
    kint = 0.7
    dpx, dpy = _kicks(c, 2, kint, 0.0)
    for ds in (1e-5, 1e-6):
        m = ph.quad_matrix(ds, kint / ds, REF)
        assert m[ph.PX, ph.X] == pytest.approx(-kint, rel=5 * kint * ds)
        assert m[ph.PY, ph.Y] == pytest.approx(kint, rel=5 * kint * ds)
    assert np.allclose(dpx, -kint * c[ph.X], rtol=1e-14, atol=0)
    assert np.allclose(dpy, kint * c[ph.Y], rtol=1e-14, atol=0)


def test_sextupole_textbook_kick():
    c = _points()
    k = 37.0
    dpx, dpy = _kicks(c, 3, k, 0.0)
    x, y = c[ph.X], c[ph.Y]
    assert np.allclose(dpx, -0.5 * k * (x * x - y * y), rtol=1e-13, atol=1e-22)
    assert np.allclose(dpy, k * x * y, rtol=1e-13, atol=1e-22)


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6, 8])
def test_kick_obeys_maxwell_in_the_gap(order):
    # dpx = -L B_y/(B rho), dpy = L B_x/(B rho): div B = 0 makes the Jacobian
    # symmetric (d dpx/dy = d dpy/dx), curl B = 0 makes it traceless
    rng = np.random.default_rng(order)
    kn, ks = rng.normal(size=2) * math.factorial(order - 1) * 1e3 ** (order - 1) * 1e-5
    c = _points(16, seed=order)
    h = 1e-7
    jac = np.zeros((2, 2, c.shape[1]))
    for j, d in enumerate((ph.X, ph.Y)):
        cp, cm = c.copy(), c.copy()
        cp[d] += h
        cm[d] -= h
        fp, fm = _kicks(cp, order, kn, ks), _kicks(cm, order, kn, ks)
        for i in range(2):
            jac[i, j] = (fp[i] - fm[i]) / (2 * h)
    scale = np.max(np.abs(jac)) + 1e-300
    if order == 1:
        assert scale < 1e-9  # a dipole kick does not depend on position
        return
    assert np.max(np.abs(jac[0, 1] - jac[1, 0])) < 1e-6 * scale
    assert np.max(np.abs(jac[0, 0] + jac[1, 1])) < 1e-6 * scale


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 6])
def test_skew_multipole_is_the_normal_one_rotated(order):
    # a magnet rotated about s by phi kicks as R(phi) k(R(-phi) r); the skew
    # multipole of order m is the normal one rotated by -pi/(2m)
    c = _points(32, seed=10 + order)
    k = 1.3 * math.factorial(order - 1) * 1e3 ** (order - 1) * 1e-5
    phi = -math.pi / (2 * order)
    cs, sn = math.cos(phi), math.sin(phi)
    r = c.copy()
    r[ph.X] = cs * c[ph.X] + sn * c[ph.Y]       # R(-phi) r
    r[ph.Y] = -sn * c[ph.X] + cs * c[ph.Y]
    ax, ay = _kicks(r, order, k, 0.0)
    want_x = cs * ax - sn * ay                   # R(phi) kick
    want_y = sn * ax + cs * ay
    gx, gy = _kicks(c, order, 0.0, k)
    scale = np.max(np.abs(np.concatenate([gx, gy])))
    assert np.max(np.abs(gx - want_x)) < 1e-12 * scale
    assert np.max(np.abs(gy - want_y)) < 1e-12 * scale


def test_tracking_through_multipoles_is_symplectic():
    # the composed map of thick linear elements and thin multipoles (space
    # charge off) has a symplectic Jacobian at any particle
    lat = bg.fodo_multipole_lattice(2)
    z = np.array([3e-3, 3e-4, -2.4e-3, 1.5e-4, 3e-3, 3e-4])
    t = tr.Tracker(REF, 1e-9, 8, space_charge=False)
    eps = np.array([1e-8, 1e-9, 1e-8, 1e-9, 1e-8, 1e-9])   # central differences, O(eps^2)
    jac = np.zeros((6, 6))
    for j in range(6):
        zp, zm = z.copy(), z.copy()
        zp[j] += eps[j]
        zm[j] -= eps[j]
        jac[:, j] = (t.track(zp[:, None], lat)[:, 0] - t.track(zm[:, None], lat)[:, 0]) / (2 * eps[j])
    s = ph.symplectic_form()
    assert np.max(np.abs(jac.T @ s @ jac - s)) < 1e-8
    # and the nonlinear terms matter at this amplitude
    lin = [e for e in lat if e.kind != ph.MULTIPOLE or e.order <= 2]
    zl = t.track(z[:, None], lin)[:, 0]
    zn = t.track(z[:, None], lat)[:, 0]
    assert np.max(np.abs(zn - zl)) > 3e-5


def test_multipoles_between_slices_and_split_calls():
    lat = bg.fodo_multipole_lattice(3)
    c0 = bg.gaussian6d(100, seed=4)
    t = tr.Tracker(REF, 1e-9, 8, space_charge=False)
    got = t.track(c0, lat)
    # manual: whole elements in beamline order (space charge off)
    c = c0.copy()
    for e in lat:
        if e.kind == ph.MULTIPOLE:
            c = ph.multipole_kick(c, e.order, e.k, e.k2)
        else:
            c = ph.push(c, ph.element_matrix(e.kind, e.length, e.k, e.angle, e.length, REF, e.k2))
    assert np.allclose(got, c, rtol=1e-12, atol=1e-18)
    # split calls: a multipole between the two calls acts once
    t2 = tr.Tracker(REF, 1e-9, 8, space_charge=False)
    half = len(ph.slice_schedule(lat)) // 2
    c2 = t2.track(t2.track(c0, lat, 0, half), lat, half, None)
    assert np.allclose(c2, got, rtol=1e-12, atol=1e-18)


def test_reverse_mode_refuses_multipoles():
    from oracle import adjoint as ad
    with pytest.raises(ValueError):
        ad.forward(bg.gaussian6d(10, seed=1), bg.fodo_multipole_lattice(1), REF, 1e-9, 8)
