"""Pins of the oracle's reverse mode (oracle/adjoint.py) against things other
than itself: sympy derivatives of the closed-form maps and moments, adjoint
identities against the pinned forward solve and field, directional and
central finite differences of the forward tracking (box sequence replayed),
and the bitwise agreement of its forward with track.Tracker."""
from __future__ import annotations

import math

import numpy as np
import pytest
import sympy as sp

import beamgen as bg
from oracle import adjoint as adj
from oracle import physics as ph
from oracle import spacecharge as sc
from oracle import track as tr

REF = ph.RefPart(bg.MASS_PROTON_MEV, 1000.0, 1.0)


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ----------------------------------------------------------- map derivative

@pytest.mark.parametrize("kv", [1.3, -0.7, 0.05, -2.2])
def test_focus_block_dk_matches_sympy(kv):
    k, s = sp.symbols("k s", real=True)
    L = 0.37
    if kv > 0:
        w = sp.sqrt(k)
        blk = sp.Matrix([[sp.cos(w * s), sp.sin(w * s) / w], [-w * sp.sin(w * s), sp.cos(w * s)]])
    else:
        w = sp.sqrt(-k)
        blk = sp.Matrix([[sp.cosh(w * s), sp.sinh(w * s) / w], [w * sp.sinh(w * s), sp.cosh(w * s)]])
    want = np.array(blk.diff(k).subs({k: kv, s: L}).evalf(30), dtype=float)
    got = adj._focus_block_dk(L, kv)
    assert np.allclose(got, want, rtol=1e-13, atol=1e-15)


def test_element_dk_against_map_differences():
    ds = 0.25
    for kv in (1.0, -1.0, 0.0):
        h = 1e-6
        fd = (ph.element_matrix(ph.QUAD, 1.0, kv + h, 0.0, ds, REF)
              - ph.element_matrix(ph.QUAD, 1.0, kv - h, 0.0, ds, REF)) / (2 * h)
        got = adj.element_matrix_dk(ph.QUAD, ds, kv)
        assert np.allclose(got, fd, rtol=1e-7, atol=1e-9)
    assert not np.any(adj.element_matrix_dk(ph.DRIFT, ds, 0.0))
    assert not np.any(adj.element_matrix_dk(ph.SBEND, ds, 0.0))


# --------------------------------------------------------------- objectives

def test_objectives_adjoint_matches_sympy_on_tiny_bunch():
    rng = bg.standard_normal6(5, seed=11) * 1e-3
    zs = sp.Matrix(6, 5, lambda i, j: sp.Symbol(f"z{i}_{j}"))
    n = 5

    def cov(a, b):
        ma = sum(zs[a, j] for j in range(n)) / n
        mb = sum(zs[b, j] for j in range(n)) / n
        return sum((zs[a, j] - ma) * (zs[b, j] - mb) for j in range(n)) / n

    objs = [sp.sqrt(cov(0, 0) * cov(1, 1) - cov(0, 1) ** 2),
            sp.sqrt(cov(2, 2) * cov(3, 3) - cov(2, 3) ** 2),
            sp.sqrt(cov(0, 0)), sp.sqrt(cov(2, 2))]
    subs = {zs[i, j]: sp.Float(rng[i, j], 30) for i in range(6) for j in range(n)}
    for oi in range(4):
        w = np.zeros(4)
        w[oi] = 1.0
        got = adj.objectives_adjoint(rng, w)
        want = np.array([[float(sp.diff(objs[oi], zs[i, j]).subs(subs)) for j in range(n)]
                         for i in range(6)])
        assert _rel(got, want) < 1e-12
    assert np.allclose(adj.objectives(rng), [float(o.subs(subs)) for o in objs], rtol=1e-13)


# ------------------------------------------------------- adjoint identities

def test_solve_adjoint_identity():
    n = 8
    rng = np.random.default_rng(4)
    h = (1.1e-3, 0.9e-3, 2.3e-3)
    ghat = sc.green_hat(n, h)
    rho = rng.standard_normal((n, n, n))
    phibar = rng.standard_normal((n + 2,) * 3)
    lhs = float(np.sum(sc.solve(rho, h, ghat) * phibar))
    rhs = float(np.sum(rho * adj.solve_adjoint(phibar, ghat, n)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_solve_adjoint_matches_direct_sum():
    # rhobar_j = sum_i G(i - j) phibar_i over nodes i = -1..n: the transpose
    # written out with the IGF octant table (brute force, G even)
    n = 4
    h = (1e-3, 1.5e-3, 0.8e-3)
    rng = np.random.default_rng(5)
    phibar = rng.standard_normal((n + 2,) * 3)
    oct_ = sc.igf_octant(n, h)
    want = np.zeros((n, n, n))
    nodes = np.arange(-1, n + 1)
    for l in range(n):
        for j in range(n):
            for i in range(n):
                g = oct_[np.ix_(np.abs(nodes - l), np.abs(nodes - j), np.abs(nodes - i))]
                want[l, j, i] = np.sum(g * phibar)
    got = adj.solve_adjoint(phibar, sc.green_hat(n, h), n)
    assert _rel(got, want) < 1e-13


def test_field_adjoint_identity():
    n = 6
    rng = np.random.default_rng(6)
    h = (1e-3, 2e-3, 3e-3)
    phi = rng.standard_normal((n + 2,) * 3)
    ebar = rng.standard_normal((3, n, n, n))
    lhs = float(np.sum(sc.field(phi, h) * ebar))
    rhs = float(np.sum(phi * adj.field_adjoint(ebar, h)))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


# ----------------------------------------------- kick: directional derivative

def _kick_fixed(a, box, ghat, q, ds, n):
    pos = sc.rest_frame(a, REF)
    h = box.h(n)
    phi = sc.solve(sc.deposit(pos, q, box, n), h, ghat)
    return sc.kick(a, sc.gather(pos, sc.field(phi, h), box), ds, REF)


def test_kick_adjoint_directional_derivative():
    n = 8
    a = bg.gaussian6d(300, seed=7)
    box, _ = sc.box_rule(sc.rest_frame(a, REF), None)
    h = box.h(n)
    ghat = sc.green_hat(n, h)
    q = sc.macro_charge(50e-9, a.shape[1], REF)
    ds = 0.5
    r = adj.Record()
    r.a, r.box, r.h, r.ghat, r.q, r.ds = a, box, h, ghat, q, ds
    pos = sc.rest_frame(a, REF)
    r.efield = sc.field(sc.solve(sc.deposit(pos, q, box, n), h, ghat), h)
    rng = np.random.default_rng(8)
    bbar = rng.standard_normal(a.shape)
    abar = adj.kick_adjoint(r, bbar, REF, n)
    for trial in range(3):
        v = rng.standard_normal(a.shape) * np.array([1e-3, 1e-4, 1e-3, 1e-4, 1e-3, 1e-4])[:, None]
        eps = 1e-7   # moves particles by ~1e-10 m: no cell boundary crossed
        fp = _kick_fixed(a + eps * v, box, ghat, q, ds, n)
        fm = _kick_fixed(a - eps * v, box, ghat, q, ds, n)
        fd = float(np.sum(bbar * (fp - fm))) / (2 * eps)
        ad = float(np.sum(abar * v))
        assert abs(fd - ad) <= 1e-7 * abs(ad)
    # the position terms matter: drop the momentum pass-through and compare
    # the position part alone
    pos_part = abar - bbar
    assert np.max(np.abs(pos_part[[0, 2, 4]])) > 1e-3 * np.max(np.abs(bbar))


# ------------------------------------------------------------ whole tracking

def test_forward_matches_tracker_bitwise_and_replays():
    lat = bg.fodo8_lattice(bg.KS_FODO8, periods=1, nslice=1)
    z0 = bg.gaussian6d(500, seed=2)
    t = tr.Tracker(REF, 20e-9, 8)
    want = t.track(z0, lat)
    zf, recs, boxes = adj.forward(z0, lat, REF, 20e-9, 8)
    assert np.array_equal(zf, want)
    assert len(recs) == 20 and len(boxes) == 20
    zf2, _, boxes2 = adj.forward(z0, lat, REF, 20e-9, 8, boxes=boxes)
    assert np.array_equal(zf2, want) and boxes2 == boxes


def _fd_twiss_and_k(xi, twiss, ks, charge, n, weights, boxes, h_rel=1e-6, space_charge=True):
    def f(tw, kk):
        lat = bg.fodo8_lattice(kk, periods=1, nslice=1)
        z0 = adj.twiss_bunch(xi, tw)
        zf, _, _ = adj.forward(z0, lat, REF, charge, n, boxes=boxes, space_charge=space_charge)
        return float(np.dot(weights, adj.objectives(zf)))
    dk = np.zeros(8)
    for i in range(8):
        kp, km = list(ks), list(ks)
        d = h_rel * abs(ks[i])
        kp[i] += d
        km[i] -= d
        dk[i] = (f(twiss, kp) - f(twiss, km)) / (2 * d)
    dt = np.zeros(6)
    for i in range(6):
        tp, tm = list(twiss), list(twiss)
        d = h_rel * abs(twiss[i])
        tp[i] += d
        tm[i] -= d
        dt[i] = (f(tp, ks) - f(tm, ks)) / (2 * d)
    return dk, dt


def _family_sum(lat, dk_elem):
    fam = bg.fodo8_families(lat)
    out = np.zeros(8)
    for i, f in enumerate(fam):
        if f >= 0:
            out[f] += dk_elem[i]
    return out


def test_twiss_gradient_through_drift_closed_form():
    # after a drift of length L (no space charge), x = A xi_x + B xi_px with
    # A = sqrt(eps beta) - L alpha sqrt(eps/beta), B = L sqrt(eps/beta); sigma_x
    # and eps_x follow from the sample second moments of xi in closed form
    xi = bg.standard_normal6(3000, seed=3)
    twiss = (-0.8, 3.0, 2e-7, 0.5, 1.5, 3e-7, 1e-3, 1e-4)
    L = 1.7
    lat = [bg.drift(L, 4)]
    S = np.cov(xi[:2], bias=True)
    a, b, e = sp.symbols("a b e", real=True)
    A = sp.sqrt(e * b) - L * a * sp.sqrt(e / b)
    B = L * sp.sqrt(e / b)
    sig = sp.sqrt(A ** 2 * S[0, 0] + 2 * A * B * S[0, 1] + B ** 2 * S[1, 1])
    eps = e * sp.sqrt(S[0, 0] * S[1, 1] - S[0, 1] ** 2)   # drift preserves it
    at = {a: twiss[0], b: twiss[1], e: twiss[2]}
    for w, expr in (((0, 0, 1, 0), sig), ((1, 0, 0, 0), eps)):
        g = adj.gradients(xi, twiss, lat, REF, 0.0, 8, w, space_charge=False)
        want = [float(sp.diff(expr, v).subs(at)) for v in (a, b, e)]
        assert np.allclose(g["dtwiss"][:3], want, rtol=1e-10, atol=1e-14 * max(map(abs, want)))
        assert np.all(g["dtwiss"][3:] == 0.0)


def test_gradients_no_space_charge_match_central_differences():
    xi = bg.standard_normal6(400, seed=9)
    ks = [1.1, -0.9, 1.0, -1.05, 0.95, -1.0, 1.02, -0.97]
    lat = bg.fodo8_lattice(ks, periods=1, nslice=1)
    w = np.array([0.3, -0.5, 1.0, 0.7])
    g = adj.gradients(xi, bg.TWISS_FODO, lat, REF, 0.0, 8, w, space_charge=False)
    dk_fd, dt_fd = _fd_twiss_and_k(xi, bg.TWISS_FODO, ks, 0.0, 8, w, None, space_charge=False)
    assert _rel(_family_sum(lat, g["dk"]), dk_fd) < 1e-7
    assert _rel(g["dtwiss"], dt_fd) < 1e-7


@pytest.mark.slow
def test_gradients_space_charge_match_central_differences_box_replayed():
    xi = bg.standard_normal6(400, seed=10)
    ks = list(bg.KS_FODO8)
    lat = bg.fodo8_lattice(ks, periods=1, nslice=1)
    charge, n = 30e-9, 8
    w = np.array([1.0, 0.5, -0.8, 0.25])
    g = adj.gradients(xi, bg.TWISS_FODO, lat, REF, charge, n, w)
    dk_fd, dt_fd = _fd_twiss_and_k(xi, bg.TWISS_FODO, ks, charge, n, w, g["boxes"])
    dk = _family_sum(lat, g["dk"])
    assert _rel(dk, dk_fd) < 1e-6
    assert _rel(g["dtwiss"], dt_fd) < 1e-6
    # space charge changes the gradient well above the tolerance
    g0 = adj.gradients(xi, bg.TWISS_FODO, lat, REF, 0.0, n, w, space_charge=False)
    assert _rel(_family_sum(lat, g0["dk"]), dk) > 1e-3


def test_gradients_through_thin_elements_match_central_differences():
    # a FODO with thin edges between its elements (no space charge):
    # the reverse sweep passes the thin maps transposed
    xi = bg.standard_normal6(300, seed=12)
    ks = [1.1, -0.9, 1.0, -1.05, 0.95, -1.0, 1.02, -0.97]

    def lattice(kk):
        lat = []
        for e in bg.fodo8_lattice(kk, periods=1, nslice=2):
            lat += [e, bg.dipedge(0.02, 0.3)]
        return lat

    w = np.array([0.3, -0.5, 1.0, 0.7])
    lat = lattice(ks)
    g = adj.gradients(xi, bg.TWISS_FODO, lat, REF, 0.0, 8, w, space_charge=False)
    fam = bg.fodo8_families([e for e in lat if e.kind != bg.DIPEDGE])
    # family index per element of `lat` (edges have none)
    fam_full = []
    it = iter(fam)
    for e in lat:
        fam_full.append(-1 if e.kind == bg.DIPEDGE else next(it))
    dk = np.zeros(8)
    for i, f in enumerate(fam_full):
        if f >= 0:
            dk[f] += g["dk"][i]

    def f(kk):
        zf, _, _ = adj.forward(adj.twiss_bunch(xi, bg.TWISS_FODO), lattice(kk), REF, 0.0, 8,
                               space_charge=False)
        return float(np.dot(w, adj.objectives(zf)))

    for i in (0, 5):
        kp, km = list(ks), list(ks)
        kp[i] += 1e-6
        km[i] -= 1e-6
        fd = (f(kp) - f(km)) / 2e-6
        assert abs(fd - dk[i]) <= 1e-7 * np.max(np.abs(dk))
