"""Reverse-mode derivatives of the tracking step with space charge, and the
Twiss-parametrised initial bunch.

Oracle (test infrastructure only; see oracle/__init__.py).

Paper anchors (arXiv:2208.02382): §Introduction and §Outlook motivate a code
that can be coupled to machine-learning workflows (differentiable modelling);
the paper gives no adjoint.  What is differentiated is the tracking of
track.Tracker: per slice map(ds/2) -> space-charge kick over ds -> map(ds/2)
(§Model Assumptions), objectives the rms beam size and unnormalised rms
emittance of the final bunch (§Benchmark FODO / IOTA observables).  Every
reverse step below is the transpose of the Jacobian of the forward step it
names, derived by hand from that forward step:

  * map z' = H z                 -> zbar = H^T zbar',  Hbar += zbar' z^T
  * kick p' = p + c * E(X)       -> pbar = pbar';  Ebar_node += w * c pbar'
                                    (scatter) and Xbar += c pbar' . dE/dX with
                                    the CIC weight derivatives (gather term)
  * field E = -D phi             -> phibar = -D^T Ebar
  * solve phi = crop C pad rho   -> rhobar = pad^T C^T crop^T phibar; the
                                    circulant C of the even doubled Green's
                                    function is symmetric
  * deposit rho = (q/V) sum w    -> Xbar += (q/V) sum_nodes rhobar dw/dX
  * rest frame X = x, Y = y, Z = -beta gamma t

Reading (the paper is silent): the grid box is piecewise constant in the
particle coordinates (it changes only at a regrid, as a function of the extreme
particles), and the reverse treats the box sequence of a run as fixed.  The
function whose exact derivative this is, is tracking with that box sequence
replayed (forward(..., boxes=recorded)); finite differences are taken on it.
"""
from __future__ import annotations

import math

import numpy as np

from . import physics as ph
from . import spacecharge as sc
from . import track as tr
from .physics import PT, PX, PY, T, X, Y

# ----------------------------------------------------------- initial bunch


def twiss_bunch(xi: np.ndarray, twiss) -> np.ndarray:
    """Initial bunch from standard-normal draws xi (6, n) and the Twiss
    parametrisation of each transverse plane (Courant-Snyder):

        u  = sqrt(eps beta) xi_u
        pu = sqrt(eps / beta) (xi_pu - alpha xi_u)

    twiss = (alpha_x, beta_x, eps_x, alpha_y, beta_y, eps_y, sigma_t, sigma_pt);
    t = sigma_t xi_t, pt = sigma_pt xi_pt (longitudinal plane held fixed)."""
    ax, bx, ex, ay, by, ey, st, spt = (float(v) for v in twiss)
    z = np.empty_like(xi, dtype=np.float64)
    z[X] = math.sqrt(ex * bx) * xi[X]
    z[PX] = math.sqrt(ex / bx) * (xi[PX] - ax * xi[X])
    z[Y] = math.sqrt(ey * by) * xi[Y]
    z[PY] = math.sqrt(ey / by) * (xi[PY] - ay * xi[Y])
    z[T] = st * xi[T]
    z[PT] = spt * xi[PT]
    return z


def twiss_grad(zbar0: np.ndarray, xi: np.ndarray, twiss) -> np.ndarray:
    """dL/d(alpha_x, beta_x, eps_x, alpha_y, beta_y, eps_y) from dL/dz0, by the
    chain rule through twiss_bunch (its derivatives written out per term)."""
    out = np.zeros(6)
    for plane, (u, pu) in enumerate(((X, PX), (Y, PY))):
        a, b, e = (float(v) for v in twiss[3 * plane:3 * plane + 3])
        xu, xp = xi[u], xi[pu]
        # d u / d(alpha, beta, eps)
        du = (np.zeros_like(xu), 0.5 * math.sqrt(e / b) * xu, 0.5 * math.sqrt(b / e) * xu)
        # d pu / d(alpha, beta, eps)
        dpu = (-math.sqrt(e / b) * xu,
               -0.5 * math.sqrt(e) * b ** -1.5 * (xp - a * xu),
               0.5 / math.sqrt(e * b) * (xp - a * xu))
        for j in range(3):
            out[3 * plane + j] = float(np.sum(zbar0[u] * du[j]) + np.sum(zbar0[pu] * dpu[j]))
    return out


# -------------------------------------------------------------- objectives

OBJECTIVES = ("eps_x", "eps_y", "sigma_x", "sigma_y")


def objectives(z: np.ndarray) -> np.ndarray:
    """(eps_x, eps_y, sigma_x, sigma_y) of the bunch (track.moments)."""
    m = tr.moments(z)
    return np.array([m["eps_x"], m["eps_y"], m["sigma"][X], m["sigma"][Y]])


def objectives_adjoint(z: np.ndarray, weights) -> np.ndarray:
    """dL/dz for L = sum_i weights[i] * objectives(z)[i].

    With d = z - <z> and C the centred second moments (1/n normalisation),
    dC_ab/dz_a,p = d_b,p / n (the mean terms cancel because sum_p d = 0), so
        d sigma_u / d u_p        = d_u,p / (n sigma_u)
        d eps_u / d u_p          = (C_pp d_u,p - C_up d_pu,p) / (n eps_u)
        d eps_u / d pu_p         = (C_uu d_pu,p - C_up d_u,p) / (n eps_u)."""
    n = z.shape[1]
    m = tr.moments(z)
    d = z - m["mean"][:, None]
    cov = m["cov"]
    zbar = np.zeros_like(z)
    w = [float(v) for v in weights]
    for i, (u, pu) in enumerate(((X, PX), (Y, PY))):
        eps = math.sqrt(cov[u, u] * cov[pu, pu] - cov[u, pu] ** 2)
        if w[i] != 0.0:
            zbar[u] += w[i] * (cov[pu, pu] * d[u] - cov[u, pu] * d[pu]) / (n * eps)
            zbar[pu] += w[i] * (cov[u, u] * d[pu] - cov[u, pu] * d[u]) / (n * eps)
        if w[2 + i] != 0.0:
            zbar[u] += w[2 + i] * d[u] / (n * math.sqrt(cov[u, u]))
    return zbar


# ------------------------------------------------------ map derivatives


def _focus_block_dk(ds: float, k: float) -> np.ndarray:
    """d/dk of the 2x2 block of u'' = -k u over ds (physics._focus_block)."""
    if k > 0.0:
        w = math.sqrt(k)
        c, s = math.cos(w * ds), math.sin(w * ds)
        dw = 0.5 / w
        # d/dw of [[c, s/w], [-w s, c]]
        dm = np.array([[-ds * s, (ds * c * w - s) / (w * w)],
                       [-s - w * ds * c, -ds * s]])
        return dm * dw
    if k < 0.0:
        w = math.sqrt(-k)
        c, s = math.cosh(w * ds), math.sinh(w * ds)
        dw = -0.5 / w
        # d/dw of [[c, s/w], [w s, c]]
        dm = np.array([[ds * s, (ds * c * w - s) / (w * w)],
                       [s + w * ds * c, ds * s]])
        return dm * dw
    # k = 0: first-order Taylor term of the block in k
    return np.array([[-ds * ds / 2.0, -ds ** 3 / 6.0], [-ds, -ds * ds / 2.0]])


def element_matrix_dk(kind: int, ds: float, k: float) -> np.ndarray:
    """d/dk of physics.element_matrix for a piece ds (quadrupole only; other
    elements do not depend on k)."""
    m = np.zeros((6, 6))
    if kind == ph.QUAD:
        m[X:X + 2, X:X + 2] = _focus_block_dk(ds, k)
        m[Y:Y + 2, Y:Y + 2] = -_focus_block_dk(ds, -k)
    return m


# ------------------------------------------------------------------ forward


class Record:
    """What the reverse needs of one kick: element, slice length, half map,
    the coordinates before the first half map (z_in), before the kick (a) and
    after it (b), the box, cell size, Green's spectrum and node field."""
    __slots__ = ("ie", "ds", "half", "z_in", "a", "b", "box", "h", "ghat", "efield", "q", "pre")


def forward(z0: np.ndarray, lattice, ref: ph.RefPart, bunch_charge_C: float, n_grid: int,
            boxes=None, space_charge: bool = True):
    """The tracking of track.Tracker over the whole lattice, step for step the
    same calls, keeping a Record per kick.  With `boxes` (one sc.Box per kick)
    the box of each kick is taken from the list instead of the box rule
    (replay).  Returns (final coordinates, records, boxes used)."""
    if any(ph.is_thin(e) and not ph.is_linear_thin(e) for e in lattice):
        raise ValueError("reverse mode: thin multipoles are not supported (linear thin "
                         "elements only)")
    sched = ph.slice_schedule(lattice)
    before, after = ph.thin_schedule(lattice)
    c = np.array(z0, dtype=np.float64, copy=True)
    npart = c.shape[1]
    q = sc.macro_charge(bunch_charge_C, npart, ref)
    box, ghat, ghat_h = None, None, None
    recs, used = [], []
    for k, (ie, ds) in enumerate(sched):
        e = lattice[ie]
        pre = ph.thin_matrix(lattice, before[k], ref)
        for it in before[k]:
            c = ph.push(c, ph.thin_matrix(lattice, [it], ref))
        half = ph.element_matrix(e.kind, e.length, e.k, e.angle, 0.5 * ds, ref,
                                 getattr(e, "k2", 0.0))
        r = Record()
        r.ie, r.ds, r.half, r.z_in, r.pre = ie, ds, half, c, pre
        c = ph.push(c, half)
        r.a = c
        if space_charge:
            pos = sc.rest_frame(c, ref)
            if boxes is None:
                box, _ = sc.box_rule(pos, box)
            else:
                box = boxes[k]
            h = box.h(n_grid)
            if ghat is None or ghat_h != h:
                ghat, ghat_h = sc.green_hat(n_grid, h), h
            rho = sc.deposit(pos, q, box, n_grid)
            phi = sc.solve(rho, h, ghat)
            ef = sc.field(phi, h)
            c = sc.kick(c, sc.gather(pos, ef, box), ds, ref)
            r.box, r.h, r.ghat, r.efield, r.q = box, h, ghat, ef, q
            used.append(box)
        r.b = c
        c = ph.push(c, half)
        recs.append(r)
    for it in after:
        c = ph.push(c, ph.thin_matrix(lattice, [it], ref))
    return c, recs, used


# ------------------------------------------------------------------ reverse


def solve_adjoint(phibar: np.ndarray, ghat: np.ndarray, n: int) -> np.ndarray:
    """Transpose of spacecharge.solve: phibar on nodes -1..n ((n+2)^3, index =
    node + 1) -> rhobar on nodes 0..n-1.  solve is crop(C(pad(rho))) with C
    the circulant of the doubled Green's function (symmetric, G even); its
    transpose is pad^T C crop^T: place phibar at (node mod 2n), apply C,
    keep nodes 0..n-1."""
    m = 2 * n
    full = np.zeros((m, m, m))
    k = np.arange(-1, n + 1) % m
    full[np.ix_(k, k, k)] += phibar
    conv = np.fft.irfftn(np.fft.rfftn(full) * ghat, s=(m, m, m), axes=(0, 1, 2))
    return conv[:n, :n, :n].copy()


def field_adjoint(ebar: np.ndarray, h) -> np.ndarray:
    """Transpose of spacecharge.field: ebar (3, n, n, n) -> phibar (n+2)^3.
    E_x[l, j, i] = -(phi[l+1, j+1, i+2] - phi[l+1, j+1, i]) / (2 h_x), etc."""
    n = ebar.shape[1]
    pb = np.zeros((n + 2,) * 3)
    pb[1:-1, 1:-1, 2:] -= ebar[0] / (2.0 * h[0])
    pb[1:-1, 1:-1, :-2] += ebar[0] / (2.0 * h[0])
    pb[1:-1, 2:, 1:-1] -= ebar[1] / (2.0 * h[1])
    pb[1:-1, :-2, 1:-1] += ebar[1] / (2.0 * h[1])
    pb[2:, 1:-1, 1:-1] -= ebar[2] / (2.0 * h[2])
    pb[:-2, 1:-1, 1:-1] += ebar[2] / (2.0 * h[2])
    return pb


def kick_adjoint(r: Record, bbar: np.ndarray, ref: ph.RefPart, n: int) -> np.ndarray:
    """abar from bbar for the space-charge kick of record r (box fixed)."""
    pos = sc.rest_frame(r.a, ref)
    (i, j, l), (fx, fy, fz) = sc.cic_cells(pos, r.box, n)
    h = r.h
    w = ((1.0 - fx, fx), (1.0 - fy, fy), (1.0 - fz, fz))
    dw = (-1.0, 1.0)                       # d w / d f for the lower and upper node
    s = ref.charge_sign
    kt = s * r.ds / (ref.mass_eV * ref.betagamma ** 2)
    kz = -s * r.ds / (ref.mass_eV * ref.betagamma)
    # adjoint of the field at each particle
    eat_bar = np.stack([kt * bbar[PX], kt * bbar[PY], kz * bbar[PT]])
    abar = bbar.copy()
    posbar = np.zeros_like(pos)
    ebar = np.zeros((3, n, n, n))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                node = (l + dz, j + dy, i + dx)
                wgt = w[0][dx] * w[1][dy] * w[2][dz]
                # gather transpose: scatter of the field adjoint
                for cc in range(3):
                    np.add.at(ebar[cc], node, wgt * eat_bar[cc])
                # gather's dependence on the particle position
                g = sum(eat_bar[cc] * r.efield[cc][node] for cc in range(3))
                posbar[0] += g * dw[dx] * w[1][dy] * w[2][dz] / h[0]
                posbar[1] += g * w[0][dx] * dw[dy] * w[2][dz] / h[1]
                posbar[2] += g * w[0][dx] * w[1][dy] * dw[dz] / h[2]
    rhobar = solve_adjoint(field_adjoint(ebar, h), r.ghat, n)
    qv = r.q / (h[0] * h[1] * h[2])
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                rb = qv * rhobar[l + dz, j + dy, i + dx]
                posbar[0] += rb * dw[dx] * w[1][dy] * w[2][dz] / h[0]
                posbar[1] += rb * w[0][dx] * dw[dy] * w[2][dz] / h[1]
                posbar[2] += rb * w[0][dx] * w[1][dy] * dw[dz] / h[2]
    abar[X] += posbar[0]
    abar[Y] += posbar[1]
    abar[T] += -ref.betagamma * posbar[2]
    return abar


def reverse(recs, zbar: np.ndarray, lattice, ref: ph.RefPart, n_grid: int,
            space_charge: bool = True):
    """Backward sweep over the records.  Returns (dL/dz0, dL/dk per lattice
    element index, dL/dH per kick (list of 6x6))."""
    dk = np.zeros(len(lattice))
    hbars = [None] * len(recs)
    zb = np.array(zbar, dtype=np.float64, copy=True)
    _, after = ph.thin_schedule(lattice)
    zb = ph.thin_matrix(lattice, after, ref).T @ zb      # thin elements past the last slice
    for idx in range(len(recs) - 1, -1, -1):
        r = recs[idx]
        H = r.half
        hbar = zb @ r.b.T                  # second half map, input b
        bbar = H.T @ zb
        abar = kick_adjoint(r, bbar, ref, n_grid) if space_charge else bbar
        hbar = hbar + abar @ r.z_in.T      # first half map, input z_in
        zb = r.pre.T @ (H.T @ abar)        # then the thin elements before the slice
        hbars[idx] = hbar
        e = lattice[r.ie]
        dk[r.ie] += float(np.sum(hbar * element_matrix_dk(e.kind, 0.5 * r.ds, e.k)))
    return zb, dk, hbars


def gradients(xi: np.ndarray, twiss, lattice, ref: ph.RefPart, bunch_charge_C: float,
              n_grid: int, weights, space_charge: bool = True, boxes=None):
    """Objectives and their gradients for the bunch twiss_bunch(xi, twiss):
    returns dict(obj, dk (per element), dtwiss (6), zbar0, boxes)."""
    z0 = twiss_bunch(xi, twiss)
    zf, recs, used = forward(z0, lattice, ref, bunch_charge_C, n_grid, boxes=boxes,
                             space_charge=space_charge)
    zbar = objectives_adjoint(zf, weights)
    zbar0, dk, _ = reverse(recs, zbar, lattice, ref, n_grid, space_charge)
    return {"obj": objectives(zf), "dk": dk, "dtwiss": twiss_grad(zbar0, xi, twiss),
            "zbar0": zbar0, "boxes": used, "z0": z0, "zf": zf}
