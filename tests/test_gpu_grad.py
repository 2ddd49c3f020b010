"""GPU reverse mode (bx_grad_* through the C ABI) against the oracle's reverse
mode and against central finite differences of the GPU forward with the box
sequence replayed.

Tolerances: the gradients agree with the oracle's to 1e-9 relative (of each
gradient vector's largest entry): the forward states agree to ~1e-12 and the
reverse adds the fixed-point scatter (resolution below 2^-40 of its largest
value) and FP64 rounding.  Central finite differences agree to 1e-6
relative at h = 1e-8 relative.  The tracked function is only piecewise
smooth (a CIC weight's derivative jumps when a particle crosses a cell face):
with a few thousand particles a step of 1e-6 straddles such crossings, and on
this case the oracle's own central differences miss its exact reverse-mode
gradient by 2.5e-5 at h = 1e-6, 5e-6 at 1e-7 and 7e-9 at 1e-8; the
round-off of f / h stays near 1e-10 at 1e-8."""
import numpy as np
import pytest
import torch

import beamgen as bg
from oracle import adjoint as adj
from tests.parity import coord_rel_err, oracle_ref

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SPECIES = bg.PROTON_1GEV
KS = [1.05, -0.95, 1.0, -1.02, 0.97, -1.0, 1.03, -0.98]
GRAD_TOL = 1e-9
FD_TOL = 1e-6


@pytest.fixture(scope="module")
def bt():
    import paper_2208_02382_b300 as p
    from paper_2208_02382_b300 import build
    build.build()
    return p


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _family_sum(lat, dk):
    fam = bg.fodo8_families(lat)
    out = np.zeros(8)
    for i, f in enumerate(fam):
        if f >= 0:
            out[f] += dk[i]
    return out


def _setup(bt, npart, n, periods, charge, seed=3):
    xi = bg.standard_normal6(npart, seed=seed)
    lat = bg.fodo8_lattice(KS, periods=periods, nslice=1)
    sp = bt.Species(SPECIES.mass_MeV, SPECIES.kinetic_MeV, SPECIES.charge_sign)
    xi_t = torch.tensor(xi, dtype=torch.float64, device=DEV)
    return xi, xi_t, lat, sp


def _gpu_grad(bt, trk, xi_t, lat, sp, charge, w, C, replay=None, space_charge=True):
    coords = bt.twiss_beam(bg.TWISS_FODO, xi_t)
    beam = bt.Beam(coords, sp, charge)
    trk.grad_forward(beam, lat, C, box_replay=replay, space_charge=space_charge)
    # the recording forward re-bins the particles: compare in id order
    order = np.argsort(beam.ids.cpu().numpy())
    final = beam.coords.cpu().numpy()[:, order]
    boxes = trk.grad_boxes()
    dk, S, zb = trk.grad_backward(beam, w)
    dtw = bt.twiss_grad(bg.TWISS_FODO, S)
    return {"dk": np.array(dk), "S": np.array(S), "dtwiss": np.array(dtw),
            "zbar0": zb.cpu().numpy()[:, order], "final": final, "boxes": boxes}


@pytest.mark.parametrize("space_charge", [True, False])
def test_gradients_match_oracle_reverse_mode(bt, space_charge):
    npart, n, charge = 3001, 16, 10e-9
    xi, xi_t, lat, sp = _setup(bt, npart, n, 1, charge)
    w = np.array([1.0, 0.5, -0.8, 0.25])
    trk = bt.Tracker(n)
    g = _gpu_grad(bt, trk, xi_t, lat, sp, charge, w, C=6, space_charge=space_charge)
    ref = oracle_ref(SPECIES)
    o = adj.gradients(xi, bg.TWISS_FODO, lat, ref, charge, n, w, space_charge=space_charge)
    assert coord_rel_err(g["final"], o["zf"]) < 1e-11
    if space_charge:
        ob = np.array([[*b.lo, *b.hi] for b in o["boxes"]])
        gb = np.array([row[:6] for row in g["boxes"]])
        assert np.max(np.abs(gb - ob) / np.abs(ob).max(axis=0)) < 1e-12
    e_dk = _rel(g["dk"], o["dk"])
    e_tw = _rel(g["dtwiss"], o["dtwiss"])
    e_z = max(_rel(g["zbar0"][r], o["zbar0"][r]) for r in range(6) if np.any(o["zbar0"][r]))
    print(f"rel err dk {e_dk:.2e} dtwiss {e_tw:.2e} zbar0 {e_z:.2e}")
    assert e_dk < GRAD_TOL and e_tw < GRAD_TOL and e_z < GRAD_TOL


def test_gradients_match_central_differences_box_replayed(bt):
    npart, n, charge = 4000, 16, 10e-9
    xi, xi_t, lat, sp = _setup(bt, npart, n, 1, charge, seed=5)
    w = np.array([0.7, -0.3, 1.0, 0.4])
    trk = bt.Tracker(n)
    g = _gpu_grad(bt, trk, xi_t, lat, sp, charge, w, C=7)
    dk = _family_sum(lat, g["dk"])
    fd_trk = bt.Tracker(n)

    def f(ks, tw):
        els = bg.fodo8_lattice(ks, periods=1, nslice=1)
        beam = bt.Beam(bt.twiss_beam(tw, xi_t), sp, charge)
        fd_trk.grad_forward(beam, els, 20, box_replay=g["boxes"])
        m = fd_trk.moments(beam).cpu().numpy()
        obj = [np.sqrt(m[6] * m[12] - m[7] ** 2), np.sqrt(m[17] * m[21] - m[18] ** 2),
               np.sqrt(m[6]), np.sqrt(m[17])]
        return float(np.dot(w, obj))

    h = 1e-8
    for i in (0, 3, 6):
        kp, km = list(KS), list(KS)
        kp[i] += h * abs(KS[i])
        km[i] -= h * abs(KS[i])
        fd = (f(kp, bg.TWISS_FODO) - f(km, bg.TWISS_FODO)) / (2 * h * abs(KS[i]))
        assert abs(fd - dk[i]) <= FD_TOL * np.max(np.abs(dk)), (i, fd, dk[i])
    for i in (0, 1, 2, 4):
        tp, tm = list(bg.TWISS_FODO), list(bg.TWISS_FODO)
        d = h * abs(bg.TWISS_FODO[i])
        tp[i] += d
        tm[i] -= d
        fd = (f(KS, tp) - f(KS, tm)) / (2 * d)
        assert abs(fd - g["dtwiss"][i]) <= FD_TOL * np.max(np.abs(g["dtwiss"][:3])), (i, fd)


def test_gradients_independent_of_checkpoint_interval_and_reproducible(bt):
    # the recording forward re-bins the bunch at every checkpoint, so another
    # interval means another particle order and FP64 sums in another order:
    # equal to rounding; the same interval twice is bitwise the same
    npart, n, charge = 2000, 16, 10e-9
    xi, xi_t, lat, sp = _setup(bt, npart, n, 1, charge, seed=7)
    w = np.array([1.0, 1.0, 1.0, 1.0])
    trk = bt.Tracker(n)
    runs = [_gpu_grad(bt, trk, xi_t, lat, sp, charge, w, C=c) for c in (1, 7, 20, 20)]
    for r in runs[1:3]:
        assert _rel(r["dk"], runs[0]["dk"]) < 1e-12
        assert _rel(r["S"], runs[0]["S"]) < 1e-12
        assert max(_rel(r["zbar0"][q], runs[0]["zbar0"][q]) for q in range(6)) < 1e-12
        assert np.array_equal(r["final"], runs[0]["final"])
    for key in ("dk", "S", "zbar0", "final"):
        assert np.array_equal(runs[3][key], runs[2][key])


def test_autograd_function(bt):
    npart, n, charge = 2000, 16, 10e-9
    xi, xi_t, lat, sp = _setup(bt, npart, n, 1, charge, seed=9)
    fam = bg.fodo8_families(lat).tolist()
    els = [bt.Element(e.kind, e.length, e.k, e.angle, e.nslice) for e in lat]
    ks = torch.tensor(KS, dtype=torch.float64, requires_grad=True)
    tw = torch.tensor(bg.TWISS_FODO, dtype=torch.float64, requires_grad=True)
    trk = bt.Tracker(n)
    obj = bt.track_objectives(ks, tw, xi_t, trk, els, fam, sp, charge, 5)
    w = torch.tensor([0.2, 0.4, -1.0, 0.3], dtype=torch.float64)
    (obj * w).sum().backward()
    ref = oracle_ref(SPECIES)
    o = adj.gradients(xi, bg.TWISS_FODO, lat, ref, charge, n, w.numpy())
    assert np.allclose(obj.detach().numpy(), o["obj"], rtol=1e-11)
    assert _rel(ks.grad.numpy(), _family_sum(lat, o["dk"])) < GRAD_TOL
    assert _rel(tw.grad.numpy()[:6], o["dtwiss"]) < GRAD_TOL
    assert np.all(tw.grad.numpy()[6:] == 0.0)
