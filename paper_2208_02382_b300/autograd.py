"""torch.autograd binding of the reverse-mode tracking (libbeamtrack's
bx_grad_* calls): objectives of the final bunch as a differentiable function
of the quadrupole strengths and the initial Twiss parameters.  Argument
marshalling only; the forward tracking, the checkpoint recomputation and every
reverse step run in the library's CUDA kernels."""
from __future__ import annotations

import torch

from . import api


class TrackObjectives(torch.autograd.Function):
    """(eps_x, eps_y, sigma_x, sigma_y) of the bunch after tracking
    twiss_beam(twiss, xi) through `elements` with quadrupole strengths
    ks[families[e]] (families[e] = -1: the element's own k is kept).

    forward(ks (m,) float64, twiss (8,) float64, xi (6, n) CUDA float64,
            tracker, elements, families, species, bunch_charge_C,
            checkpoint_interval, space_charge) -> (4,) float64 on the host.
    Gradients flow to ks and to twiss[:6]; xi is not differentiated.  The
    grid box sequence is held fixed (its derivative is taken as zero)."""

    @staticmethod
    def forward(ctx, ks, twiss, xi, tracker, elements, families, species, bunch_charge_C,
                checkpoint_interval=20, space_charge=True):
        kv = [float(v) for v in ks.detach().cpu().tolist()]
        els = [api.Element(e.kind, e.length, kv[f] if f >= 0 else e.k, e.angle, e.nslice,
                           getattr(e, "k2", 0.0)) for e, f in zip(elements, families)]
        tw = [float(v) for v in twiss.detach().cpu().tolist()]
        coords = api.twiss_beam(tw, xi)
        beam = api.Beam(coords, species, bunch_charge_C)
        tracker.grad_forward(beam, els, checkpoint_interval, space_charge=space_charge)
        out = torch.tensor(api.objectives(tracker.moments(beam).cpu().tolist()),
                           dtype=torch.float64)
        ctx.tracker, ctx.beam, ctx.families, ctx.tw = tracker, beam, list(families), tw
        ctx.nk = ks.numel()
        return out

    @staticmethod
    def backward(ctx, gout):
        w = [float(v) for v in gout.detach().cpu().tolist()]
        dk_el, S, _ = ctx.tracker.grad_backward(ctx.beam, w, want_zbar0=False)
        dks = torch.tensor(api.family_grad(dk_el, ctx.families, ctx.nk), dtype=torch.float64)
        dtw = torch.zeros(8, dtype=torch.float64)
        dtw[:6] = torch.tensor(api.twiss_grad(ctx.tw, S), dtype=torch.float64)
        return dks, dtw, None, None, None, None, None, None, None, None


def track_objectives(ks, twiss, xi, tracker, elements, families, species, bunch_charge_C,
                     checkpoint_interval=20, space_charge=True):
    return TrackObjectives.apply(ks, twiss, xi, tracker, elements, families, species,
                                 bunch_charge_C, checkpoint_interval, space_charge)
