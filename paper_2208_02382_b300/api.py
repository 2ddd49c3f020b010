"""Python binding of libbeamtrack: the same calls as the C ABI, taking torch
CUDA tensors for device memory and torch's current stream.  Argument
marshalling only; every step of the tracking path runs in the library's CUDA
kernels (there is no CPU fallback)."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Sequence

import torch

from . import _lib as L


def _check(lib, ctx, rc):
    if rc != L.BX_OK:
        msg = lib.bx_last_error(ctx)
        raise L.BeamtrackError(rc, msg.decode() if msg else "")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass
class Species:
    mass_MeV: float
    kinetic_MeV: float
    charge_sign: float


@dataclass(frozen=True)
class Element:
    """One lattice element (Listing 1 elements): kind L.BX_DRIFT / BX_QUAD /
    BX_SBEND / BX_DIPEDGE / BX_CONSTF / BX_MULTIPOLE, length [m], strength k
    [1/m^2] (edge: curvature 1/rho; multipole: kn), bend or edge angle [rad],
    slices (space-charge kicks; 0 for a thin element), k2 [1/m^2] (constant
    focusing in y; multipole: ks), order (multipole order m)."""
    kind: int
    length: float
    k: float
    angle: float
    nslice: int
    k2: float = 0.0
    order: int = 0


def _ptr6(t: torch.Tensor):
    """Six device pointers of the rows of a contiguous (6, n) float64 tensor."""
    n = t.shape[1]
    base = t.data_ptr()
    return (ctypes.c_void_p * 6)(*[base + 8 * n * k for k in range(6)])


def twiss_beam(twiss, xi: torch.Tensor) -> torch.Tensor:
    """(6, n) bunch from standard-normal draws xi and the Twiss parameters
    (alpha_x, beta_x, eps_x, alpha_y, beta_y, eps_y, sigma_t, sigma_pt)."""
    lib = L.load()
    xi = xi.contiguous()
    out = torch.empty_like(xi)
    tw = (ctypes.c_double * 8)(*[float(v) for v in twiss])
    _check(lib, None, lib.bx_twiss_beam(tw, _ptr6(xi), xi.shape[1], _ptr6(out), _stream()))
    return out


def distribution_beam(kind: str, params, normals: torch.Tensor,
                      uniforms: torch.Tensor | None = None) -> torch.Tensor:
    """(6, n) bunch in the Listing-1 parametrisation: kind "gaussian" or
    "waterbag", params = (sigmaX, sigmaY, sigmaT, sigmaPx, sigmaPy, sigmaPt,
    muxpx, muypy, mutpt), normals (6, n) standard normal draws, uniforms (n,)
    draws in [0, 1) for the Waterbag."""
    lib = L.load()
    k = {"gaussian": 0, "waterbag": 1}[kind]
    normals = normals.contiguous()
    out = torch.empty_like(normals)
    pp = (ctypes.c_double * 9)(*[float(v) for v in params])
    up = ctypes.c_void_p(uniforms.contiguous().data_ptr()) if uniforms is not None else None
    _check(lib, None, lib.bx_distribution_beam(k, pp, _ptr6(normals), up, normals.shape[1],
                                                _ptr6(out), _stream()))
    return out


def twiss_grad(twiss, S) -> list:
    """dL/d(alpha_x, beta_x, eps_x, alpha_y, beta_y, eps_y) from
    S[i][j] = sum_p dL/dz0_i z0_j."""
    lib = L.load()
    tw = (ctypes.c_double * 8)(*[float(v) for v in twiss])
    ss = (ctypes.c_double * 36)(*[float(v) for v in list(S)])
    out = (ctypes.c_double * 6)()
    _check(lib, None, lib.bx_twiss_grad(tw, ss, out))
    return list(out)


def objectives(moments) -> list:
    """(eps_x, eps_y, sigma_x, sigma_y) from the 27 moments (bx_objectives)."""
    lib = L.load()
    m = (ctypes.c_double * 27)(*[float(v) for v in moments])
    out = (ctypes.c_double * 4)()
    _check(lib, None, lib.bx_objectives(m, out))
    return list(out)


def family_grad(dk_element, family, nfamilies: int) -> list:
    """Per-family sums of per-element dL/dk (bx_family_grad)."""
    lib = L.load()
    n = len(dk_element)
    if len(family) != n:
        raise ValueError("one family index per element")
    dk = (ctypes.c_double * max(1, n))(*[float(v) for v in dk_element])
    fam = (ctypes.c_int32 * max(1, n))(*[int(v) for v in family])
    out = (ctypes.c_double * max(1, int(nfamilies)))()
    _check(lib, None, lib.bx_family_grad(dk, fam, n, int(nfamilies), out))
    return [out[i] for i in range(int(nfamilies))]


class Beam:
    """A bunch on the device: `coords` is a (6, n) float64 CUDA tensor
    (x, px, y, py, t, pt), `ids` an int64 CUDA tensor of length n."""

    def __init__(self, coords: torch.Tensor, species: Species, bunch_charge_C: float,
                 ids: torch.Tensor | None = None):
        if coords.dtype != torch.float64 or coords.dim() != 2 or coords.shape[0] != 6:
            raise ValueError("coords must be a (6, n) float64 tensor")
        if not coords.is_cuda:
            raise ValueError("coords must live on a CUDA device")
        self.coords = coords.contiguous()
        n = self.coords.shape[1]
        self.ids = ids if ids is not None else torch.arange(n, dtype=torch.int64,
                                                            device=coords.device)
        self.species = species
        self.bunch_charge_C = float(bunch_charge_C)

    @property
    def n(self) -> int:
        return self.coords.shape[1]

    def c_struct(self) -> L.bx_beam:
        b = L.bx_beam()
        base = self.coords.data_ptr()
        n = self.n
        for k in range(6):
            b.coord[k] = base + 8 * n * k if n > 0 else None
        b.id = self.ids.data_ptr() if n > 0 else None
        b.n = n
        b.charge_sign = float(self.species.charge_sign)
        b.bunch_charge_C = self.bunch_charge_C
        b.mass_MeV = float(self.species.mass_MeV)
        b.kinetic_MeV = float(self.species.kinetic_MeV)
        return b


def lattice_struct(elements: Sequence, space_charge: bool):
    """elements: objects with kind, length, k, angle, nslice (beamgen.Element)."""
    arr = (L.bx_element * max(1, len(elements)))()
    for i, e in enumerate(elements):
        arr[i].type = int(e.kind)
        arr[i].nslice = int(e.nslice)
        arr[i].length = float(e.length)
        arr[i].k = float(e.k)
        arr[i].angle = float(e.angle)
        arr[i].k2 = float(getattr(e, "k2", 0.0))
        arr[i].order = int(getattr(e, "order", 0))
    lat = L.bx_lattice()
    lat.elements = ctypes.cast(arr, ctypes.POINTER(L.bx_element))
    lat.count = len(elements)
    lat.space_charge = 1 if space_charge else 0
    return lat, arr


class Grid:
    """rho (n^3) and phi ((n+2)^3) device tensors with the box."""

    def __init__(self, n: int, device, lo=None, hi=None):
        self.n = n
        self.rho = torch.zeros(n ** 3, dtype=torch.float64, device=device)
        self.phi = torch.zeros((n + 2) ** 3, dtype=torch.float64, device=device)
        self.lo = list(lo) if lo is not None else [0.0] * 3
        self.hi = list(hi) if hi is not None else [0.0] * 3
        self.h = [0.0] * 3
        self.use_box = lo is not None

    def c_struct(self) -> L.bx_grid:
        g = L.bx_grid()
        g.n = self.n
        g.use_box = 1 if self.use_box else 0
        for d in range(3):
            g.lo[d], g.hi[d], g.h[d] = self.lo[d], self.hi[d], self.h[d]
        g.rho = self.rho.data_ptr()
        g.phi = self.phi.data_ptr()
        return g

    def read_back(self, g: L.bx_grid):
        self.lo = [g.lo[d] for d in range(3)]
        self.hi = [g.hi[d] for d in range(3)]
        self.h = [g.h[d] for d in range(3)]


class Tracker:
    """A libbeamtrack context (bx_create) on the current CUDA device."""

    def __init__(self, n_grid: int, shape_order: int = 1, rebin_interval: int = 0,
                 bin_edge: int = 0, cell_order: int = 0):
        self.lib = L.load()
        opt = L.bx_options()
        opt.n_grid = int(n_grid)
        opt.shape_order = int(shape_order)
        opt.rebin_interval = int(rebin_interval)
        opt.bin_edge = int(bin_edge)
        opt.cell_order = int(cell_order)
        ctx = ctypes.c_void_p()
        rc = self.lib.bx_create(ctypes.byref(ctx), ctypes.byref(opt))
        _check(self.lib, None, rc)
        self.ctx = ctx
        self.n = int(n_grid)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.bx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        _check(self.lib, self.ctx, self.lib.bx_reset(self.ctx))

    def set_shard(self, allreduce, n_total: int = 0):
        """Make this context one rank of a particle-sharded run (bx_set_shard):
        `allreduce(t, op)` must reduce the int64 CUDA tensor t in place over all
        ranks (op one of BX_OP_SUM/MIN/MAX; e.g. torch_allreduce()); n_total:
        particles of the whole bunch.  allreduce=None ends the shard."""
        if allreduce is None:
            _check(self.lib, self.ctx, self.lib.bx_set_shard(self.ctx, None))
            self._shard = None
            return
        dev = torch.cuda.current_device()

        def cb(ptr, count, op, stream, user):
            try:
                allreduce(torch.as_tensor(_DeviceInt64(ptr, count), device=dev), int(op))
                return 0
            except Exception as exc:   # reported by track() after the call fails
                self._shard_error = exc
                return 1
        fn = L.bx_allreduce_fn(cb)
        sh = L.bx_shard(fn, None, int(n_total))
        self._shard = (fn, sh)         # the callback must outlive the calls that use it
        self._shard_error = None
        _check(self.lib, self.ctx, self.lib.bx_set_shard(self.ctx, ctypes.byref(sh)))

    def track(self, beam: Beam, elements, first_kick: int = 0, nkicks: int = -1,
              space_charge: bool = True, diagnostics: bool = False):
        """Track; with diagnostics, return the (kicks, 27) moments at every
        slice end (layout of moments())."""
        b = beam.c_struct()
        lat, keep = lattice_struct(elements, space_charge)
        if not diagnostics:
            rc = self.lib.bx_track(self.ctx, ctypes.byref(b), ctypes.byref(lat), int(first_kick),
                                   int(nkicks), _stream())
            if rc == L.BX_COLLECTIVE and getattr(self, "_shard_error", None) is not None:
                err, self._shard_error = self._shard_error, None
                raise L.BeamtrackError(rc, f"allreduce callback: {err!r}") from err
            _check(self.lib, self.ctx, rc)
            return None
        total = sum(int(e.nslice) for e in elements if int(e.kind) != L.BX_DIPEDGE)
        nk = total - int(first_kick) if nkicks < 0 else int(nkicks)
        out = torch.empty((max(nk, 0), 27), dtype=torch.float64, device=beam.coords.device)
        rc = self.lib.bx_track_diagnostics(self.ctx, ctypes.byref(b), ctypes.byref(lat),
                                           int(first_kick), int(nkicks),
                                           ctypes.c_void_p(out.data_ptr()), _stream())
        _check(self.lib, self.ctx, rc)
        return out

    def deposit(self, beam: Beam, grid: Grid) -> Grid:
        b = beam.c_struct()
        g = grid.c_struct()
        _check(self.lib, self.ctx, self.lib.bx_deposit(self.ctx, ctypes.byref(b), ctypes.byref(g),
                                                       _stream()))
        grid.read_back(g)
        return grid

    def solve(self, grid: Grid) -> Grid:
        g = grid.c_struct()
        _check(self.lib, self.ctx, self.lib.bx_solve(self.ctx, ctypes.byref(g), _stream()))
        return grid

    def gather_kick(self, beam: Beam, grid: Grid, ds: float):
        b = beam.c_struct()
        g = grid.c_struct()
        _check(self.lib, self.ctx, self.lib.bx_gather_kick(self.ctx, ctypes.byref(b),
                                                           ctypes.byref(g), float(ds), _stream()))

    def moments(self, beam: Beam) -> torch.Tensor:
        out = torch.empty(27, dtype=torch.float64, device=beam.coords.device)
        b = beam.c_struct()
        _check(self.lib, self.ctx, self.lib.bx_moments(self.ctx, ctypes.byref(b),
                                                       ctypes.c_void_p(out.data_ptr()), _stream()))
        return out

    def green_table(self, h, device) -> torch.Tensor:
        out = torch.empty((self.n + 1) ** 3, dtype=torch.float64, device=device)
        hh = (ctypes.c_double * 3)(*[float(v) for v in h])
        _check(self.lib, self.ctx, self.lib.bx_green_table(self.ctx, hh,
                                                           ctypes.c_void_p(out.data_ptr()),
                                                           _stream()))
        return out

    def regrid_log(self) -> list:
        cnt = ctypes.c_int64()
        _check(self.lib, self.ctx, self.lib.bx_regrid_log(self.ctx, None, 0, ctypes.byref(cnt)))
        buf = (ctypes.c_int64 * max(1, cnt.value))()
        _check(self.lib, self.ctx, self.lib.bx_regrid_log(self.ctx, buf, cnt.value,
                                                          ctypes.byref(cnt)))
        return [buf[i] for i in range(cnt.value)]

    def box(self):
        lo, hi, h = (ctypes.c_double * 3)(), (ctypes.c_double * 3)(), (ctypes.c_double * 3)()
        _check(self.lib, self.ctx, self.lib.bx_get_box(self.ctx, lo, hi, h))
        return list(lo), list(hi), list(h)

    def profile(self, timing: bool = True):
        _check(self.lib, self.ctx, self.lib.bx_profile(self.ctx, 1 if timing else 0))

    def profile_read(self) -> dict:
        """{kernel name: (device ms, launches)} since the last profile() call."""
        cap = 64
        ms = (ctypes.c_double * cap)()
        cnt = (ctypes.c_int64 * cap)()
        k = ctypes.c_int32()
        _check(self.lib, self.ctx, self.lib.bx_profile_read(self.ctx, ms, cnt, cap,
                                                            ctypes.byref(k)))
        return {self.lib.bx_kernel_name(i).decode(): (ms[i], cnt[i]) for i in range(k.value)}

    def sync(self):
        _check(self.lib, self.ctx, self.lib.bx_sync(self.ctx, _stream()))

    def selftest_wait_timeout(self, limit_ms: float):
        """Run the self-test of the bounded device wait; the next sync() raises
        BeamtrackError with code BX_DEVICE_TIMEOUT."""
        _check(self.lib, self.ctx, self.lib.bx_selftest_wait_timeout(self.ctx, float(limit_ms),
                                                                     _stream()))

    # ---- tuning
    def set_binning(self, rebin_interval: int, bin_edge: int, cell_order: int = 0):
        _check(self.lib, self.ctx, self.lib.bx_set_binning(self.ctx, int(rebin_interval),
                                                           int(bin_edge), int(cell_order)))

    def autotune_binning(self, beam: Beam, elements, kicks: int = 32, space_charge: bool = True):
        """Time the binning candidates on this problem and keep the fastest;
        returns ((rebin_interval, bin_edge, cell_order), [ms per candidate])."""
        b = beam.c_struct()
        lat, keep = lattice_struct(elements, space_charge)
        chosen = (ctypes.c_int32 * 3)()
        cap = 64
        ms = (ctypes.c_double * cap)()
        cnt = ctypes.c_int32()
        rc = self.lib.bx_autotune_binning(self.ctx, ctypes.byref(b), ctypes.byref(lat), int(kicks),
                                          chosen, ms, cap, ctypes.byref(cnt), _stream())
        _check(self.lib, self.ctx, rc)
        return (chosen[0], chosen[1], chosen[2]), [ms[i] for i in range(min(cap, cnt.value))]

    # ---- differentiation
    def grad_forward(self, beam: Beam, elements, checkpoint_interval: int = 20,
                     box_replay=None, space_charge: bool = True):
        """Track the whole lattice, recording what the reverse pass needs.
        box_replay: (K, 12) boxes of an earlier run (grad_boxes) or None."""
        b = beam.c_struct()
        lat, keep = lattice_struct(elements, space_charge)
        rp = None
        if box_replay is not None:
            flat = [float(v) for row in box_replay for v in row]
            rp = (ctypes.c_double * len(flat))(*flat)
        rc = self.lib.bx_grad_forward(self.ctx, ctypes.byref(b), ctypes.byref(lat),
                                      int(checkpoint_interval), rp, _stream())
        _check(self.lib, self.ctx, rc)
        self._grad_nelem = len(elements)

    def grad_backward(self, beam: Beam, weights, want_zbar0: bool = True):
        """dL/dk per element, S = sum_p dL/dz0 z0^T (36, row-major) and
        (optionally) dL/dz0 as a (6, n) tensor, for L = weights . (eps_x,
        eps_y, sigma_x, sigma_y) of the final bunch."""
        b = beam.c_struct()
        w = (ctypes.c_double * 4)(*[float(v) for v in weights])
        ne = getattr(self, "_grad_nelem", 0)
        dk = (ctypes.c_double * max(1, ne))()
        S = (ctypes.c_double * 36)()
        zb = torch.empty_like(beam.coords) if want_zbar0 else None
        rc = self.lib.bx_grad_backward(self.ctx, ctypes.byref(b), w, dk, S,
                                       _ptr6(zb) if zb is not None else None, _stream())
        _check(self.lib, self.ctx, rc)
        return [dk[i] for i in range(ne)], list(S), zb

    def grad_boxes(self) -> list:
        cnt = ctypes.c_int64()
        _check(self.lib, self.ctx, self.lib.bx_grad_boxes(self.ctx, None, 0, ctypes.byref(cnt)))
        buf = (ctypes.c_double * (12 * max(1, cnt.value)))()
        _check(self.lib, self.ctx, self.lib.bx_grad_boxes(self.ctx, buf, cnt.value,
                                                          ctypes.byref(cnt)))
        return [[buf[12 * i + j] for j in range(12)] for i in range(cnt.value)]


class _DeviceInt64:
    """Zero-copy view of `count` int64 values at a device address (the
    library's box keys and charge accumulators) for torch.as_tensor."""

    def __init__(self, ptr: int, count: int):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<i8",
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def torch_allreduce(group=None):
    """The collective of a sharded run over torch.distributed, for
    Tracker.set_shard: with NCCL in place on the device (stream-ordered); with
    other backends (gloo) through host memory (the copy to the host waits for
    the stream, the copy back is ordered on it)."""
    import torch.distributed as dist
    ops = {L.BX_OP_SUM: dist.ReduceOp.SUM, L.BX_OP_MIN: dist.ReduceOp.MIN,
           L.BX_OP_MAX: dist.ReduceOp.MAX}
    on_device = dist.get_backend(group) == "nccl"

    def reduce(t: torch.Tensor, op: int):
        if on_device:
            dist.all_reduce(t, op=ops[op], group=group)
        else:
            h = t.cpu()
            dist.all_reduce(h, op=ops[op], group=group)
            t.copy_(h)
    return reduce


def shard_range(n_total: int, rank: int, world: int):
    """[start, stop) of the particles rank `rank` holds when a bunch of
    n_total particles is split over `world` ranks in contiguous, near-equal
    shares."""
    if not (0 <= rank < world):
        raise ValueError("rank outside the world")
    base, extra = divmod(int(n_total), int(world))
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def autotune_batch(trackers: Sequence[Tracker], beams: Sequence[Beam], lattices, kicks: int = 32):
    """Binning autotuning for a batch: problems with the same grid size and
    particle count within a factor of two share one tuning (of the first of
    them).  Returns {(n_grid, bucket): (rebin_interval, bin_edge, cell_order)}."""
    import math
    groups = {}
    for t, b, lat in zip(trackers, beams, lattices):
        key = (t.n, int(math.floor(math.log2(max(1, b.n)))))
        groups.setdefault(key, []).append((t, b, lat))
    chosen = {}
    for key, members in groups.items():
        t, b, lat = members[0]
        choice, _ = t.autotune_binning(b, lat, kicks)
        chosen[key] = choice
        for t2, _, _ in members[1:]:
            t2.set_binning(*choice)
    return chosen


class Batch:
    """Independent tracking problems (tracker, beam, elements) run by one CUDA
    graph launch (bx_batch_*): each problem tracks its whole lattice exactly
    as tracker.reset() + tracker.track(beam, elements) would."""

    def __init__(self, trackers: Sequence[Tracker], beams: Sequence[Beam], lattices,
                 space_charge: bool = True):
        self.lib = L.load()
        n = len(trackers)
        if not (n == len(beams) == len(lattices)) or n == 0:
            raise ValueError("one beam and one lattice per tracker")
        self._keep = []
        ctxs = (ctypes.c_void_p * n)(*[t.ctx for t in trackers])
        bs = [b.c_struct() for b in beams]
        lats = []
        for els in lattices:
            lat, arr = lattice_struct(els, space_charge)
            lats.append(lat)
            self._keep.append(arr)
        bp = (ctypes.POINTER(L.bx_beam) * n)(*[ctypes.pointer(b) for b in bs])
        lp = (ctypes.POINTER(L.bx_lattice) * n)(*[ctypes.pointer(x) for x in lats])
        self._keep += [bs, lats, trackers, beams]
        h = ctypes.c_void_p()
        rc = self.lib.bx_batch_create(ctypes.byref(h), n, ctxs, bp, lp, _stream())
        if rc != L.BX_OK:
            msg = self.lib.bx_batch_last_error(None)
            raise L.BeamtrackError(rc, msg.decode() if msg else "")
        self.handle = h

    def launch(self):
        rc = self.lib.bx_batch_launch(self.handle, _stream())
        if rc != L.BX_OK:
            msg = self.lib.bx_batch_last_error(self.handle)
            raise L.BeamtrackError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "handle", None):
            self.lib.bx_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
