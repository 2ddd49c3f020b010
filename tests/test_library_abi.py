"""CPU-side checks of the C ABI: the library loads, exports every function
declared in include/beamtrack.h, its struct layouts match the header, and
argument errors are caught on the host before any CUDA call."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2208_02382_b300 import _lib as L
from paper_2208_02382_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "beamtrack.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return L.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\S.*?\b(bx_[a-z_]+)\s*\(", text, flags=re.M)))


def test_header_declares_the_bound_functions():
    assert declared_functions() == sorted(L.SIGNATURES)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (bx_[a-z_]+)\b", out))
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "beamtrack.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(bx_options), sizeof(bx_beam), sizeof(bx_element),
         sizeof(bx_lattice), sizeof(bx_grid));
  printf("%zu %zu %zu %zu\\n", offsetof(bx_beam, n), offsetof(bx_beam, kinetic_MeV),
         offsetof(bx_grid, h), offsetof(bx_grid, phi));
  printf("%d %d %d %d %d %d %d %d %d\\n", BX_OK, BX_BAD_ARG, BX_NONFINITE, BX_OUT_OF_MEMORY,
         BX_DEVICE_TIMEOUT, BX_CUDA, BX_DRIFT, BX_QUAD, BX_SBEND);
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(v) for v in lines[0].split()]
    assert sizes == [ctypes.sizeof(L.bx_options), ctypes.sizeof(L.bx_beam),
                     ctypes.sizeof(L.bx_element), ctypes.sizeof(L.bx_lattice),
                     ctypes.sizeof(L.bx_grid)]
    offs = [int(v) for v in lines[1].split()]
    assert offs == [L.bx_beam.n.offset, L.bx_beam.kinetic_MeV.offset, L.bx_grid.h.offset,
                    L.bx_grid.phi.offset]
    codes = [int(v) for v in lines[2].split()]
    assert codes == [L.BX_OK, L.BX_BAD_ARG, L.BX_NONFINITE, L.BX_OUT_OF_MEMORY,
                     L.BX_DEVICE_TIMEOUT, L.BX_CUDA, L.BX_DRIFT, L.BX_QUAD, L.BX_SBEND]


@pytest.mark.parametrize("n_grid,order", [(7, 1), (12, 1), (4, 1), (512, 1), (32, 3), (32, 0)])
def test_create_rejects_bad_options_on_host(lib, n_grid, order):
    opt = L.bx_options()
    opt.n_grid, opt.shape_order = n_grid, order
    ctx = ctypes.c_void_p()
    rc = lib.bx_create(ctypes.byref(ctx), ctypes.byref(opt))
    assert rc == L.BX_BAD_ARG
    assert not ctx.value
    assert lib.bx_last_error(None)


def test_null_context_calls_are_rejected(lib):
    assert lib.bx_track(None, None, None, 0, 0, None) == L.BX_BAD_ARG
    assert lib.bx_solve(None, None, None) == L.BX_BAD_ARG
    assert lib.bx_sync(None, None) == L.BX_BAD_ARG
    assert lib.bx_destroy(None) == L.BX_OK


@pytest.mark.parametrize("n_grid,interval,edge", [(32, -2, 0), (32, 0, 3), (32, 0, 32),
                                                  (256, 0, 4), (64, 8, 1)])
def test_create_rejects_bad_binning_on_host(lib, n_grid, interval, edge):
    opt = L.bx_options()
    opt.n_grid, opt.shape_order = n_grid, 1
    opt.rebin_interval, opt.bin_edge = interval, edge
    ctx = ctypes.c_void_p()
    assert lib.bx_create(ctypes.byref(ctx), ctypes.byref(opt)) == L.BX_BAD_ARG
    assert b"bin" in lib.bx_last_error(None)


# last: reloads the binding module (new ctypes classes)
def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib
    monkeypatch.setattr(L, "_LIB", None)
    with pytest.raises(ImportError):
        L.load(str(tmp_path / "missing.so"))
    importlib.reload(L)


def test_objectives_match_the_oracle_definition(lib):
    """bx_objectives (host): eps = sqrt(<du^2><dpu^2> - <du dpu>^2), sigma =
    sqrt(<du^2>) from the 27 moments, against the oracle's own moments and
    emittances of a correlated bunch."""
    import numpy as np

    import beamgen as bg
    import paper_2208_02382_b300 as bt
    from oracle import track as tr
    c = bg.gaussian6d(5_000, seed=4)
    c[1] += 0.3 * c[0] / 1e-3 * 1e-4          # x-px correlation
    m = tr.moments(c)
    got = bt.objectives(tr.moments_vector(c))
    want = [m["eps_x"], m["eps_y"], float(m["sigma"][0]), float(m["sigma"][2])]
    assert np.allclose(got, want, rtol=1e-14, atol=0.0)


def test_family_grad_sums_elements_and_rejects_bad_indices(lib):
    import paper_2208_02382_b300 as bt
    assert bt.family_grad([1.0, 2.0, 3.0, 4.0, 5.0], [0, -1, 1, 0, 1], 2) == [5.0, 8.0]
    assert bt.family_grad([], [], 3) == [0.0, 0.0, 0.0]
    with pytest.raises(L.BeamtrackError):
        bt.family_grad([1.0], [2], 2)
