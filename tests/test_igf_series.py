"""CPU checks of the far-field series of the cell-integrated Green's function
(paper_2208_02382_b300/csrc/gen_igf_far.py, used by the CUDA IGF for cells
whose corner radius is at most 1/8 of their distance): its derivative
polynomials against sympy, and the truncated series against the cell integral
in closed form (the 8-corner sum of the antiderivative of 1/r, Qiang et al.
2006) at 60 digits."""
import importlib.util
import os

import mpmath as mp
import pytest
import sympy as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _gen():
    path = os.path.join(ROOT, "paper_2208_02382_b300", "csrc", "gen_igf_far.py")
    spec = importlib.util.spec_from_file_location("gen_igf_far", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("alpha", [(2, 0, 0), (0, 2, 2), (4, 2, 0), (2, 2, 2), (6, 0, 4)])
def test_derivative_polynomials_match_sympy(alpha):
    g = _gen()
    polys = g.deriv_polys(sum(alpha))
    x, y, z = sp.symbols("x y z", positive=True)
    R = sp.sqrt(x ** 2 + y ** 2 + z ** 2)
    d = sp.diff(1 / R, x, alpha[0], y, alpha[1], z, alpha[2])
    want = sp.expand(sp.simplify(d * R ** (2 * sum(alpha) + 1)))
    got = sum(c * x ** i * y ** j * z ** k for (i, j, k), c in polys[alpha].items())
    assert sp.expand(got - want) == 0


def _series(g, rows, R, a):
    x, y, z = R
    R2 = x * x + y * y + z * z
    Rn = mp.sqrt(R2)
    U, V, W = x * x / R2, y * y / R2, z * z / R2
    tot = 1 / Rn
    idx = 0
    for n in range(1, g.L + 1):
        tr = g.triples(n)
        qn = 0
        for (p, q, t) in tr:
            coef = rows[idx][1]
            idx += 1
            A = a[0] ** (2 * p) * a[1] ** (2 * q) * a[2] ** (2 * t)
            qn += A * sum(mp.mpf(c.numerator) / c.denominator * U ** i * V ** j * W ** k
                          for c, (i, j, k) in zip(coef, tr))
        tot += qn / Rn ** (2 * n + 1)
    return 8 * a[0] * a[1] * a[2] * tot


@pytest.mark.parametrize("R,a", [((3.0, 2.0, 1.0), (0.11, 0.07, 0.05)),
                                 ((8.0, 0.5, 0.3), (0.25, 0.25, 0.25)),
                                 ((0.2, 0.1, 9.0), (0.02, 0.03, 0.5)),
                                 ((4.1, 1.0, 0.5), (0.3, 0.3, 0.3)),
                                 ((0.3, 0.2, 4.2), (0.1, 0.1, 0.5))])
def test_series_matches_quadrature_at_the_far_threshold(R, a):
    g = _gen()
    mp.mp.dps = 40
    R = tuple(mp.mpf(v) for v in R)
    a = tuple(mp.mpf(v) for v in a)
    rho = mp.sqrt(sum(v * v for v in a)) / mp.sqrt(sum(v * v for v in R))
    assert rho <= mp.mpf(1) / 8
    mp.mp.dps = 60

    def F(x, y, z):
        r = mp.sqrt(x * x + y * y + z * z)
        return (-z * z / 2 * mp.atan(x * y / (z * r)) - y * y / 2 * mp.atan(x * z / (y * r))
                - x * x / 2 * mp.atan(y * z / (x * r)) + y * z * mp.log(x + r)
                + x * z * mp.log(y + r) + x * y * mp.log(z + r))

    exact = mp.mpf(0)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                sign = -1 if (dx + dy + dz) % 2 == 0 else 1
                exact += sign * F(R[0] + (2 * dx - 1) * a[0], R[1] + (2 * dy - 1) * a[1],
                                  R[2] + (2 * dz - 1) * a[2])
    got = _series(g, g.table(), R, a)
    # the Legendre bound rho^(2L+2)/(1 - rho^2), L = 8
    assert abs((got - exact) / exact) < rho ** 18 / (1 - rho ** 2) + 1e-30
