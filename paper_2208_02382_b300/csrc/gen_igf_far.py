"""Writes igf_far.cuh: the far-field series of the cell-integrated Green's
function used by igf.cu.

For a cell of half-sides a = h/2 centred at R (|R| well above |a|), Taylor
expansion of 1/|R + s| and integration over the cell (odd orders vanish):

    int_cell d^3s / |R + s| = V sum_{p,q,t} a_x^2p a_y^2q a_z^2t
                              / ((2p+1)! (2q+1)! (2t+1)!) * d_x^2p d_y^2q d_z^2t (1/R)

and d^alpha (1/R) = P_alpha(x, y, z) / R^(2|alpha|+1) with P_alpha homogeneous
of degree |alpha|, from P_0 = 1 and
    P_{alpha + e_x} = (x^2 + y^2 + z^2) dP_alpha/dx - (2|alpha| + 1) x P_alpha.
With u = x/R etc. the order-2n term is P(u, v, w)/R^(2n+1); for even alpha
P holds only even powers, so it is a polynomial in U = u^2, V = v^2, W = w^2.
The table holds, for n = 1..L and each (p, q, t) with p+q+t = n, the
coefficients of that polynomial over the monomials U^i V^j W^k (i+j+k = n),
divided by (2p+1)!(2q+1)!(2t+1)!.  Both orderings run p (resp. i) from n down
to 0, then q (resp. j) from n-p down to 0.

The order-l Taylor term of 1/|R+s| is |s|^l P_l(cos)/R^(l+1) with |P_l| <= 1,
so after the order-2L term the relative truncation error is below
rho^(2L+2)/(1 - rho^2), rho = |a|/|R|; igf.cu uses the series where
rho <= 1/8, L = 8 (below 5.6e-17), fewer orders farther out.

Run:  python gen_igf_far.py   (rewrites igf_far.cuh next to this file)
"""
from __future__ import annotations

import os
from fractions import Fraction
from math import factorial

L = 8


def poly_mul_r2_dx(P, var):
    """(x^2+y^2+z^2) dP/dvar for P a dict {(i,j,k): int} over x^i y^j z^k."""
    out = {}
    for (i, j, k), c in P.items():
        e = (i, j, k)[var]
        if e == 0:
            continue
        d = list((i, j, k))
        d[var] -= 1
        for sq in range(3):
            m = list(d)
            m[sq] += 2
            key = tuple(m)
            out[key] = out.get(key, 0) + c * e
    return out


def deriv_polys(maxorder):
    """P_alpha for all alpha with |alpha| <= maxorder, by the recursion."""
    polys = {(0, 0, 0): {(0, 0, 0): 1}}
    for order in range(maxorder):
        for alpha, P in list(polys.items()):
            if sum(alpha) != order:
                continue
            for var in range(3):
                beta = list(alpha)
                beta[var] += 1
                beta = tuple(beta)
                if beta in polys:
                    continue
                Q = poly_mul_r2_dx(P, var)
                for (i, j, k), c in P.items():
                    m = [i, j, k]
                    m[var] += 1
                    key = tuple(m)
                    Q[key] = Q.get(key, 0) - (2 * order + 1) * c
                polys[beta] = {kk: v for kk, v in Q.items() if v != 0}
    return polys


def triples(n):
    return [(p, q, n - p - q) for p in range(n, -1, -1) for q in range(n - p, -1, -1)]


def table():
    polys = deriv_polys(2 * L)
    rows = []
    for n in range(1, L + 1):
        for (p, q, t) in triples(n):
            P = polys[(2 * p, 2 * q, 2 * t)]
            den = factorial(2 * p + 1) * factorial(2 * q + 1) * factorial(2 * t + 1)
            coef = []
            for (i, j, k) in triples(n):
                c = P.get((2 * i, 2 * j, 2 * k), 0)
                coef.append(Fraction(c, den))
            # every monomial of P has even exponents
            assert all(e % 2 == 0 for key in P for e in key)
            rows.append(((n, p, q, t), coef))
    return rows


def main():
    rows = table()
    lines = [
        "// Generated by gen_igf_far.py: far-field series of the cell-integrated",
        "// Green's function (see that script for the derivation and ordering).",
        "#pragma once",
        "",
        "namespace bt {",
        "",
        f"constexpr int IGF_FAR_L = {L};",
        "// offsets of order n's block (n = 1..L) in IGF_FAR_P",
    ]
    offs, o = [], 0
    for n in range(1, L + 1):
        offs.append(o)
        nt = (n + 1) * (n + 2) // 2
        o += nt * nt
    lines.append("__constant__ int IGF_FAR_OFF[IGF_FAR_L + 1] = {" + ", ".join(str(v) for v in offs + [o]) + "};")
    vals = []
    for (_, coef) in rows:
        vals += [repr(float(c)) for c in coef]
    # global memory, read through the read-only path: the coefficient kernel's
    # threads read different entries (constant memory would serialize them)
    lines.append(f"__device__ const double IGF_FAR_P[{len(vals)}] = {{")
    for i in range(0, len(vals), 4):
        lines.append("    " + ", ".join(vals[i:i + 4]) + ",")
    lines.append("};")
    lines += ["", "}  // namespace bt", ""]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "igf_far.cuh")
    with open(out, "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
