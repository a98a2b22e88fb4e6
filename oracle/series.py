"""Zernike series and its adjoint, summed exactly over the oracle's float64 basis.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper motivates series of Zernike functions (the spectral-expansion footnote of
Sec. 3) but prints no series routine; the definitions used are the plain ones:
    F[p, s]       = sum_j Z_j(p) C[j, s]
    dL/dC[j, s]   = sum_p Z_j(p) G[p, s]                        (G = dL/dF)
    dL/dr[p]      = sum_j sum_s dZ_j/drho(p) C[j, s] G[p, s]
    dL/dtheta[p]  = sum_j sum_s dZ_j/dtheta(p) C[j, s] G[p, s]
Z and its derivatives are the oracle's correctly rounded float64 values; C and G are the
caller's float64 values.  Every sum of products is formed exactly in integers (each float64
is a dyadic rational) and rounded once.
"""
from __future__ import annotations

from . import basis as _basis


def _dy(x: float) -> tuple[int, int]:
    a, d = float(x).as_integer_ratio()
    return a, d.bit_length() - 1


def exact_sum_of_products(terms) -> float:
    """Correctly rounded float64 of sum_i prod_j x_ij for float64 factors x_ij.
    `terms` is an iterable of tuples of floats."""
    parts = []
    emax = 0
    for t in terms:
        a, e = 1, 0
        for x in t:
            ai, ei = _dy(x)
            a *= ai
            e += ei
        if a:
            parts.append((a, e))
            emax = max(emax, e)
    num = 0
    for a, e in parts:
        num += a << (emax - e)
    return num / (1 << emax)


def series_eval(ns, ms, rs, thetas, coeffs):
    """F[p][s] for coefficient sets coeffs[j][s]."""
    zk, _ = _basis.basis_table(ns, ms, rs, thetas, 0)
    z = zk[0]
    J, P, S = len(ns), len(rs), len(coeffs[0]) if len(coeffs) else 0
    return [[exact_sum_of_products((z[j][p], coeffs[j][s]) for j in range(J)) for s in range(S)]
            for p in range(P)]


def series_adjoint(ns, ms, rs, thetas, coeffs, grad_out):
    """(grad_C[j][s], grad_r[p], grad_theta[p]) for upstream grad_out[p][s]."""
    zk, zt = _basis.basis_table(ns, ms, rs, thetas, 1, with_dtheta=True)
    z, zr = zk[0], zk[1]
    J, P = len(ns), len(rs)
    S = len(coeffs[0]) if J else 0
    gC = [[exact_sum_of_products((z[j][p], grad_out[p][s]) for p in range(P)) for s in range(S)]
          for j in range(J)]
    gr = [exact_sum_of_products((zr[j][p], coeffs[j][s], grad_out[p][s])
                                for j in range(J) for s in range(S)) for p in range(P)]
    gt = [exact_sum_of_products((zt[j][p], coeffs[j][s], grad_out[p][s])
                                for j in range(J) for s in range(S)) for p in range(P)]
    return gC, gr, gt


def point_hessian(ns, ms, rs, thetas, coeffs, grad_out):
    """Per point p, for L = sum_{p,s} F[p,s] G[p,s]: (dL/dr_p, dL/dtheta_p, d2L/dr_p^2,
    d2L/dr_p dtheta_p, d2L/dtheta_p^2), each the exact sum over j, s of the corresponding
    derivative of Z_j at p (oracle basis, rounded once) times C[j, s] G[p, s], rounded once."""
    J, P = len(ns), len(rs)
    S = len(coeffs[0]) if J else 0
    out = []
    for kr, kt in ((1, 0), (0, 1), (2, 0), (1, 1), (0, 2)):
        vals = []
        for p in range(P):
            z = [_basis.basis_deriv(int(ns[j]), int(ms[j]), float(rs[p]), float(thetas[p]), kr, kt) for j in range(J)]
            vals.append(exact_sum_of_products((z[j], coeffs[j][s], grad_out[p][s]) for j in range(J) for s in range(S)))
        out.append(vals)
    return tuple(out)
