"""Three-centre 1s integrals by Gaussian transforms: an integration route that shares nothing
with the prolate-spheroidal quadrature (no grid, no spheroidal coordinates), used to pin the
oracle's three-centre V_ne and (P|ij) values.

Every factor of the integrand is written as a superposition of Gaussians exp(-u r^2):

* a 1s Slater function:  e^{-z r} = int_0^inf z/(2 sqrt(pi)) u^{-3/2} e^{-z^2/(4u)} e^{-u r^2} du
  (the Laplace-transform identity behind the "Gaussian transform" of Slater functions);
* the Coulomb operator:  1/r = int_0^inf (pi u)^{-1/2} e^{-u r^2} du;
* the screened operator: e^{-a r}/r = int_0^inf (pi u)^{-1/2} e^{-a^2/(4u)} e^{-u r^2} du.

Three Gaussians on centres A, B, C integrate in closed form (the Gaussian product theorem):
int e^{-a r_A^2 - b r_B^2 - c r_C^2} d^3r = (pi/p)^{3/2} exp(-(ab AB^2 + ac AC^2 + bc BC^2)/p),
p = a + b + c.  What is left is a triple integral over (u_a, u_b, u_c) of smooth functions;
with u = e^x (or e^{2y}) the integrands decay exponentially at both ends and the trapezoidal
rule converges geometrically in the step (checked against the two-centre closed forms of
``closed_forms``).
"""
import math

import numpy as np


def _sto_factor(zeta, h, lo=-14.0, hi=18.0):
    """Nodes u and weights per node of e^{-zeta r} (u = e^x, trapezoid step h in x)."""
    x = np.arange(lo, hi + 0.5 * h, h)
    u = np.exp(x)
    w = h * u * zeta / (2.0 * math.sqrt(math.pi)) * u ** -1.5 * np.exp(-zeta * zeta / (4.0 * u))
    return u, w


def _coulomb_factor(alpha, h, lo=-40.0, hi=14.0):
    """Nodes and weights of e^{-alpha r}/r (alpha = 0: 1/r); u = e^{2y}, step h in y (callers
    pass half the Slater factors' step: the same spacing in ln u)."""
    y = np.arange(lo, hi + 0.5 * h, h)
    u = np.exp(2.0 * y)
    w = h * 2.0 * u / np.sqrt(math.pi * u)
    if alpha > 0:
        w = w * np.exp(-alpha * alpha / (4.0 * u))
    return u, w


def _gauss3(ua, wa, ub, wb, uc, wc, A, B, C):
    """sum_ijk wa_i wb_j wc_k (pi/p)^{3/2} exp(-(ab AB^2 + ac AC^2 + bc BC^2)/p)."""
    AB2 = float(np.sum((np.asarray(A) - np.asarray(B)) ** 2))
    AC2 = float(np.sum((np.asarray(A) - np.asarray(C)) ** 2))
    BC2 = float(np.sum((np.asarray(B) - np.asarray(C)) ** 2))
    a = ua[:, None]
    b = ub[None, :]
    wab = wa[:, None] * wb[None, :]
    total = 0.0
    for c, w in zip(uc, wc):
        p = a + b + c
        e = (a * b * AB2 + a * c * AC2 + b * c * BC2) / p
        total += w * float(np.sum(wab * (math.pi / p) ** 1.5 * np.exp(-e)))
    return total


def product_integral(za, A, zb, B, C, op, alpha=0.0, h=0.125):
    """int e^{-za r_A} e^{-zb r_B} O(r_C) d^3r for O = 1/r ('coulomb'), e^{-alpha r}/r
    ('screened') or e^{-alpha r} ('exp'); unnormalised 1s functions."""
    ua, wa = _sto_factor(za, h)
    ub, wb = _sto_factor(zb, h)
    if op == "coulomb":
        uc, wc = _coulomb_factor(0.0, 0.5 * h)
    elif op == "screened":
        uc, wc = _coulomb_factor(alpha, 0.5 * h)
    elif op == "exp":
        uc, wc = _sto_factor(alpha, h)
    else:
        raise ValueError(op)
    return _gauss3(ua, wa, ub, wb, uc, wc, A, B, C)


def overlap_integral(za, A, zb, B, h=0.125):
    """int e^{-za r_A} e^{-zb r_B} d^3r (two Gaussians: the product theorem with c = 0)."""
    ua, wa = _sto_factor(za, h)
    ub, wb = _sto_factor(zb, h)
    return _gauss3(ua, wa, ub, wb, np.zeros(1), np.ones(1), A, B, A)


def norm1s(z):
    return math.sqrt(z ** 3 / math.pi)


def nuclear_attraction(za, A, zb, B, C, h=0.125):
    """<a | 1/r_C | b> for normalised 1s functions a on A, b on B."""
    return norm1s(za) * norm1s(zb) * product_integral(za, A, zb, B, C, "coulomb", h=h)


def three_index_coulomb(alpha, C, za, A, zb, B, h=0.125):
    """(P|ab) = int V_P(r) a(r) b(r) d^3r for a normalised 1s aux function P of exponent alpha on
    C, whose potential is N_P 8 pi/alpha^3 [1/r - e^{-alpha r}/r - (alpha/2) e^{-alpha r}] (the
    Coulomb potential of the density e^{-alpha r}), and normalised 1s functions a on A, b on B."""
    i_c = product_integral(za, A, zb, B, C, "coulomb", h=h)
    i_s = product_integral(za, A, zb, B, C, "screened", alpha=alpha, h=h)
    i_e = product_integral(za, A, zb, B, C, "exp", alpha=alpha, h=h)
    return (norm1s(za) * norm1s(zb) * norm1s(alpha) * 8.0 * math.pi / alpha ** 3
            * (i_c - i_s - 0.5 * alpha * i_e))
