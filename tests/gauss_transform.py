"""Three-centre 1s integrals by Gaussian transforms: an integration route that shares nothing
with the prolate-spheroidal quadrature (no grid, no spheroidal coordinates), used to pin the
oracle's three-centre V_ne and (P|ij) values.

Every factor of the integrand is written as a superposition of Gaussians exp(-u r^2):

* a 1s Slater function:  e^{-z r} = int_0^inf z/(2 sqrt(pi)) u^{-3/2} e^{-z^2/(4u)} e^{-u r^2} du
  (the Laplace-transform identity behind the "Gaussian transform" of Slater functions), and
  r e^{-z r} = -d/dz e^{-z r} (2s) by the z-derivative of that weight; 2p functions carry
  a Cartesian factor (x_k - A_k), which becomes a moment of the product Gaussian;
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


def _sto2s_factor(zeta, h, lo=-14.0, hi=18.0):
    """Nodes and weights of r e^{-zeta r} = -d/dzeta e^{-zeta r}: the zeta-derivative of the 1s
    weight, 1/(2 sqrt(pi)) u^{-3/2} e^{-zeta^2/(4u)} (zeta^2/(2u) - 1)."""
    x = np.arange(lo, hi + 0.5 * h, h)
    u = np.exp(x)
    w = h * u / (2.0 * math.sqrt(math.pi)) * u ** -1.5 * np.exp(-zeta * zeta / (4.0 * u)) * (
        zeta * zeta / (2.0 * u) - 1.0)
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


# Normalised STOs of eq 1 for n <= 2, l <= 1 (radial N = (2 zeta)^(n+1/2)/sqrt((2n)!), real
# orthonormal harmonics without the Condon-Shortley phase: Y_1,-1 ~ y, Y_1,0 ~ z, Y_1,1 ~ x)
# as (zeta, radial 'e' (e^{-zeta r}) or 're' (r e^{-zeta r}), Cartesian index or None,
# constant).
def sto(n, l, m, zeta):
    N = (2.0 * zeta) ** (n + 0.5) / math.sqrt(math.factorial(2 * n))
    if (n, l) == (1, 0):
        return (zeta, "e", None, N / math.sqrt(4 * math.pi))
    if (n, l) == (2, 0):
        return (zeta, "re", None, N / math.sqrt(4 * math.pi))
    if (n, l) == (2, 1):
        return (zeta, "e", {-1: 1, 0: 2, 1: 0}[m], N * math.sqrt(3.0 / (4 * math.pi)))
    raise ValueError((n, l))


def _weights(fs, h):
    """Per function the transform weights on the common nodes u = e^x, times its constant."""
    return np.stack([(_sto_factor(f[0], h) if f[1] == "e" else _sto2s_factor(f[0], h))[1] * f[3] for f in fs])


def sto_matrix(fas, A, fbs, B, C, op, alpha=0.0, h=0.125):
    """M[i][j] = int a_i(r) b_j(r) O(r_C) d^3r for normalised STOs a_i on A and b_j on B (from
    sto()) and O = 1/r ('coulomb'), e^{-alpha r}/r ('screened'), e^{-alpha r} ('exp') or 1
    ('one').  The Cartesian factors (x_k - A_k), (x_k - B_k) of p functions enter through the
    moments of the product Gaussian, centred at P = (aA + bB + cC)/p: (P - A)_k, (P - B)_k and
    (P - A)_k (P - B)_k' + delta_kk'/(2p)."""
    A, B, C = (np.asarray(v, dtype=float) for v in (A, B, C))
    u, _ = _sto_factor(1.0, h)
    WA, WB = _weights(fas, h), _weights(fbs, h)
    if op == "coulomb":
        uc, wc = _coulomb_factor(0.0, 0.5 * h)
    elif op == "screened":
        uc, wc = _coulomb_factor(alpha, 0.5 * h)
    elif op == "exp":
        uc, wc = _sto_factor(alpha, h)
    elif op == "one":
        uc, wc = np.zeros(1), np.ones(1)
    else:
        raise ValueError(op)
    AB2, AC2, BC2 = float(np.sum((A - B) ** 2)), float(np.sum((A - C) ** 2)), float(np.sum((B - C) ** 2))
    a, b = u[:, None], u[None, :]
    ka = [f[2] for f in fas]
    kb = [f[2] for f in fbs]
    out = np.zeros((len(fas), len(fbs)))
    for c, w in zip(uc, wc):
        p = a + b + c
        g = w * (math.pi / p) ** 1.5 * np.exp(-(a * b * AB2 + a * c * AC2 + b * c * BC2) / p)
        PA = [(b * (B[k] - A[k]) + c * (C[k] - A[k])) / p for k in range(3)]
        PB = [(a * (A[k] - B[k]) + c * (C[k] - B[k])) / p for k in range(3)]
        for i, ki in enumerate(ka):
            for j, kj in enumerate(kb):
                if ki is None and kj is None:
                    f = g
                elif kj is None:
                    f = g * PA[ki]
                elif ki is None:
                    f = g * PB[kj]
                else:
                    f = g * (PA[ki] * PB[kj] + (0.5 / p if ki == kj else 0.0))
                out[i, j] += WA[i] @ f @ WB[j]
    return out


def sto_three_index_matrix(alpha, C, fas, A, fbs, B, h=0.125):
    """(P|a_i b_j) for a normalised 1s aux function P of exponent alpha on C (potential as in
    three_index_coulomb) and normalised STOs a_i on A, b_j on B from sto()."""
    i_c = sto_matrix(fas, A, fbs, B, C, "coulomb", h=h)
    i_s = sto_matrix(fas, A, fbs, B, C, "screened", alpha=alpha, h=h)
    i_e = sto_matrix(fas, A, fbs, B, C, "exp", alpha=alpha, h=h)
    return norm1s(alpha) * 8.0 * math.pi / alpha ** 3 * (i_c - i_s - 0.5 * alpha * i_e)


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
