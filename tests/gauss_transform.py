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


# ------------------------------------------------------------------ any n, l

def solid_harmonic(l, m, rng_seed=11):
    """Coefficients {(i, j, k): c} of the homogeneous polynomial r^l Y_lm(x, y, z) = sum c x^i
    y^j z^k for the real orthonormal harmonics without the Condon-Shortley phase (m > 0: cos,
    m < 0: sin), fitted by least squares to scipy's complex harmonics at random points (exact
    up to rounding: the monomials of degree l span the solid harmonics)."""
    import scipy.special as sp
    mons = [(i, j, l - i - j) for i in range(l + 1) for j in range(l + 1 - i)]
    rng = np.random.default_rng(rng_seed)
    d = rng.normal(size=(4 * len(mons) + 20, 3))
    r = np.linalg.norm(d, axis=1)
    theta, phi = np.arccos(d[:, 2] / r), np.arctan2(d[:, 1], d[:, 0])
    am = abs(m)
    c = sp.sph_harm_y(l, am, theta, phi) if hasattr(sp, "sph_harm_y") else sp.sph_harm(am, l, phi, theta)
    y = c.real if m == 0 else math.sqrt(2.0) * (-1) ** am * (c.real if m > 0 else c.imag)
    X = np.stack([d[:, 0] ** i * d[:, 1] ** j * d[:, 2] ** k for (i, j, k) in mons], axis=1)
    coef = np.linalg.lstsq(X, y * r ** l, rcond=None)[0]
    return {mo: float(v) for mo, v in zip(mons, coef) if abs(v) > 1e-12}


def _radial_weights(zeta, k, h, lo=-14.0, hi=18.0):
    """Weights of r^k e^{-zeta r} = (-d/dzeta)^k e^{-zeta r} on the nodes u = e^x: (-1)^k times
    the k-th zeta-derivative of zeta/(2 sqrt(pi)) u^{-3/2} e^{-zeta^2/(4u)}, with
    d^k/dzeta^k e^{-zeta^2/(4u)} = (-1)^k (4u)^{-k/2} H_k(zeta/(2 sqrt u)) e^{-zeta^2/(4u)}
    (physicists' Hermite polynomials) and d^k (zeta E) = zeta E^(k) + k E^(k-1)."""
    from numpy.polynomial import hermite
    x = np.arange(lo, hi + 0.5 * h, h)
    u = np.exp(x)
    y = zeta / (2.0 * np.sqrt(u))
    E = np.exp(-y * y)

    def dE(q):
        if q < 0:
            return np.zeros_like(u)
        return (-1) ** q * (4.0 * u) ** (-q / 2.0) * hermite.hermval(y, [0] * q + [1]) * E

    dk = zeta * dE(k) + k * dE(k - 1)
    return u, h * u * (-1) ** k / (2.0 * math.sqrt(math.pi)) * u ** -1.5 * dk


def sto_nlm(n, l, m, zeta):
    """Normalised STO of eq 1 (N = (2 zeta)^(n+1/2)/sqrt((2n)!)) as (zeta, radial power
    n - 1 - l, {monomial: coefficient}) of N r^(n-1-l) e^{-zeta r} (r^l Y_lm)."""
    N = (2.0 * zeta) ** (n + 0.5) / math.sqrt(math.factorial(2 * n))
    return (zeta, n - 1 - l, {mo: N * c for mo, c in solid_harmonic(l, m).items()})


def _moments(p, PA, PB, la, lb):
    """m[i][j] = int (t - A)^i (t - B)^j e^{-p (t - P)^2} dt / sqrt(pi/p) along one axis, with
    PA = P - A, PB = P - B, by the recurrences m[i+1][j] = PA m[i][j] + (i m[i-1][j] +
    j m[i][j-1]) / (2p) and m[i][j+1] = PB m[i][j] + (i m[i-1][j] + j m[i][j-1]) / (2p)
    (differentiate the Gaussian about P), m[0][0] = 1."""
    h2 = 0.5 / p
    m = [[None] * (lb + 1) for _ in range(la + 1)]
    m[0][0] = np.ones_like(p)
    for i in range(la + 1):
        for j in range(lb + 1):
            if i == 0 and j == 0:
                continue
            if i > 0:
                v = PA * m[i - 1][j]
                if i > 1:
                    v = v + (i - 1) * h2 * m[i - 2][j]
                if j > 0:
                    v = v + j * h2 * m[i - 1][j - 1]
            else:
                v = PB * m[i][j - 1]
                if j > 1:
                    v = v + (j - 1) * h2 * m[i][j - 2]
            m[i][j] = v
    return m


def nlm_matrix(fas, A, fbs, B, C, op, alpha=0.0, h=0.125, chunk=48):
    """M[i][j] = int a_i(r) b_j(r) O(r_C) d^3r for STOs from sto_nlm() (any n, l) on A and B and
    O as in sto_matrix(): the polynomial factors integrate as products of one-dimensional
    moments of the product Gaussian about its centre P = (aA + bB + cC)/p.  The operator's
    nodes are processed `chunk` at a time."""
    A, B, C = (np.asarray(v, dtype=float) for v in (A, B, C))
    WA = np.stack([_radial_weights(f[0], f[1], h)[1] for f in fas])
    WB = np.stack([_radial_weights(f[0], f[1], h)[1] for f in fbs])
    u = _radial_weights(1.0, 0, h)[0]
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
    mons_a = sorted({mo for f in fas for mo in f[2]})
    mons_b = sorted({mo for f in fbs for mo in f[2]})
    CA = np.array([[f[2].get(mo, 0.0) for mo in mons_a] for f in fas])
    CB = np.array([[f[2].get(mo, 0.0) for mo in mons_b] for f in fbs])
    la = max(sum(mo) for mo in mons_a)
    lb = max(sum(mo) for mo in mons_b)
    AB2, AC2, BC2 = float(np.sum((A - B) ** 2)), float(np.sum((A - C) ** 2)), float(np.sum((B - C) ** 2))
    a, b = u[None, :, None], u[None, None, :]
    out = np.zeros((len(fas), len(fbs)))
    for c0 in range(0, len(uc), chunk):
        c = uc[c0:c0 + chunk, None, None]
        w = wc[c0:c0 + chunk, None, None]
        p = a + b + c
        g = w * (math.pi / p) ** 1.5 * np.exp(-(a * b * AB2 + a * c * AC2 + b * c * BC2) / p)
        mom = [_moments(p, (b * (B[k] - A[k]) + c * (C[k] - A[k])) / p,
                        (a * (A[k] - B[k]) + c * (C[k] - B[k])) / p, la, lb) for k in range(3)]
        for ia, (i1, j1, k1) in enumerate(mons_a):
            for ib, (i2, j2, k2) in enumerate(mons_b):
                T = np.sum(g * mom[0][i1][i2] * mom[1][j1][j2] * mom[2][k1][k2], axis=0)
                out += np.outer(CA[:, ia], CB[:, ib]) * (WA @ T @ WB.T)
    return out


def nlm_three_index_matrix(alpha, C, fas, A, fbs, B, h=0.125):
    """(P|a_i b_j) for a normalised 1s aux function P of exponent alpha on C and STOs from
    sto_nlm() on A and B."""
    i_c = nlm_matrix(fas, A, fbs, B, C, "coulomb", h=h)
    i_s = nlm_matrix(fas, A, fbs, B, C, "screened", alpha=alpha, h=h)
    i_e = nlm_matrix(fas, A, fbs, B, C, "exp", alpha=alpha, h=h)
    return norm1s(alpha) * 8.0 * math.pi / alpha ** 3 * (i_c - i_s - 0.5 * alpha * i_e)
