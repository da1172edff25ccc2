"""Closed-form 1s-1s integrals used to pin the oracle (no code shared with it).

Prolate spheroidal coordinates xi = cosh mu in [1, inf), eta = cos nu in [-1, 1] with atom A at
(0,0,+a): r_A = a(xi - eta), r_B = a(xi + eta), dV = a^3 (xi^2 - eta^2) dxi deta dphi.  For
normalised 1s functions N e^{-zeta r}, N = sqrt(zeta^3/pi), every two-centre 1s-1s integral
reduces to the textbook auxiliary integrals A_k(p) = int_1^inf x^k e^{-px} dx and
B_k(q) = int_-1^1 x^k e^{-qx} dx, here evaluated with mpmath at 30 digits.
"""
import math

import mpmath as mp

mp.mp.dps = 30


def A(k, p):
    return mp.quad(lambda x: x ** k * mp.e ** (-p * x), [1, mp.inf])


def B(k, q):
    return mp.quad(lambda x: x ** k * mp.e ** (-q * x), [-1, 1])


def norm1s(z):
    return math.sqrt(z ** 3 / math.pi)


def _pq(R, za, zb):
    a = R / 2.0
    # exponent -za a (xi - eta) - zb a (xi + eta) = -p xi - q eta
    return a, a * (za + zb), a * (zb - za)


def overlap(R, za, zb):
    a, p, q = _pq(R, za, zb)
    return float(2 * mp.pi * a ** 3 * norm1s(za) * norm1s(zb) * (A(2, p) * B(0, q) - A(0, p) * B(2, q)))


def overlap_equal(R, z):
    rho = z * R
    return math.exp(-rho) * (1 + rho + rho * rho / 3)


def hybrid_over_rb(R, za, zb):
    """<a | 1/r_B | b>, a on A, b on B."""
    a, p, q = _pq(R, za, zb)
    return float(2 * mp.pi * a ** 2 * norm1s(za) * norm1s(zb) * (A(1, p) * B(0, q) - A(0, p) * B(1, q)))


def hybrid_over_ra(R, za, zb):
    """<a | 1/r_A | b>, a on A, b on B."""
    a, p, q = _pq(R, za, zb)
    return float(2 * mp.pi * a ** 2 * norm1s(za) * norm1s(zb) * (A(1, p) * B(0, q) + A(0, p) * B(1, q)))


def one_centre_over_r(z):
    """<a | 1/r_A | a> = zeta."""
    return z


def other_nucleus(R, z):
    """<a | 1/r_B | a> for a on A, nucleus B at distance R."""
    return 1.0 / R - (z + 1.0 / R) * math.exp(-2 * z * R)


def kinetic(R, za, zb):
    """<a | -1/2 lap | b> = -zb^2/2 S + zb <a|1/r_B|b>."""
    return -0.5 * zb * zb * overlap(R, za, zb) + zb * hybrid_over_rb(R, za, zb)


def potential_1s_unnormalised(alpha, r):
    """Coulomb potential of the density e^{-alpha r}: 8 pi/(alpha^3 r) [1 - (1 + alpha r/2) e^{-alpha r}]
    (evaluated at 30 digits: the bracket cancels for small alpha r)."""
    a, x = mp.mpf(alpha), mp.mpf(r)
    return float(8 * mp.pi / (a ** 3 * x) * (1 - (1 + a * x / 2) * mp.e ** (-a * x)))


def coulomb_2c(R, alpha, beta):
    """(P|Q) = int int chi_P(1) chi_Q(2) / r12 for normalised 1s aux functions, P on A, Q on B.

    (P|Q) = N_P N_Q 8pi/alpha^3 [ I1 - I2 - I3 ] with I1 = int e^{-beta r_B}/r_A (the potential
    of e^{-beta r} at distance R), I2 = int e^{-alpha r_A - beta r_B}/r_A, I3 = alpha/2 int
    e^{-alpha r_A - beta r_B}."""
    a, p, q = _pq(R, alpha, beta)
    I1 = potential_1s_unnormalised(beta, R)
    I2 = 2 * mp.pi * a ** 2 * (A(1, p) * B(0, q) + A(0, p) * B(1, q))
    I3 = alpha / 2 * 2 * mp.pi * a ** 3 * (A(2, p) * B(0, q) - A(0, p) * B(2, q))
    return float(norm1s(alpha) * norm1s(beta) * 8 * mp.pi / alpha ** 3 * (I1 - I2 - I3))


def coulomb_1c_equal(alpha):
    """(P|P) for one normalised 1s function: 20 pi^2/alpha^5 * N^2 = 20 pi / alpha^2."""
    return 20 * math.pi / alpha ** 2


def coulomb_1c(alpha, beta):
    """(P|Q) for two normalised 1s functions on one centre: N_P N_Q int V_alpha(r) e^{-beta r} 4 pi r^2 dr."""
    f = lambda r: 8 * mp.pi / (alpha ** 3 * r) * (1 - (1 + alpha * r / 2) * mp.e ** (-alpha * r)) \
        * mp.e ** (-beta * r) * 4 * mp.pi * r * r
    return float(norm1s(alpha) * norm1s(beta) * mp.quad(f, [0, mp.inf]))
