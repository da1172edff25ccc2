"""Plain FP64 CPU oracle: prolate-spheroidal (PS) quadrature of Slater-orbital integrals.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module.  The library in
``paper_2510_15204_gb300`` never calls it and shares no code with it.

Everything is numpy float64, written step by step from the paper (Stark et al., "Numerical
Integration of Slater Basis Functions Over Prolate Spheroidal Grids", arXiv 2510.15204):

* Section 2.1, eqs 2-7: PS coordinates, focal distances, the tanh^-1 radial map.
* Section 2.1, eqs 9-11: Gauss-Legendre product quadrature per volume element and weights.
* Section 2.2 / 2.3 (Fig. 2, Algorithms 1-2): cell discretisation, moving the nearest mu
  and nu lines onto a third centre, splitting the cells around it N_SP ways per dimension.
* Section 3, eq 17: C1 = 2.3 a^(1/4).
* eq 1: STOs; eqs 15-16: the RI Coulomb integrals through the auxiliary potential V^P.

Where the paper is silent the oracle takes these readings (the CUDA path takes the same):
focus A (lower atom index) at (0,0,+a), so r_A = a(cosh mu - cos nu); G in eq 10 is the
[-1,1] Gauss-Legendre weight times half the cell width; real orthonormal harmonics without
the Condon-Shortley phase, m = -l..l; radial normalisation N = (2 xi)^(n+1/2)/sqrt((2n)!);
kinetic integrals in the Laplacian form, symmetrised; V^P written out through incomplete
gamma functions (Laplace expansion of 1/r12); each molecule-matrix element is integrated on
exactly one grid chosen by the centres of its integrand (one centre: the grid of that atom
with its nearest neighbour; two: their pair grid; three: the pair grid of the two basis
atoms refined around the third), except one-centre overlap and kinetic elements, which take
their closed forms (Table 1's kinetic RMSE for SO2 is reproduced by that reading).

Parity is pinned, not assumed: ``tests/test_oracle_*.py`` check this module against
closed-form 1s-1s integrals, textbook Gauss-Legendre rules, scipy's Legendre functions and
incomplete gamma, Poisson's equation for V^P, partition invariants of the grid, symmetry,
permutation equivariance, and the SO2 overlap eigenvalue printed in Section 4.  The
3-centre V_ne and (P|ij) values have no closed form; for basis functions up to 4f and a 1s
aux function they are pinned by convergence, as the refined grid grows, to an independent
evaluation by Gaussian transforms (``tests/gauss_transform.py``), besides the grid-choice
and convergence invariants.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

S, T, V, J2, J3 = 1, 2, 4, 8, 16
ALL = S | T | V | J2 | J3

ON_AXIS_TOL = 1e-10  # a third centre closer than this * a to the focal axis is "on axis"


# ----------------------------------------------------------------------------------------
# Gauss-Legendre rule (Section 2.1: Gauss-Legendre quadrature in every dimension)
# ----------------------------------------------------------------------------------------

def gauss_legendre(q: int):
    """Nodes (ascending, in (-1,1)) and weights (sum 2) of the q-point Gauss-Legendre rule.

    Newton's method on P_q, with P_q and P_q' from the Bonnet recurrence
    (k P_k = (2k-1) x P_{k-1} - (k-1) P_{k-2}) and P_q' = q (x P_q - P_{q-1}) / (x^2 - 1);
    weights 2 / ((1 - x^2) P_q'(x)^2).
    """
    if q < 1:
        raise ValueError("q >= 1")
    x = np.cos(np.pi * (np.arange(1, q + 1) - 0.25) / (q + 0.5))

    def legendre(xv):
        p_prev, p = np.ones_like(xv), xv.copy()
        for k in range(2, q + 1):
            p_prev, p = p, ((2 * k - 1) * xv * p - (k - 1) * p_prev) / k
        if q == 1:
            p_prev = np.ones_like(xv)
        dp = q * (xv * p - p_prev) / (xv * xv - 1.0)
        return p, dp

    for _ in range(100):
        p, dp = legendre(x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p, dp = legendre(x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return x[order], w[order]


# ----------------------------------------------------------------------------------------
# Pair frame (Section 2.1: foci at (0,0,+-a); the grid is rotated and translated onto a pair)
# ----------------------------------------------------------------------------------------

def pair_frame(RA, RB, RC=None):
    """Half-distance a, midpoint M and rotation Rm (columns = pair-frame x', y', z' axes in
    molecule coordinates) for the pair (A, B) with A on +z'.

    For a grid refined around a third centre C the x' axis points to C's perpendicular
    offset, so C sits at phi = 0 (Section 2.3).  Otherwise x' is the global x axis made
    perpendicular to z' (the global y axis if z' is within 60 degrees of x).
    """
    RA, RB = np.asarray(RA, float), np.asarray(RB, float)
    d = RA - RB
    R = float(np.linalg.norm(d))
    a = 0.5 * R
    M = 0.5 * (RA + RB)
    ez = d / R
    ex = None
    if RC is not None:
        v = np.asarray(RC, float) - M
        perp = v - np.dot(v, ez) * ez
        if np.linalg.norm(perp) > ON_AXIS_TOL * a:
            ex = perp / np.linalg.norm(perp)
    if ex is None:
        e = np.array([1.0, 0.0, 0.0])
        ex = e - np.dot(e, ez) * ez
        if np.linalg.norm(ex) < 0.5:
            e = np.array([0.0, 1.0, 0.0])
            ex = e - np.dot(e, ez) * ez
        ex = ex / np.linalg.norm(ex)
    ey = np.cross(ez, ex)
    return a, M, np.stack([ex, ey, ez], axis=1)


# ----------------------------------------------------------------------------------------
# Cell edges (eqs 7, 12, 17; Algorithm 1)
# ----------------------------------------------------------------------------------------

def cell_edges(spec, a):
    """mu edges C1 atanh(i/(N_mu+1)), i=0..N_mu (eq 7, 12) with C1 = 2.3 a^(1/4) (eq 17);
    nu edges j pi / N_nu; phi edges 2 pi k / N_phi (Section 2.3)."""
    n_mu, n_nu, n_phi = spec[0], spec[1], spec[2]
    C1 = 2.3 * a ** 0.25
    t = np.arange(n_mu + 1) / (n_mu + 1.0)
    mu = C1 * np.arctanh(t)
    nu = np.pi * np.arange(n_nu + 1) / n_nu
    phi = 2.0 * np.pi * np.arange(n_phi + 1) / n_phi
    return mu, nu, phi


def third_centre_coords(a, C_pair):
    """(mu_C, nu_C) of a point in the pair frame, from r_A, r_B (eqs 5-6 inverted):
    cosh mu = (r_A + r_B)/(2a), cos nu = (r_B - r_A)/(2a)."""
    rho = math.hypot(C_pair[0], C_pair[1])
    zc = C_pair[2]
    rA = math.hypot(rho, zc - a)
    rB = math.hypot(rho, zc + a)
    mu_c = math.acosh(max(1.0, (rA + rB) / (2 * a)))
    nu_c = math.acos(min(1.0, max(-1.0, (rB - rA) / (2 * a))))
    return mu_c, nu_c, rho


def place_third_centre(mu, nu, n_phi, a, C_pair):
    """Move the nearest interior mu and nu grid lines onto the third centre (Section 2.2,
    Fig. 2 A->B) and return (mu, nu, (mu_rows, nu_rows, phi_cells)), the rows/cells of the
    volume elements that touch it, or None when the centre lies outside mu_max (no change).

    Off the focal axis the touching cells are the 8 of Fig. 2; on the axis every phi cell
    touches it, and the axis line itself (mu = 0 or nu = 0, pi) never moves.
    """
    n_mu, n_nu = len(mu) - 1, len(nu) - 1
    if n_mu < 2 or n_nu < 2:
        raise ValueError("a refined grid needs N_mu >= 2 and N_nu >= 2")
    mu_c, nu_c, rho = third_centre_coords(a, C_pair)
    if mu_c >= mu[-1]:
        return None
    mu, nu = mu.copy(), nu.copy()
    on_axis = rho <= ON_AXIS_TOL * a
    zc = C_pair[2]
    if on_axis and abs(zc) < a:  # on the segment between the foci: mu_C = 0
        mu_rows = (0,)
    else:
        i = 1 + int(np.argmin(np.abs(mu[1:n_mu] - mu_c)))
        mu[i] = mu_c
        mu_rows = (i - 1, i)
    if on_axis and abs(zc) >= a:  # on the axis beyond A (nu = 0) or beyond B (nu = pi)
        nu_rows = (0,) if zc > 0 else (n_nu - 1,)
    else:
        j = 1 + int(np.argmin(np.abs(nu[1:n_nu] - nu_c)))
        nu[j] = nu_c
        nu_rows = (j - 1, j)
    phi_cells = tuple(range(n_phi)) if on_axis else tuple(sorted({n_phi - 1, 0}))
    return mu, nu, (mu_rows, nu_rows, phi_cells)


def grid_cells(spec, a, C_pair=None):
    """Volume elements (mu0, mu1, nu0, nu1, phi0, phi1) of a pair grid (Algorithm 1), with
    the cells touching a third centre split N_SP ways in each of mu, nu, phi (Section 2.2).

    Order: untouched cells in (i, j, k) order, then for each touching cell in (i, j, k)
    order its N_SP^3 sub-cells in (si, sj, sk) order.
    """
    mu, nu, phi = cell_edges(spec, a)
    n_mu, n_nu, n_phi, n_sp = spec[0], spec[1], spec[2], spec[6]
    touch = None
    if C_pair is not None:
        res = place_third_centre(mu, nu, n_phi, a, C_pair)
        if res is not None:
            mu, nu, touch = res
    regular, split = [], []
    for i in range(n_mu):
        for j in range(n_nu):
            for k in range(n_phi):
                box = (mu[i], mu[i + 1], nu[j], nu[j + 1], phi[k], phi[k + 1])
                if touch and i in touch[0] and j in touch[1] and k in touch[2]:
                    split.append(box)
                else:
                    regular.append(box)
    boxes = list(regular)
    for (m0, m1, n0, n1, p0, p1) in split:
        for si in range(n_sp):
            for sj in range(n_sp):
                for sk in range(n_sp):
                    boxes.append((m0 + (m1 - m0) * si / n_sp, m0 + (m1 - m0) * (si + 1) / n_sp,
                                  n0 + (n1 - n0) * sj / n_sp, n0 + (n1 - n0) * (sj + 1) / n_sp,
                                  p0 + (p1 - p0) * sk / n_sp, p0 + (p1 - p0) * (sk + 1) / n_sp))
    return np.array(boxes, dtype=float).reshape(-1, 6)


# ----------------------------------------------------------------------------------------
# Quadrature points and weights (eqs 2-6, 9-11; Algorithm 2)
# ----------------------------------------------------------------------------------------

def grid_points(boxes, q, a, M, Rm):
    """Gauss-Legendre points of every volume element, mapped to the molecule frame.

    Returns dict with P (K,3) molecule coordinates, w (K,) weights
    w = (g_i dmu/2)(g_j dnu/2)(g_k dphi/2) a^3 sinh mu sin nu (sinh^2 mu + sin^2 nu)
    (eqs 10-11, Jacobian at the node), rA, rB (eqs 5-6 in the cancellation-free form
    2a(sinh^2(mu/2) + sin^2(nu/2)) and 2a(sinh^2(mu/2) + cos^2(nu/2))), and dA, dB, the
    molecule-frame offsets of the point from A and B (z' offset a(cosh mu cos nu -+ 1)
    written as 2a(sinh^2(mu/2) cos nu -+ sin^2 / cos^2 (nu/2))).
    """
    qm, qn, qp = q
    xm, gm = gauss_legendre(qm)
    xn, gn = gauss_legendre(qn)
    xp, gp = gauss_legendre(qp)
    b = np.asarray(boxes)
    cm, hm = 0.5 * (b[:, 0] + b[:, 1]), 0.5 * (b[:, 1] - b[:, 0])
    cn, hn = 0.5 * (b[:, 2] + b[:, 3]), 0.5 * (b[:, 3] - b[:, 2])
    cp, hp = 0.5 * (b[:, 4] + b[:, 5]), 0.5 * (b[:, 5] - b[:, 4])
    mu = (cm[:, None] + hm[:, None] * xm[None, :])[:, :, None, None]
    nu = (cn[:, None] + hn[:, None] * xn[None, :])[:, None, :, None]
    ph = (cp[:, None] + hp[:, None] * xp[None, :])[:, None, None, :]
    wm = (hm[:, None] * gm[None, :])[:, :, None, None]
    wn = (hn[:, None] * gn[None, :])[:, None, :, None]
    wp = (hp[:, None] * gp[None, :])[:, None, None, :]
    shape = (len(b), qm, qn, qp)
    mu, nu, ph = [np.broadcast_to(v, shape).reshape(-1) for v in (mu, nu, ph)]
    wq = np.broadcast_to(wm * wn * wp, shape).reshape(-1)
    sh, ch = np.sinh(mu), np.cosh(mu)
    sn, cs = np.sin(nu), np.cos(nu)
    w = wq * a ** 3 * sh * sn * (sh * sh + sn * sn)
    x = a * sh * sn * np.cos(ph)
    y = a * sh * sn * np.sin(ph)
    z = a * ch * cs
    s2m = np.sinh(0.5 * mu) ** 2
    s2n = np.sin(0.5 * nu) ** 2
    c2n = np.cos(0.5 * nu) ** 2
    rA = 2 * a * (s2m + s2n)
    rB = 2 * a * (s2m + c2n)
    zA = 2 * a * (s2m * cs - s2n)
    zB = 2 * a * (s2m * cs + c2n)
    P = M[None, :] + np.stack([x, y, z], axis=1) @ Rm.T
    dA = np.stack([x, y, zA], axis=1) @ Rm.T
    dB = np.stack([x, y, zB], axis=1) @ Rm.T
    return {"P": P, "w": w, "rA": rA, "rB": rB, "dA": dA, "dB": dB}


def build_grid(job_atoms, spec, A, B, C=None):
    """Points of the pair grid (A, B), refined around atom C when C is given."""
    RA, RB = np.array(job_atoms[A][1]), np.array(job_atoms[B][1])
    RC = None if C is None else np.array(job_atoms[C][1])
    a, M, Rm = pair_frame(RA, RB, RC)
    C_pair = None if C is None else Rm.T @ (RC - M)
    boxes = grid_cells(spec, a, C_pair)
    g = grid_points(boxes, (spec[3], spec[4], spec[5]), a, M, Rm)
    g.update({"A": A, "B": B, "C": C, "a": a, "M": M, "Rm": Rm, "boxes": boxes})
    return g


# ----------------------------------------------------------------------------------------
# Real spherical harmonics and STOs (eq 1)
# ----------------------------------------------------------------------------------------

def real_spherical_harmonics(lmax, d, r):
    """Orthonormal real Y_lm(d/r), m = -l..l, for l <= lmax; returns [array (2l+1, K)].

    Y_l0 = K_l0 P_l(cos t); Y_lm = sqrt2 K_lm P_l^m(cos t) cos(m phi) (m > 0) and
    sqrt2 K_l|m| P_l^|m|(cos t) sin(|m| phi) (m < 0), K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
    P_l^m without the Condon-Shortley phase, from the standard recurrences in l.
    """
    ct = np.clip(d[:, 2] / r, -1.0, 1.0)
    st = np.hypot(d[:, 0], d[:, 1]) / r
    ph = np.arctan2(d[:, 1], d[:, 0])
    P = {}
    for m in range(lmax + 1):
        pmm = math.prod(range(1, 2 * m, 2)) * st ** m  # (2m-1)!! sin^m
        P[(m, m)] = pmm
        if m + 1 <= lmax:
            P[(m + 1, m)] = (2 * m + 1) * ct * pmm
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * ct * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    out = []
    for l in range(lmax + 1):
        Y = np.empty((2 * l + 1, len(r)))
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                Y[l + m] = K * P[(l, 0)]
            elif m > 0:
                Y[l + m] = math.sqrt(2.0) * K * P[(l, am)] * np.cos(am * ph)
            else:
                Y[l + m] = math.sqrt(2.0) * K * P[(l, am)] * np.sin(am * ph)
        out.append(Y)
    return out


def sto_norm(n, zeta):
    """Radial normalisation N = (2 zeta)^(n + 1/2) / sqrt((2n)!) of r^(n-1) e^(-zeta r)."""
    return (2.0 * zeta) ** (n + 0.5) / math.sqrt(math.factorial(2 * n))


def sto_values(shells, r, d, with_laplacian=False):
    """chi_nlm = N r^(n-1) e^(-zeta r) Y_lm (eq 1) for the shells of one centre; rows in
    shell order, m = -l..l.  With ``with_laplacian`` also returns the kinetic operand
    lap chi = [(n(n-1) - l(l+1))/r^2 - 2 n zeta / r + zeta^2] chi (derived from eq 1)."""
    if not shells:
        z = np.zeros((0, len(r)))
        return (z, z) if with_laplacian else z
    lmax = max(s[2] for s in shells)
    Y = real_spherical_harmonics(lmax, d, r)
    rows, laps = [], []
    for (_, n, l, zeta) in shells:
        radial = sto_norm(n, zeta) * r ** (n - 1) * np.exp(-zeta * r)
        chi = radial[None, :] * Y[l]
        rows.append(chi)
        if with_laplacian:
            f = (n * (n - 1) - l * (l + 1)) / r ** 2 - 2 * n * zeta / r + zeta * zeta
            laps.append(f[None, :] * chi)
    F = np.concatenate(rows, axis=0)
    if with_laplacian:
        return F, np.concatenate(laps, axis=0)
    return F


def one_centre_st(shells):
    """Overlap and kinetic blocks of the functions of one centre (eq 1), from their closed
    forms (the reading of Table 1 this module takes: one-centre S and T are not integrated on
    a grid).  With I(k) = int_0^inf r^k e^(-(zeta_a + zeta_b) r) dr = k! / (zeta_a + zeta_b)^(k+1),
    same l and m:  S_ab = N_a N_b I(n_a + n_b),
    T_ab = -1/2 N_a N_b [(n_b(n_b - 1) - l(l + 1)) I(n_a + n_b - 2) - 2 n_b zeta_b I(n_a + n_b - 1)
                         + zeta_b^2 I(n_a + n_b)]
    (the radial Laplacian of r^(n-1) e^(-zeta r) written out; symmetrised); 0 otherwise."""
    fns = [(n, l, m, z) for (_, n, l, z) in shells for m in range(-l, l + 1)]
    nf = len(fns)
    Sm, Tm = np.zeros((nf, nf)), np.zeros((nf, nf))
    for a, (na, la, ma, za) in enumerate(fns):
        for b, (nb, lb, mb, zb) in enumerate(fns):
            if la != lb or ma != mb:
                continue
            zs = za + zb
            I = lambda k: math.factorial(k) / zs ** (k + 1)
            NN = sto_norm(na, za) * sto_norm(nb, zb)
            Sm[a, b] = NN * I(na + nb)
            Tm[a, b] = -0.5 * NN * ((nb * (nb - 1) - lb * (lb + 1)) * I(na + nb - 2)
                                    - 2 * nb * zb * I(na + nb - 1) + zb * zb * I(na + nb))
    return Sm, 0.5 * (Tm + Tm.T)


# ----------------------------------------------------------------------------------------
# Incomplete gamma functions of integer order and the auxiliary potential (eqs 15-16)
# ----------------------------------------------------------------------------------------

def upper_gamma_int(k, x):
    """Gamma(k, x) = (k-1)! e^-x sum_{j<k} x^j / j!  (k >= 1 integer)."""
    x = np.asarray(x, float)
    s = np.zeros_like(x)
    term = np.ones_like(x)
    for j in range(k):
        if j > 0:
            term = term * x / j
        s = s + term
    return math.factorial(k - 1) * np.exp(-x) * s


def lower_gamma_int(k, x):
    """gamma(k, x) for integer k >= 1: the series x^k e^-x sum_i x^i / (k (k+1) .. (k+i))
    for x < k (no cancellation), (k-1)! - Gamma(k, x) for x >= k."""
    x = np.asarray(x, float)
    out = np.empty_like(x)
    small = x < k
    if np.any(small):
        xs = x[small]
        term = np.full_like(xs, 1.0 / k)
        total = term.copy()
        i = 0
        while True:
            i += 1
            term = term * xs / (k + i)
            total = total + term
            if np.all(term <= 1e-17 * total) or i > 1000:
                break
        out[small] = xs ** k * np.exp(-xs) * total
    if np.any(~small):
        out[~small] = math.factorial(k - 1) - upper_gamma_int(k, x[~small])
    return out


def aux_potential_values(shells, r, d):
    """Coulomb potential V^P(r) = int chi_P(r') / |r - r'| dr' of each aux function (eq 16),
    from the Laplace expansion of 1/r12 for chi_P = N s^(n-1) e^(-zeta s) Y_lm:
    V^P = 4 pi/(2l+1) N Y_lm(r^) [ r^(-l-1) gamma(n+l+2, zeta r)/zeta^(n+l+2)
                                   + r^l Gamma(n-l+1, zeta r)/zeta^(n-l+1) ]."""
    if not shells:
        return np.zeros((0, len(r)))
    lmax = max(s[2] for s in shells)
    Y = real_spherical_harmonics(lmax, d, r)
    rows = []
    for (_, n, l, zeta) in shells:
        x = zeta * r
        inner = lower_gamma_int(n + l + 2, x) / zeta ** (n + l + 2) * r ** (-l - 1)
        outer = upper_gamma_int(n - l + 1, x) / zeta ** (n - l + 1) * r ** l
        radial = 4 * math.pi / (2 * l + 1) * sto_norm(n, zeta) * (inner + outer)
        rows.append(radial[None, :] * Y[l])
    return np.concatenate(rows, axis=0)


# ----------------------------------------------------------------------------------------
# Molecule assembly (Section 4: integrals over subsets of at most 3 atoms)
# ----------------------------------------------------------------------------------------

def nearest_other(atoms, A):
    """Nearest other atom to A; ties go to the lower index."""
    RA = np.array(atoms[A][1])
    best, bd = None, None
    for B in range(len(atoms)):
        if B == A:
            continue
        dist = float(np.linalg.norm(RA - np.array(atoms[B][1])))
        if bd is None or dist < bd:
            best, bd = B, dist
    return best


def grid_key(atoms, A, B, C):
    """The one grid that integrates a term whose basis functions sit on A and B and whose
    operator / aux function sits on C: its distinct centres decide (one centre: the pair
    grid of that atom and its nearest neighbour; two: their pair grid; three: the pair grid
    of A, B refined around C)."""
    s = sorted({A, B, C})
    if len(s) == 1:
        X, Y = s[0], nearest_other(atoms, s[0])
        return ("base", min(X, Y), max(X, Y))
    if len(s) == 2:
        return ("base", s[0], s[1])
    return ("ref", min(A, B), max(A, B), C)


def _shells_by_atom(shells, n_atoms):
    if any(shells[i][0] > shells[i + 1][0] for i in range(len(shells) - 1)):
        raise ValueError("shells must be grouped by atom in ascending atom order")
    out = [[] for _ in range(n_atoms)]
    offs = [[] for _ in range(n_atoms)]
    off = 0
    for sh in shells:
        out[sh[0]].append(sh)
        offs[sh[0]].append(off)
        off += 2 * sh[2] + 1
    starts = []
    for a in range(n_atoms):
        starts.append(offs[a][0] if offs[a] else off)
    return out, starts


class _GridCache:
    """Builds each grid once and evaluates each centre's functions on it once."""

    def __init__(self, job):
        self.job = job
        self.grids = {}
        self.vals = {}
        self.basis, _ = _shells_by_atom(job.basis, job.n_atoms)
        self.aux, _ = _shells_by_atom(job.aux, job.n_atoms)

    def grid(self, key):
        if key not in self.grids:
            if key[0] == "base":
                _, A, B = key
                self.grids[key] = build_grid(self.job.atoms, self.job.spec_for_pair(A, B), A, B)
            else:
                _, A, B, C = key
                self.grids[key] = build_grid(self.job.atoms, self.job.spec_for_pair(A, B), A, B, C)
        return self.grids[key]

    def rd(self, key, X):
        """(r, d) of the grid's points from atom X: the PS forms for the foci."""
        g = self.grid(key)
        if X == g["A"]:
            return g["rA"], g["dA"]
        if X == g["B"]:
            return g["rB"], g["dB"]
        d = g["P"] - np.array(self.job.atoms[X][1])[None, :]
        return np.sqrt(np.sum(d * d, axis=1)), d

    def basis_vals(self, key, X):
        k = (key, "b", X)
        if k not in self.vals:
            r, d = self.rd(key, X)
            self.vals[k] = sto_values(self.basis[X], r, d, with_laplacian=True)
        return self.vals[k]

    def aux_vals(self, key, X):
        k = (key, "a", X)
        if k not in self.vals:
            r, d = self.rd(key, X)
            self.vals[k] = sto_values(self.aux[X], r, d)
        return self.vals[k]

    def aux_pot(self, key, X):
        k = (key, "p", X)
        if k not in self.vals:
            r, d = self.rd(key, X)
            self.vals[k] = aux_potential_values(self.aux[X], r, d)
        return self.vals[k]


def compute(job, mask=None, with_abs=True, j3_triples=None, pairs=None, aux_pairs=None):
    """All requested integral matrices of a job on their PS grids, FP64.

    Returns {"S","T","V": (n_bf, n_bf), "J2": (n_aux, n_aux), "J3": (n_aux, n_bf, n_bf)}
    for the classes in ``mask``, and with ``with_abs`` the matching sums of absolute terms
    (keys "absS", ...) that measure how much cancellation each element's sum carries.
    ``j3_triples`` restricts J3 to the listed (C_aux, A, B) atom blocks, ``pairs`` restricts
    S, T, V to the listed (A, B) atom blocks and ``aux_pairs`` J2 to the listed (C, D) blocks
    (A <= B, C <= D; the other blocks stay 0).
    Quadrature per block is eq 9: sum_p w_p f(p) O(p) g(p).
    """
    mask = job.mask if mask is None else mask
    nat = job.n_atoms
    _, bstart = _shells_by_atom(job.basis, nat)
    _, astart = _shells_by_atom(job.aux, nat)
    bcount = [sum(2 * s[2] + 1 for s in job.basis if s[0] == X) for X in range(nat)]
    acount = [sum(2 * s[2] + 1 for s in job.aux if s[0] == X) for X in range(nat)]
    cache = _GridCache(job)
    nb, na = job.n_bf, job.n_aux
    out = {}

    def put(name, shape):
        out[name] = np.zeros(shape)
        if with_abs:
            out["abs" + name] = np.zeros(shape)

    if mask & S:
        put("S", (nb, nb))
    if mask & T:
        put("T", (nb, nb))
    if mask & V:
        put("V", (nb, nb))
    if mask & J2:
        put("J2", (na, na))
    if mask & J3:
        put("J3", (na, nb, nb))

    def bsl(X):
        return slice(bstart[X], bstart[X] + bcount[X])

    def asl(X):
        return slice(astart[X], astart[X] + acount[X])

    for A in range(nat):
        for B in range(A, nat):
            if bcount[A] == 0 or bcount[B] == 0:
                continue
            if pairs is not None and (A, B) not in pairs:
                continue
            if mask & (S | T) and A == B:
                # one centre: closed forms (no cancellation: the absolute-term sum is |value|)
                Sm, Tm = one_centre_st([sh for sh in job.basis if sh[0] == A])
                if mask & S:
                    out["S"][bsl(A), bsl(A)] = Sm
                    if with_abs:
                        out["absS"][bsl(A), bsl(A)] = np.abs(Sm)
                if mask & T:
                    out["T"][bsl(A), bsl(A)] = Tm
                    if with_abs:
                        out["absT"][bsl(A), bsl(A)] = np.abs(Tm)
            elif mask & (S | T):
                key = grid_key(job.atoms, A, B, A)
                g = cache.grid(key)
                w = g["w"]
                FA, LA = cache.basis_vals(key, A)
                FB, LB = cache.basis_vals(key, B)
                if mask & S:
                    blk = (FA * w) @ FB.T
                    _put_sym(out["S"], bsl(A), bsl(B), blk)
                    if with_abs:
                        _put_sym(out["absS"], bsl(A), bsl(B), np.abs(FA * w) @ np.abs(FB).T)
                if mask & T:
                    blk = -0.25 * ((FA * w) @ LB.T + (LA * w) @ FB.T)
                    _put_sym(out["T"], bsl(A), bsl(B), blk)
                    if with_abs:
                        ab = 0.25 * (np.abs(FA * w) @ np.abs(LB).T + np.abs(LA * w) @ np.abs(FB).T)
                        _put_sym(out["absT"], bsl(A), bsl(B), ab)
            if mask & V:
                blk = np.zeros((bcount[A], bcount[B]))
                ab = np.zeros_like(blk)
                for C in range(nat):
                    Z = job.atoms[C][0]
                    key = grid_key(job.atoms, A, B, C)
                    g = cache.grid(key)
                    rC, _ = cache.rd(key, C)
                    FA, _ = cache.basis_vals(key, A)
                    FB, _ = cache.basis_vals(key, B)
                    blk += -Z * ((FA * (g["w"] / rC)) @ FB.T)
                    if with_abs:
                        ab += abs(Z) * (np.abs(FA * (g["w"] / rC)) @ np.abs(FB).T)
                if A == B:
                    blk = 0.5 * (blk + blk.T)
                    ab = 0.5 * (ab + ab.T)
                _put_sym(out["V"], bsl(A), bsl(B), blk)
                if with_abs:
                    _put_sym(out["absV"], bsl(A), bsl(B), ab)

    if mask & J2:
        for C in range(nat):
            for D in range(C, nat):
                if acount[C] == 0 or acount[D] == 0:
                    continue
                if aux_pairs is not None and (C, D) not in aux_pairs:
                    continue
                key = grid_key(job.atoms, C, D, C)
                g = cache.grid(key)
                w = g["w"]
                UC, UD = cache.aux_pot(key, C), cache.aux_pot(key, D)
                GC, GD = cache.aux_vals(key, C), cache.aux_vals(key, D)
                blk = 0.5 * ((UC * w) @ GD.T + ((UD * w) @ GC.T).T)
                _put_sym(out["J2"], asl(C), asl(D), blk)
                if with_abs:
                    ab = 0.5 * (np.abs(UC * w) @ np.abs(GD).T + (np.abs(UD * w) @ np.abs(GC).T).T)
                    _put_sym(out["absJ2"], asl(C), asl(D), ab)

    if mask & J3:
        triples = j3_triples
        if triples is None:
            triples = [(C, A, B) for C in range(nat) for A in range(nat) for B in range(A, nat)]
        for (C, A, B) in triples:
            if A > B:
                A, B = B, A
            if acount[C] == 0 or bcount[A] == 0 or bcount[B] == 0:
                continue
            key = grid_key(job.atoms, A, B, C)
            g = cache.grid(key)
            UwC = cache.aux_pot(key, C) * g["w"]
            FA, _ = cache.basis_vals(key, A)
            FB, _ = cache.basis_vals(key, B)
            blk = np.empty((acount[C], bcount[A], bcount[B]))
            ab = np.empty_like(blk) if with_abs else None
            for i in range(bcount[A]):
                blk[:, i, :] = (UwC * FA[i]) @ FB.T
                if with_abs:
                    ab[:, i, :] = np.abs(UwC * FA[i]) @ np.abs(FB).T
            if A == B:
                blk = 0.5 * (blk + blk.transpose(0, 2, 1))
                if with_abs:
                    ab = 0.5 * (ab + ab.transpose(0, 2, 1))
            out["J3"][asl(C), bsl(A), bsl(B)] = blk
            out["J3"][asl(C), bsl(B), bsl(A)] = blk.transpose(0, 2, 1)
            if with_abs:
                out["absJ3"][asl(C), bsl(A), bsl(B)] = ab
                out["absJ3"][asl(C), bsl(B), bsl(A)] = ab.transpose(0, 2, 1)
    out["_grids"] = {k: len(g["w"]) for k, g in cache.grids.items()}
    return out


def _put_sym(M, rs, cs, blk):
    """Write a block and its mirror; a diagonal block is symmetrised first."""
    if rs == cs:
        blk = 0.5 * (blk + blk.T)
    M[rs, cs] = blk
    M[cs, rs] = blk.T


def rmse(ref, g):
    """Root mean square error over all elements (eq 13)."""
    ref, g = np.asarray(ref), np.asarray(g)
    return float(np.sqrt(np.mean((ref - g) ** 2)))


def contractions(job, mask=None):
    """Useful point-basis^2 contractions of a job: for every grid block the oracle sums,
    rows x cols x points (J3 blocks count each (P, i<=j) once on one-atom pairs)."""
    mask = job.mask if mask is None else mask
    nat = job.n_atoms
    bcount = [sum(2 * s[2] + 1 for s in job.basis if s[0] == X) for X in range(nat)]
    acount = [sum(2 * s[2] + 1 for s in job.aux if s[0] == X) for X in range(nat)]
    npts = {}

    def K(key):
        if key not in npts:
            spec = job.spec_for_pair(key[1], key[2])
            q3 = spec[3] * spec[4] * spec[5]
            base = spec[0] * spec[1] * spec[2]
            if key[0] == "ref":
                # point count needs the geometry: build the cell list (cheap)
                RA, RB, RC = (np.array(job.atoms[i][1]) for i in key[1:])
                a, M, Rm = pair_frame(RA, RB, RC)
                base = len(grid_cells(spec, a, Rm.T @ (RC - M)))
            npts[key] = base * q3
        return npts[key]

    total = 0
    for A in range(nat):
        for B in range(A, nat):
            nab = bcount[A] * bcount[B] if A != B else bcount[A] * (bcount[A] + 1) // 2
            if mask & S:
                total += nab * K(grid_key(job.atoms, A, B, A))
            if mask & T:
                total += nab * K(grid_key(job.atoms, A, B, A))
            if mask & V:
                for C in range(nat):
                    total += nab * K(grid_key(job.atoms, A, B, C))
            if mask & J3:
                for C in range(nat):
                    total += acount[C] * nab * K(grid_key(job.atoms, A, B, C))
    if mask & J2:
        for C in range(nat):
            for D in range(C, nat):
                ncd = acount[C] * acount[D] if C != D else acount[C] * (acount[C] + 1) // 2
                total += ncd * K(grid_key(job.atoms, C, D, C))
    return total
