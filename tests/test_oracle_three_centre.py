"""Pins of the oracle's three-centre values against an independent integration route.

The three-centre nuclear attraction <a_A | 1/r_C | b_B> and the three-centre Coulomb integral
(P_C | a_A b_B) have no closed form for Slater functions, but through Gaussian transforms
they reduce to smooth triple integrals of the Gaussian product theorem and its moments
(``gauss_transform``), which a trapezoidal rule in logarithmic variables evaluates to ~1e-12
(checked here against the two-centre closed forms and one-centre overlaps first); here with
1s, 2s, 2p, 3d and 4f functions and a 1s aux function.  The oracle integrates the same
elements on the pair grid of A and B refined around C (Section 2.2: the nearest mu and nu
lines moved onto C, the touching cells split N_SP ways) and must converge to those values as
the grid grows.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytest.importorskip("mpmath")
import closed_forms as cf  # noqa: E402
import gauss_transform as gt  # noqa: E402

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

H = 0.25  # trapezoid step of the transform integrals (converged to ~1e-12 below)
A, B, C = (0.0, 0.0, 0.0), (0.0, 0.0, 1.4), (1.1, 0.3, 0.6)  # C off the A-B axis and plane
ZETA_A, ZETA_B, ZETA_C, ALPHA = 1.1, 0.9, 1.0, 1.4
Z = (1, 1, 2)


def test_gauss_transform_reproduces_two_centre_closed_forms():
    """With the operator on A or B the transform integrals are two-centre integrals with closed
    forms: overlap, <a|1/r_A|b>, <a|1/r_B|b>, and (e^{-alpha r_B}, e^{-alpha r_B}/r_B) times b
    as a 1s function of exponent zeta_b + alpha."""
    R, za, zb, al = 1.6, 1.3, 0.8, 1.5
    P0, P1 = (0.0, 0.0, 0.0), (0.0, 0.0, R)
    n = gt.norm1s(za) * gt.norm1s(zb)
    assert abs(n * gt.overlap_integral(za, P0, zb, P1, h=H) - cf.overlap(R, za, zb)) < 1e-12
    assert abs(gt.nuclear_attraction(za, P0, zb, P1, P0, h=H) - cf.hybrid_over_ra(R, za, zb)) < 1e-11
    assert abs(gt.nuclear_attraction(za, P0, zb, P1, P1, h=H) - cf.hybrid_over_rb(R, za, zb)) < 1e-11
    m = gt.norm1s(za) * gt.norm1s(zb + al)
    e = gt.product_integral(za, P0, zb, P1, P1, "exp", alpha=al, h=H)
    assert abs(m * e - cf.overlap(R, za, zb + al)) < 1e-12
    s = gt.product_integral(za, P0, zb, P1, P1, "screened", alpha=al, h=H)
    assert abs(m * s - cf.hybrid_over_rb(R, za, zb + al)) < 1e-11


def test_gauss_transform_2s_2p_one_centre_overlaps():
    """2s and 2p through the transform: on one centre the normalised 1s, 2s, 2p_(-1,0,1) of one
    exponent have unit norms, <1s|2s> = sqrt(3)/2 (the closed form for equal exponents) and
    every other pair is orthogonal."""
    fs = [gt.sto(1, 0, 0, 1.3), gt.sto(2, 0, 0, 1.3)] + [gt.sto(2, 1, m, 1.3) for m in (-1, 0, 1)]
    S = gt.sto_matrix(fs, A, fs, A, A, "one", h=H)
    ref = np.eye(5)
    ref[0, 1] = ref[1, 0] = math.sqrt(3.0) / 2.0
    assert np.abs(S - ref).max() < 1e-12


@pytest.fixture(scope="module")
def exact():
    vC = gt.nuclear_attraction(ZETA_A, A, ZETA_B, B, C, h=H)
    R = math.dist(A, B)
    V = (-Z[0] * cf.hybrid_over_ra(R, ZETA_A, ZETA_B) - Z[1] * cf.hybrid_over_rb(R, ZETA_A, ZETA_B)
         - Z[2] * vC)
    J3 = gt.three_index_coulomb(ALPHA, C, ZETA_A, A, ZETA_B, B, h=H)
    return V, J3


def _oracle(spec):
    atoms = [(Z[0], A), (Z[1], B), (Z[2], C)]
    basis = [(0, 1, 0, ZETA_A), (1, 1, 0, ZETA_B), (2, 1, 0, ZETA_C)]
    aux = [(2, 1, 0, ALPHA)]
    job = synth.Job("three_centre_1s", atoms, basis, aux, [spec], oracle.V | oracle.J3)
    out = oracle.compute(job, mask=oracle.V | oracle.J3, with_abs=False)
    return out["V"][0, 1], out["J3"][0, 0, 1]


def test_three_centre_values_converge_to_the_transform_integrals(exact):
    """V_ab (nuclei A, B and C; C's term on the refined grid) and (P_C|a_A b_B) approach the
    transform values as the grid grows: measured errors 7.0e-6 / 6.1e-8 on 16/12/8 (Q 4, N_SP
    2) and 1.8e-6 / 2.0e-10 on 24/16/8 (Q 6, N_SP 3); 2.7e-7 / 1.4e-11 on 32/24/12 and
    2.9e-8 / 2.2e-13 on 32/24/12 with Q 8, N_SP 4 (not run here: 8 and 20 s).  A dropped or
    misplaced third-centre term moves V_ab by ~1 and (P|ab) by ~3."""
    V, J3 = exact
    errs = []
    for spec, tv, tj in (((16, 12, 8, 4, 4, 4, 2), 1.5e-5, 2e-7), ((24, 16, 8, 6, 6, 6, 3), 4e-6, 1e-9)):
        v, j = _oracle(spec)
        errs.append((abs(v - V), abs(j - J3)))
        assert abs(v - V) < tv, (spec, v - V)
        assert abs(j - J3) < tj, (spec, j - J3)
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1]


def test_transform_values_are_three_centre():
    """The third centre matters: <a|1/r_C|b> differs from its value with C moved onto the A-B
    axis at the same distance from A (a pin that only checked an axial geometry would not see
    a lost azimuthal rotation)."""
    v_off = gt.nuclear_attraction(ZETA_A, A, ZETA_B, B, C, h=H)
    d = math.dist(A, C)
    v_axis = gt.nuclear_attraction(ZETA_A, A, ZETA_B, B, (0.0, 0.0, -d), h=H)
    assert abs(v_off - v_axis) > 1e-2
    assert np.isfinite(v_off) and 0 < v_off < 1


def test_three_centre_2s_2p_values_converge_to_the_transform_integrals():
    """The same with 2s and 2p functions (every m) on A and B, so that the harmonics and the
    rotation into the refined grid's frame (C off the A-B axis and plane) are exercised: all
    16 elements of V (nuclei A, B, C, all through the transform) and of (P_C|a_A b_B).
    Measured largest errors 1.5e-5 / 4.1e-7 on 16/12/8 (Q 4, N_SP 2), 3.4e-6 / 2.9e-10 on
    24/16/8 (Q 6, N_SP 3) and 3.7e-7 / 1.8e-11 on 32/24/12 (not run here)."""
    fa = [gt.sto(1, 0, 0, 1.1)] + [gt.sto(2, 1, m, 1.3) for m in (-1, 0, 1)]
    fb = [gt.sto(2, 0, 0, 0.9)] + [gt.sto(2, 1, m, 1.0) for m in (-1, 0, 1)]
    Vx = sum(-z * gt.sto_matrix(fa, A, fb, B, N, "coulomb", h=H) for z, N in zip(Z, (A, B, C)))
    Jx = gt.sto_three_index_matrix(ALPHA, C, fa, A, fb, B, h=H)
    atoms = [(Z[0], A), (Z[1], B), (Z[2], C)]
    basis = [(0, 1, 0, 1.1), (0, 2, 1, 1.3), (1, 2, 0, 0.9), (1, 2, 1, 1.0), (2, 1, 0, ZETA_C)]
    aux = [(2, 1, 0, ALPHA)]
    errs = []
    for spec, tv, tj in (((16, 12, 8, 4, 4, 4, 2), 3e-5, 1e-6), ((24, 16, 8, 6, 6, 6, 3), 7e-6, 1e-9)):
        job = synth.Job("three_centre_2p", atoms, basis, aux, [spec], oracle.V | oracle.J3)
        out = oracle.compute(job, mask=oracle.V | oracle.J3, with_abs=False)
        ev = np.abs(out["V"][0:4, 4:8] - Vx).max()
        ej = np.abs(out["J3"][0, 0:4, 4:8] - Jx).max()
        errs.append((ev, ej))
        assert ev < tv and ej < tj, (spec, ev, ej)
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1]


def test_gauss_transform_any_l_one_centre_overlaps():
    """The general-l route (solid harmonics fitted to scipy's, r^k e^{-zeta r} by Hermite
    derivatives of the transform weight, moments by the Gaussian recurrences): on one centre
    1s, 2s, 3s, 2p, 3d, 4f (every m) of one exponent give <nlm|n'lm> = (n + n')! /
    sqrt((2n)! (2n')!) and zero between different (l, m); and it reproduces the 2s/2p route."""
    shells = [(1, 0), (2, 0), (3, 0), (2, 1), (3, 2), (4, 3)]
    labels = [(n, l, m) for (n, l) in shells for m in range(-l, l + 1)]
    fs = [gt.sto_nlm(n, l, m, 1.3) for (n, l, m) in labels]
    S = gt.nlm_matrix(fs, A, fs, A, A, "one", h=H)
    ref = np.zeros_like(S)
    for i, (n, l, m) in enumerate(labels):
        for j, (n2, l2, m2) in enumerate(labels):
            if (l, m) == (l2, m2):
                ref[i, j] = math.factorial(n + n2) / math.sqrt(math.factorial(2 * n) * math.factorial(2 * n2))
    assert np.abs(S - ref).max() < 1e-12
    fa = [gt.sto(2, 1, m, 1.3) for m in (-1, 0, 1)]
    fb = [gt.sto(2, 0, 0, 0.9)] + [gt.sto(2, 1, m, 1.0) for m in (-1, 0, 1)]
    na = [gt.sto_nlm(2, 1, m, 1.3) for m in (-1, 0, 1)]
    nb = [gt.sto_nlm(2, 0, 0, 0.9)] + [gt.sto_nlm(2, 1, m, 1.0) for m in (-1, 0, 1)]
    assert np.abs(gt.nlm_matrix(na, A, nb, B, C, "coulomb", h=H)
                  - gt.sto_matrix(fa, A, fb, B, C, "coulomb", h=H)).max() < 1e-13


def test_three_centre_3d_4f_values_converge_to_the_transform_integrals():
    """3d functions on A and 4f on B (m = -1, 0, 2 and -2, 1, 3: the solid harmonics with one,
    three and two monomials), C off the A-B axis and plane and the only charged nucleus: the
    nine elements of V_ne (from C alone) and of (P_C|a_A b_B).  Measured largest errors 2.4e-6
    / 3.6e-6 on 16/12/8 (Q 4, N_SP 2) and 3.0e-7 / 1.2e-9 on 24/16/8 (Q 6, N_SP 3); over every
    m, 3.0e-6 / 9.8e-6, 4.9e-7 / 4.2e-9 and 4.3e-8 / 5.4e-11 on 32/24/12 (Q 6; not run here)."""
    ma, mb = (-1, 0, 2), (-2, 1, 3)
    fa = [gt.sto_nlm(3, 2, m, 1.2) for m in ma]
    fb = [gt.sto_nlm(4, 3, m, 1.0) for m in mb]
    Vx = -2.0 * gt.nlm_matrix(fa, A, fb, B, C, "coulomb", h=H)
    Jx = gt.nlm_three_index_matrix(ALPHA, C, fa, A, fb, B, h=H)
    atoms = [(0, A), (0, B), (2, C)]
    basis = [(0, 3, 2, 1.2), (1, 4, 3, 1.0), (2, 1, 0, ZETA_C)]
    aux = [(2, 1, 0, ALPHA)]
    rows, cols = [2 + m for m in ma], [5 + 3 + m for m in mb]
    errs = []
    for spec, tv, tj in (((16, 12, 8, 4, 4, 4, 2), 5e-6, 8e-6), ((24, 16, 8, 6, 6, 6, 3), 7e-7, 3e-9)):
        job = synth.Job("three_centre_df", atoms, basis, aux, [spec], oracle.V | oracle.J3)
        out = oracle.compute(job, mask=oracle.V | oracle.J3, with_abs=False)
        ev = np.abs(out["V"][np.ix_(rows, cols)] - Vx).max()
        ej = np.abs(out["J3"][0][np.ix_(rows, cols)] - Jx).max()
        errs.append((ev, ej))
        assert ev < tv and ej < tj, (spec, ev, ej)
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1]
