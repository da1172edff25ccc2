"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: closed-form 1s-1s integrals (mpmath), textbook
Gauss-Legendre rules, scipy's Legendre functions and incomplete gamma functions, Poisson's
equation and the multipole limit for V^P, finite-difference Laplacians, exact partition
invariants of the grid, symmetry and permutation equivariance, and the SO2 overlap
eigenvalue printed in Section 4 of the paper.
"""
import math

import numpy as np
import pytest

import oracle
import synth

mp = pytest.importorskip("mpmath")
scipy_special = pytest.importorskip("scipy.special")

import closed_forms as cf  # noqa: E402  (needs mpmath)

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

# A grid converged to ~1e-12 for the exponents used below (Q = 6 per dimension).
CONVERGED = (24, 16, 8, 6, 6, 6, 3)
# Coulomb integrands carry the 1/r tail of V^P: a longer radial grid (larger mu_max).
COULOMB = (48, 24, 8, 6, 6, 6, 3)


def _diatomic(R, shells_a, shells_b, aux_a=(), aux_b=(), spec=CONVERGED, Z=(1, 1)):
    atoms = [(Z[0], (0.0, 0.0, 0.0)), (Z[1], (0.0, 0.0, R))]
    basis = [(0,) + tuple(s) for s in shells_a] + [(1,) + tuple(s) for s in shells_b]
    aux = [(0,) + tuple(s) for s in aux_a] + [(1,) + tuple(s) for s in aux_b]
    return synth.Job("pin", atoms, basis, aux, [spec], oracle.ALL)


# ---------------------------------------------------------------- Gauss-Legendre

def test_gauss_legendre_q4_closed_form():
    x, w = oracle.gauss_legendre(4)
    r = math.sqrt(6.0 / 5.0)
    xin, xout = math.sqrt(3 / 7 - 2 / 7 * r), math.sqrt(3 / 7 + 2 / 7 * r)
    np.testing.assert_allclose(x, [-xout, -xin, xin, xout], rtol=0, atol=1e-15)
    win, wout = (18 + math.sqrt(30)) / 36, (18 - math.sqrt(30)) / 36
    np.testing.assert_allclose(w, [wout, win, win, wout], rtol=0, atol=1e-15)


@pytest.mark.parametrize("q", range(1, 13))
def test_gauss_legendre_matches_numpy_and_is_exact(q):
    x, w = oracle.gauss_legendre(q)
    xr, wr = np.polynomial.legendre.leggauss(q)
    np.testing.assert_allclose(x, xr, atol=2e-15)
    np.testing.assert_allclose(w, wr, atol=2e-15)
    for deg in range(2 * q):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.sum(w * x ** deg) - exact) < 1e-14


# ---------------------------------------------------------------- grid geometry

def test_focal_distances_and_offsets_match_cartesian():
    job = synth.triatomic_oh2(1)
    g = oracle.build_grid(job.atoms, (6, 5, 4, 3, 3, 3, 2), 0, 1)
    RA, RB = np.array(job.atoms[0][1]), np.array(job.atoms[1][1])
    np.testing.assert_allclose(g["rA"], np.linalg.norm(g["P"] - RA, axis=1), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(g["rB"], np.linalg.norm(g["P"] - RB, axis=1), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(g["dA"], g["P"] - RA, atol=1e-13)
    np.testing.assert_allclose(g["dB"], g["P"] - RB, atol=1e-13)
    np.testing.assert_allclose(np.linalg.norm(g["dA"], axis=1), g["rA"], rtol=1e-13)


def _spheroid_volume(a, mu_max):
    return 4 * math.pi / 3 * a ** 3 * math.cosh(mu_max) * math.sinh(mu_max) ** 2


@pytest.mark.parametrize("spec", [(15, 10, 6, 8, 4, 4, 3), (20, 15, 8, 8, 4, 4, 3), (12, 9, 5, 9, 4, 3, 2)])
def test_weight_sum_is_truncated_spheroid_volume(spec):
    """Sum of weights = (4 pi/3) a^3 cosh(mu_max) sinh^2(mu_max).  Q_mu = 8 keeps the
    Gauss-Legendre error of the wide outer mu cells (integrand ~ e^{3 mu}) below 1e-11."""
    job = synth.triatomic_oh2(2)
    g = oracle.build_grid(job.atoms, spec, 0, 1)
    a = g["a"]
    mu_max = 2.3 * a ** 0.25 * math.atanh(spec[0] / (spec[0] + 1.0))
    vol = _spheroid_volume(a, mu_max)
    assert abs(g["w"].sum() / vol - 1) < 1e-11


def test_weight_sum_cellwise_closed_form():
    """Each cell's weights integrate a^3 sinh mu sin nu (sinh^2 mu + sin^2 nu) over the cell
    (eq 11); the cell integral has a closed form; Q=6 makes GL accurate to ~1e-14 per cell."""
    job = synth.h2_fp64(0)
    spec = (6, 5, 3, 6, 6, 6, 2)
    g = oracle.build_grid(job.atoms, spec, 0, 1)
    a = g["a"]
    q3 = 6 ** 3
    for c, (m0, m1, n0, n1, p0, p1) in enumerate(g["boxes"]):
        sh3 = (math.cosh(m1) ** 3 / 3 - math.cosh(m1)) - (math.cosh(m0) ** 3 / 3 - math.cosh(m0))
        sh1 = math.cosh(m1) - math.cosh(m0)
        s1 = math.cos(n0) - math.cos(n1)
        s3 = (-math.cos(n1) + math.cos(n1) ** 3 / 3) - (-math.cos(n0) + math.cos(n0) ** 3 / 3)
        exact = a ** 3 * (p1 - p0) * (sh3 * s1 + sh1 * s3)
        got = g["w"][c * q3:(c + 1) * q3].sum()
        assert abs(got / exact - 1) < 1e-11


def test_third_centre_refinement_point_count_and_partition():
    job = synth.triatomic_oh2(0)
    spec = job.specs[0]
    base = oracle.build_grid(job.atoms, spec, 0, 1)
    ref = oracle.build_grid(job.atoms, spec, 0, 1, 2)
    n_cells = spec[0] * spec[1] * spec[2]
    q3 = spec[3] * spec[4] * spec[5]
    assert len(ref["w"]) == (n_cells - 8 + 8 * spec[6] ** 3) * q3 == 166912
    assert len(base["w"]) == n_cells * q3 == 153600
    # any partition of the truncated spheroid is a valid quadrature of its volume
    assert abs(ref["w"].sum() / base["w"].sum() - 1) < 1e-10
    # the third centre lies at phi = 0 on moved mu and nu lines
    RC = np.array(job.atoms[2][1])
    Cp = ref["Rm"].T @ (RC - ref["M"])
    assert abs(Cp[1]) < 1e-12 and Cp[0] > 0
    mu_c, nu_c, _ = oracle.third_centre_coords(ref["a"], Cp)
    b = ref["boxes"]
    assert np.any(np.abs(b[:, 0] - mu_c) < 1e-15) and np.any(np.abs(b[:, 2] - nu_c) < 1e-15)
    # refinement leaves a centre-free integrand's sum where the base grid has it
    f_ref = np.exp(-np.linalg.norm(ref["P"] - RC, axis=1))
    f_base = np.exp(-np.linalg.norm(base["P"] - RC, axis=1))
    exact = 8 * math.pi  # int e^{-r} over all space; the grid holds nearly all of it
    assert abs(np.dot(ref["w"], f_ref) - exact) < abs(np.dot(base["w"], f_base) - exact) + 1e-9


def test_third_centre_on_axis_splits_every_phi_cell():
    atoms = [(1, (0.0, 0.0, 0.0)), (1, (0.0, 0.0, 1.5)), (1, (0.0, 0.0, 3.4))]
    spec = (10, 8, 5, 8, 8, 3, 2)  # Q_mu, Q_nu = 8: GL error far below the tolerance
    ref = oracle.build_grid(atoms, spec, 0, 1, 2)
    base = oracle.build_grid(atoms, spec, 0, 1)
    n_touch = 2 * 1 * 5
    assert len(ref["w"]) == (10 * 8 * 5 - n_touch + n_touch * 8) * 8 * 8 * 3
    assert abs(ref["w"].sum() / base["w"].sum() - 1) < 1e-11


def test_third_centre_outside_mu_max_leaves_grid_unchanged():
    atoms = [(1, (0.0, 0.0, 0.0)), (1, (0.0, 0.0, 1.4)), (1, (300.0, 0.0, 0.7))]
    spec = (10, 8, 4, 3, 3, 3, 3)
    ref = oracle.build_grid(atoms, spec, 0, 1, 2)
    assert len(ref["w"]) == 10 * 8 * 4 * 27


# ---------------------------------------------------------------- harmonics, STOs

def test_real_harmonics_match_scipy():
    rng = np.random.default_rng(3)
    d = rng.normal(size=(200, 3))
    r = np.linalg.norm(d, axis=1)
    theta = np.arccos(d[:, 2] / r)
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = oracle.real_spherical_harmonics(6, d, r)
    for l in range(7):
        for m in range(-l, l + 1):
            am = abs(m)
            if hasattr(scipy_special, "sph_harm_y"):
                c = scipy_special.sph_harm_y(l, am, theta, phi)
            else:
                c = scipy_special.sph_harm(am, l, phi, theta)
            cs = (-1) ** am  # remove the Condon-Shortley phase
            ref = c.real if m == 0 else math.sqrt(2) * cs * (c.real if m > 0 else c.imag)
            np.testing.assert_allclose(Y[l][l + m], ref, atol=1e-13)


def test_real_harmonics_addition_theorem():
    rng = np.random.default_rng(4)
    d = rng.normal(size=(100, 3))
    r = np.linalg.norm(d, axis=1)
    for l, Y in enumerate(oracle.real_spherical_harmonics(7, d, r)):
        np.testing.assert_allclose(np.sum(Y * Y, axis=0), (2 * l + 1) / (4 * math.pi), rtol=1e-13)


@pytest.mark.parametrize("shell", [(1, 0, 1.0), (2, 0, 0.9), (2, 1, 1.5), (3, 2, 2.0), (4, 3, 1.3), (5, 4, 2.2)])
def test_sto_unit_self_overlap(shell):
    job = _diatomic(1.6, [shell], [(1, 0, 1.0)], spec=(32, 20, 10, 6, 6, 6, 3))
    out = oracle.compute(job, mask=oracle.S, with_abs=False)
    nf = 2 * shell[1] + 1
    np.testing.assert_allclose(np.diag(out["S"])[:nf], 1.0, rtol=0, atol=2e-11)
    # orthogonality within the shell
    assert np.max(np.abs(out["S"][:nf, :nf] - np.eye(nf))) < 2e-11


@pytest.mark.parametrize("n,l,zeta", [(1, 0, 1.2), (2, 0, 0.8), (2, 1, 1.1), (3, 2, 1.7), (4, 3, 0.9)])
def test_laplacian_operand_matches_finite_difference(n, l, zeta):
    rng = np.random.default_rng(5)
    p = rng.normal(size=(20, 3)) * 1.5
    h = 1e-3
    sh = [(0, n, l, zeta)]

    def chi(pts):
        r = np.linalg.norm(pts, axis=1)
        return oracle.sto_values(sh, r, pts)

    F, L = oracle.sto_values(sh, np.linalg.norm(p, axis=1), p, with_laplacian=True)
    lap = np.zeros_like(F)
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        lap += (-chi(p + 2 * e) + 16 * chi(p + e) - 30 * F + 16 * chi(p - e) - chi(p - 2 * e)) / (12 * h * h)
    np.testing.assert_allclose(L, lap, atol=2e-6 * np.max(np.abs(L)))


# ---------------------------------------------------------------- incomplete gamma, V^P

def test_incomplete_gamma_matches_scipy():
    x = np.concatenate([np.geomspace(1e-8, 1.0, 40), np.linspace(1.0, 60.0, 120), [100.0, 300.0]])
    for k in range(1, 16):
        g = math.gamma(k)
        lo = oracle.lower_gamma_int(k, x)
        up = oracle.upper_gamma_int(k, x)
        np.testing.assert_allclose(lo, g * scipy_special.gammainc(k, x), rtol=2e-13, atol=1e-300)
        np.testing.assert_allclose(up, g * scipy_special.gammaincc(k, x), rtol=2e-13, atol=1e-300)


def test_lower_gamma_tiny_argument_against_mpmath():
    for k in (3, 7, 13):
        for x in (1e-6, 1e-3, 0.3):
            ref = float(mp.gammainc(k, 0, x))
            assert abs(oracle.lower_gamma_int(k, np.array([x]))[0] / ref - 1) < 1e-14


def test_aux_potential_1s_closed_form():
    alpha = 1.7
    r = np.geomspace(1e-4, 30.0, 50)
    d = np.stack([0 * r, 0 * r, r], axis=1)
    Vp = oracle.aux_potential_values([(0, 1, 0, alpha)], r, d)[0]
    # chi_P = sqrt(alpha^3/pi) e^{-alpha r} (N Y_00 for n = 1)
    ref = math.sqrt(alpha ** 3 / math.pi) * np.array([cf.potential_1s_unnormalised(alpha, x) for x in r])
    np.testing.assert_allclose(Vp, ref, rtol=1e-12)


@pytest.mark.parametrize("n,l,zeta", [(1, 0, 1.3), (2, 1, 0.9), (3, 2, 2.1), (4, 3, 1.4), (6, 5, 2.5), (3, 0, 1.1)])
def test_aux_potential_satisfies_poisson(n, l, zeta):
    """lap V^P = -4 pi chi_P (finite differences, 4th order)."""
    rng = np.random.default_rng(6)
    p = rng.normal(size=(12, 3)) * 1.2
    p = p[np.linalg.norm(p, axis=1) > 0.3]
    sh = [(0, n, l, zeta)]

    def V(pts):
        return oracle.aux_potential_values(sh, np.linalg.norm(pts, axis=1), pts)

    h = 2e-3
    V0 = V(p)
    lap = np.zeros_like(V0)
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        lap += (-V(p + 2 * e) + 16 * V(p + e) - 30 * V0 + 16 * V(p - e) - V(p - 2 * e)) / (12 * h * h)
    chi = oracle.sto_values(sh, np.linalg.norm(p, axis=1), p)
    np.testing.assert_allclose(lap, -4 * math.pi * chi, atol=5e-6 * max(1.0, np.max(np.abs(chi))))


@pytest.mark.parametrize("n,l,zeta", [(2, 1, 1.0), (4, 3, 1.5), (6, 5, 2.0)])
def test_aux_potential_multipole_limit(n, l, zeta):
    rng = np.random.default_rng(7)
    u = rng.normal(size=(8, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    r = np.full(8, 80.0 / zeta)
    p = u * r[:, None]
    Vp = oracle.aux_potential_values([(0, n, l, zeta)], r, p)
    q = oracle.sto_norm(n, zeta) * math.factorial(n + l + 1) / zeta ** (n + l + 2)
    Y = oracle.real_spherical_harmonics(l, p, r)[l]
    ref = 4 * math.pi / (2 * l + 1) * q * Y / r ** (l + 1)
    np.testing.assert_allclose(Vp, ref, rtol=1e-12, atol=1e-300)


# ---------------------------------------------------------------- closed-form 1s-1s integrals

@pytest.mark.parametrize("R,za,zb", [(1.4, 1.0, 1.0), (1.6, 1.3, 0.8), (2.2, 2.5, 0.9)])
def test_1s1s_overlap_kinetic_nuclear(R, za, zb):
    job = _diatomic(R, [(1, 0, za)], [(1, 0, zb)], Z=(1, 1))
    out = oracle.compute(job, mask=oracle.S | oracle.T | oracle.V, with_abs=False)
    S_ex = cf.overlap(R, za, zb)
    if za == zb:
        assert abs(S_ex - cf.overlap_equal(R, za)) < 1e-14
    assert abs(out["S"][0, 1] - S_ex) < 5e-11
    assert abs(out["S"][0, 0] - 1) < 5e-11 and abs(out["S"][1, 1] - 1) < 5e-11
    T_ex = 0.5 * (cf.kinetic(R, za, zb) + cf.kinetic(R, zb, za))
    assert abs(out["T"][0, 1] - T_ex) < 5e-10
    assert abs(out["T"][0, 0] - za * za / 2) < 5e-10
    V01 = -cf.hybrid_over_ra(R, za, zb) - cf.hybrid_over_rb(R, za, zb)
    assert abs(out["V"][0, 1] - V01) < 5e-10
    V00 = -cf.one_centre_over_r(za) - cf.other_nucleus(R, za)
    assert abs(out["V"][0, 0] - V00) < 5e-10


@pytest.mark.parametrize("R,alpha,beta", [(1.4, 1.0, 1.0), (1.8, 1.6, 0.9), (2.5, 3.0, 1.2)])
def test_1s1s_two_centre_coulomb(R, alpha, beta):
    job = _diatomic(R, [(1, 0, 1.0)], [(1, 0, 1.0)], aux_a=[(1, 0, alpha)], aux_b=[(1, 0, beta)],
                    spec=COULOMB)
    out = oracle.compute(job, mask=oracle.J2, with_abs=False)
    ref = 0.5 * (cf.coulomb_2c(R, alpha, beta) + cf.coulomb_2c(R, beta, alpha))
    assert abs(out["J2"][0, 1] - ref) < 1e-9
    assert abs(out["J2"][0, 0] - cf.coulomb_1c_equal(alpha)) < 1e-9
    assert abs(out["J2"][1, 1] - cf.coulomb_1c_equal(beta)) < 1e-9


def test_1s1s_one_centre_coulomb_unequal():
    job = _diatomic(2.0, [(1, 0, 1.0)], [(1, 0, 1.0)], aux_a=[(1, 0, 1.1), (1, 0, 2.7)], spec=COULOMB)
    out = oracle.compute(job, mask=oracle.J2, with_abs=False)
    assert abs(out["J2"][0, 1] - cf.coulomb_1c(1.1, 2.7)) < 1e-9


def test_j3_one_centre_1s_equals_j2():
    """(P|ij) with chi_i chi_j one normalised 1s squared on the same centre as P: for
    zeta_i = zeta_j = z the density chi_i^2 = (z^3/pi) e^{-2 z r} is (up to norm) a 1s aux
    function of exponent 2z, so (P|ii) = (P|Q_{2z}) * sqrt((2z)^3/pi)^-1 * z^3/pi."""
    z, alpha = 0.9, 1.3
    job = _diatomic(2.0, [(1, 0, z)], [(1, 0, 1.0)], aux_a=[(1, 0, alpha), (1, 0, 2 * z)], spec=COULOMB)
    out = oracle.compute(job, mask=oracle.J2 | oracle.J3, with_abs=False)
    scale = (z ** 3 / math.pi) / math.sqrt((2 * z) ** 3 / math.pi)
    assert abs(out["J3"][0, 0, 0] - scale * cf.coulomb_1c(alpha, 2 * z)) < 1e-9


# ---------------------------------------------------------------- invariants

def test_symmetry_and_positive_definiteness():
    job = synth.triatomic_oh2(0)
    job.specs = [(8, 6, 4, 3, 3, 3, 2)]
    out = oracle.compute(job, with_abs=False)
    for k in ("S", "T", "V", "J2"):
        assert np.max(np.abs(out[k] - out[k].T)) == 0.0
    assert np.max(np.abs(out["J3"] - out["J3"].transpose(0, 2, 1))) == 0.0


def test_coulomb_metric_positive_definite():
    """(P|Q) is a Coulomb metric: positive definite once the grid resolves it."""
    job = synth.triatomic_oh2(0)
    out = oracle.compute(job, mask=oracle.J2, with_abs=False)
    assert np.linalg.eigvalsh(out["J2"])[0] > 0


def test_permutation_equivariance():
    """Reordering the atoms permutes every matrix: the PS grid of a pair is mirror symmetric
    (nu -> pi - nu, phi -> -phi), so swapping which atom is A changes nothing but rounding."""
    job = synth.triatomic_oh2(0)
    job.specs = [(9, 7, 4, 3, 3, 3, 2)]
    perm = [2, 0, 1]  # new atom i is old atom perm[i]
    inv = np.argsort(perm)
    atoms = [job.atoms[p] for p in perm]
    basis = sorted([(int(inv[s[0]]),) + s[1:] for s in job.basis], key=lambda s: s[0])
    aux = sorted([(int(inv[s[0]]),) + s[1:] for s in job.aux], key=lambda s: s[0])
    job2 = synth.Job("perm", atoms, basis, aux, job.specs, job.mask)

    def fn_perm(shells_old, shells_new):
        # old function index of each new function
        def table(shells):
            idx, out = 0, {}
            for k, s in enumerate(shells):
                out[k] = list(range(idx, idx + 2 * s[2] + 1))
                idx += 2 * s[2] + 1
            return out
        t_old, t_new = table(shells_old), table(shells_new)
        mapping = [None] * sum(len(v) for v in t_new.values())
        used = set()
        for kn, sn in enumerate(shells_new):
            for ko, so in enumerate(shells_old):
                if ko in used or so[1:] != sn[1:] or int(inv[so[0]]) != sn[0]:
                    continue
                used.add(ko)
                for a, b in zip(t_new[kn], t_old[ko]):
                    mapping[a] = b
                break
        return np.array(mapping)

    pb = fn_perm(job.basis, basis)
    pa = fn_perm(job.aux, aux)
    o1 = oracle.compute(job, with_abs=False)
    o2 = oracle.compute(job2, with_abs=False)
    for k in ("S", "T", "V"):
        np.testing.assert_allclose(o2[k], o1[k][np.ix_(pb, pb)], rtol=0, atol=1e-12)
    np.testing.assert_allclose(o2["J2"], o1["J2"][np.ix_(pa, pa)], rtol=0, atol=1e-11)
    np.testing.assert_allclose(o2["J3"], o1["J3"][np.ix_(pa, pb, pb)], rtol=0, atol=1e-11)


def test_rotation_invariance_of_spectra():
    job = synth.triatomic_oh2(3)
    job.specs = [(22, 16, 8, 5, 5, 5, 3)]
    job.basis = [s for s in job.basis if s[3] < 6]  # keep exponents the grid resolves well
    job.aux = []
    rng = np.random.default_rng(8)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    Rot = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                    [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                    [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    atoms2 = [(Z, tuple(Rot @ np.array(p))) for Z, p in job.atoms]
    job2 = synth.Job("rot", atoms2, job.basis, [], job.specs, oracle.S | oracle.T | oracle.V)
    o1 = oracle.compute(job, mask=oracle.S | oracle.T | oracle.V, with_abs=False)
    o2 = oracle.compute(job2, mask=oracle.S | oracle.T | oracle.V, with_abs=False)
    np.testing.assert_allclose(np.linalg.eigvalsh(o1["S"]), np.linalg.eigvalsh(o2["S"]), atol=1e-9)
    np.testing.assert_allclose(np.linalg.eigvalsh(o1["T"]), np.linalg.eigvalsh(o2["T"]), atol=1e-7)
    np.testing.assert_allclose(np.linalg.eigvalsh(o1["V"]), np.linalg.eigvalsh(o2["V"]), atol=1e-6)


def test_three_centre_nuclear_attraction_grid_choice():
    """<i_A | 1/r_C | j_B> on the grids (A,B;C), (A,C;B) and (B,C;A) agree to quadrature error."""
    job = synth.triatomic_oh2(0)
    spec = (24, 18, 10, 4, 4, 4, 3)
    RC = np.array(job.atoms[2][1])
    vals = []
    shells_A = [s for s in job.basis if s[0] == 0 and s[3] < 5][:2]
    shells_B = [s for s in job.basis if s[0] == 1 and s[3] < 5][:2]
    for (X, Y, Zc) in ((0, 1, 2), (0, 2, 1), (1, 2, 0)):
        g = oracle.build_grid(job.atoms, spec, X, Y, Zc)
        P, w = g["P"], g["w"]

        def vals_at(shells, atom):
            d = P - np.array(job.atoms[atom][1])
            return oracle.sto_values(shells, np.linalg.norm(d, axis=1), d)

        FA, FB = vals_at(shells_A, 0), vals_at(shells_B, 1)
        rC = np.linalg.norm(P - RC, axis=1)
        vals.append((FA * (w / rC)) @ FB.T)
    assert np.max(np.abs(vals[0] - vals[1])) < 2e-5
    assert np.max(np.abs(vals[0] - vals[2])) < 2e-5


def test_so2_tz_smallest_overlap_eigenvalue_matches_paper():
    """Section 4 prints 1.3e-5 for the smallest eigenvalue of the SO2 TZ overlap matrix;
    basis from Table S1 (S and O, TZ column), geometry Table S2 (Angstrom), PS grid
    26/32/14, Q 4 (the paper's BP-sized grid of Table 1).  Fixture: tests/golden/so2_tz.txt."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "so2_tz.txt")
    atoms, basis, expect = _read_golden_so2(path)
    job = synth.Job("so2", atoms, basis, [], [(26, 32, 14, 4, 4, 4, 3)], oracle.S)
    out = oracle.compute(job, mask=oracle.S, with_abs=False)
    ev = np.linalg.eigvalsh(out["S"])[0]
    assert float("%.1e" % ev) == expect


def _read_golden_so2(path):
    ang = 1.0 / 0.529177210903
    atoms, basis, expect = [], [], None
    with open(path) as f:
        for line in f:
            t = line.split("#")[0].split()
            if not t:
                continue
            if t[0] == "atom":
                atoms.append((int(t[1]), tuple(float(c) * ang for c in t[2:5])))
            elif t[0] == "shell":
                l = "spdfgh".index(t[2][-1])
                basis.append((int(t[1]), l + 1, l, float(t[3])))
            elif t[0] == "expect_min_eigenvalue":
                expect = float(t[1])
    return atoms, basis, expect


def test_assembly_matches_integration_on_other_grids():
    """Each block of a triatomic's S, T, V, J2, J3 is integrated again on a different valid
    grid than the assembly rule picks: a one-centre term on its atom's pair grid with the
    other (not the nearest) neighbour (one-centre S and T, closed forms, against their
    block's largest element), a two-centre term on that pair's grid refined around
    the remaining atom, a three-centre term (A,B;C) on the grid (A,C;B).  Agreement to
    quadrature error pins which centres, nuclei and grid each element uses."""
    job = synth.triatomic_oh2(0)
    job.specs = [(22, 16, 10, 4, 4, 4, 3)]
    out = oracle.compute(job, with_abs=True)
    atoms = job.atoms
    nn = [oracle.nearest_other(atoms, X) for X in range(3)]
    grids = {}

    def other_grid(cent, basis_pair):
        s_ = sorted(set(cent))
        if len(s_) == 1:
            X = s_[0]
            Y = [q for q in range(3) if q not in (X, nn[X])][0]
            key = (min(X, Y), max(X, Y), None)
        elif len(s_) == 2:
            Z = [q for q in range(3) if q not in s_][0]
            key = (s_[0], s_[1], Z)
        else:
            A, B = basis_pair
            C = [q for q in range(3) if q not in (A, B)][0]
            key = (min(A, C), max(A, C), B)
        if key not in grids:
            grids[key] = oracle.build_grid(atoms, job.specs[0], *key)
        return grids[key]

    def vals(g, shells, X, kind):
        sh = [s_ for s_ in shells if s_[0] == X]
        d = g["P"] - np.array(atoms[X][1])
        r = np.linalg.norm(d, axis=1)
        if kind == "aux":
            return oracle.sto_values(sh, r, d)
        if kind == "pot":
            return oracle.aux_potential_values(sh, r, d)
        return oracle.sto_values(sh, r, d, with_laplacian=True)

    def sl(shells, X):
        start = sum(2 * s_[2] + 1 for s_ in shells if s_[0] < X)
        return slice(start, start + sum(2 * s_[2] + 1 for s_ in shells if s_[0] == X))

    worst = {}

    def check(k, blk, rs, one_centre=False):
        got = out[k][rs]
        scale = np.maximum(np.abs(got), out["abs" + k][rs])
        if one_centre:  # closed forms (no quadrature sum): against the block's largest element
            scale = np.maximum(scale, np.abs(got).max())
        e = np.abs(got - blk) / np.maximum(scale, 1e-6)
        worst[k] = max(worst.get(k, 0.0), float(e.max()))

    for A in range(3):
        for B in range(A, 3):
            g = other_grid((A, B), (A, B))
            (FA, LA), (FB, LB) = vals(g, job.basis, A, "b"), vals(g, job.basis, B, "b")
            w = g["w"]
            rs = (sl(job.basis, A), sl(job.basis, B))
            check("S", (FA * w) @ FB.T, rs, A == B)
            check("T", -0.25 * ((FA * w) @ LB.T + (LA * w) @ FB.T), rs, A == B)
            for C in range(3):
                gc = other_grid((A, B, C), (A, B))
                FAc, FBc = vals(gc, job.basis, A, "b")[0], vals(gc, job.basis, B, "b")[0]
                rC = np.linalg.norm(gc["P"] - np.array(atoms[C][1]), axis=1)
                part = -atoms[C][0] * ((FAc * (gc["w"] / rC)) @ FBc.T)
                worst.setdefault("Vparts", []).append((A, B, C, part))
                U = vals(gc, job.aux, C, "pot") * gc["w"]
                check("J3", np.einsum("pk,ik,jk->pij", U, FAc, FBc), (sl(job.aux, C),) + rs)
            V = sum(p_ for (a_, b_, c_, p_) in worst.pop("Vparts"))
            check("V", V, rs)
            UA, GB = vals(g, job.aux, A, "pot"), vals(g, job.aux, B, "aux")
            UB, GA = vals(g, job.aux, B, "pot"), vals(g, job.aux, A, "aux")
            check("J2", 0.5 * ((UA * w) @ GB.T + ((UB * w) @ GA.T).T), (sl(job.aux, A), sl(job.aux, B)))
    # measured: S 2.9e-5, T 1.2e-5, V 7.6e-5, J2 6.2e-6, J3 1.5e-3 (third-centre functions
    # with zeta up to 12 on the alternative grids); a wrong centre or nucleus gives O(1)
    tol = {"S": 2e-4, "T": 2e-4, "V": 1e-3, "J2": 1e-4, "J3": 1e-2}
    for k, e in worst.items():
        assert e < tol[k], (k, e)


# ---------------------------------------------------------------- convergence

def test_grid_doubling_converges():
    """Doubling the cells in mu, nu and phi moves every class by less each time (the PS rule
    converges): |X(2N) - X(4N)| < |X(N) - X(2N)| for S, T, V and (P|Q) of H2 with the
    config-1 shells (Section 3: errors fall as the grid grows)."""
    job0 = synth.h2_fp64(0)
    out = []
    for f in (1, 2, 4):
        spec = (6 * f, 4 * f, 2 * f, 4, 4, 4, 3)
        job = synth.Job("h2", job0.atoms, job0.basis, job0.aux, [spec], oracle.S | oracle.T | oracle.V | oracle.J2)
        out.append(oracle.compute(job, with_abs=False))
    for k in ("S", "T", "V", "J2"):
        d1 = np.abs(out[0][k] - out[1][k]).max()
        d2 = np.abs(out[1][k] - out[2][k]).max()
        assert d2 < 0.5 * d1, (k, d1, d2)


def test_third_centre_split_reduces_grid_choice_spread():
    """Refining the cells around the third centre (N_SP, Section 2.3 and Fig. 5) improves the
    3-centre nuclear attraction: <i_A | 1/r_C | j_B> on the grid (A,B;C), refined around C
    where 1/r_C is singular, agrees with the same integral on (A,C;B), where C is a focus and
    the singularity is absorbed by the Jacobian, 5x better with N_SP = 3 than without the
    split (N_SP = 1) on a coarse grid."""
    job = synth.triatomic_oh2(0)
    RC = np.array(job.atoms[2][1])
    shells_A = [s for s in job.basis if s[0] == 0 and s[3] < 5][:2]
    shells_B = [s for s in job.basis if s[0] == 1 and s[3] < 5][:2]

    def spread(nsp):
        vals = []
        for (X, Y, Zc) in ((0, 1, 2), (0, 2, 1)):
            g = oracle.build_grid(job.atoms, (10, 8, 6, 4, 4, 4, nsp), X, Y, Zc)
            P, w = g["P"], g["w"]

            def vals_at(shells, atom):
                d = P - np.array(job.atoms[atom][1])
                return oracle.sto_values(shells, np.linalg.norm(d, axis=1), d)

            FA, FB = vals_at(shells_A, 0), vals_at(shells_B, 1)
            rC = np.linalg.norm(P - RC, axis=1)
            vals.append((FA * (w / rC)) @ FB.T)
        return np.abs(vals[0] - vals[1]).max()

    s1, s3 = spread(1), spread(3)
    assert s3 < 0.3 * s1, (s1, s3)
