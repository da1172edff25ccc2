"""Pins of the RI 4-index oracle (Section 3, eq 14) against closed forms and invariants."""
import math

import numpy as np
import pytest

import oracle
from oracle import ri_oracle
import synth
import closed_forms as cf

COULOMB = (48, 24, 8, 6, 6, 6, 3)  # long radial grid: Coulomb integrands carry 1/r tails


def _random_spd(rng, n, cond=100.0):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.exp(rng.uniform(0.0, math.log(cond), n))
    return (Q * ev) @ Q.T


def test_metric_times_x_gives_x_j2_x():
    """J3 = J2 X makes eq 14 exact: sum_PQ (ij|P) [J2^-1]_PQ (Q|kl) = (X^T J2 X)[ij][kl]."""
    rng = np.random.default_rng(3)
    n, nb = 7, 3
    J2 = _random_spd(rng, n)
    X = rng.standard_normal((n, nb * nb))
    got = ri_oracle.ri_eri(J2, (J2 @ X).reshape(n, nb, nb))
    np.testing.assert_allclose(got, X.T @ J2 @ X, rtol=1e-12, atol=1e-12 * np.abs(X.T @ J2 @ X).max())


def test_cholesky_and_forward_reconstruct():
    rng = np.random.default_rng(4)
    J2 = _random_spd(rng, 9)
    L = ri_oracle.cholesky(J2)
    assert np.allclose(np.triu(L, 1), 0.0) and (np.diag(L) > 0).all()
    np.testing.assert_allclose(L @ L.T, J2, rtol=0, atol=1e-13 * np.abs(J2).max())
    X = rng.standard_normal((9, 5))
    np.testing.assert_allclose(L @ ri_oracle.forward(L, X), X, rtol=0, atol=1e-13 * np.abs(X).max())


@pytest.fixture(scope="module")
def exact_fit():
    """Two H atoms; basis 1s(za) on A, 1s(zb) on B; aux holds 1s(2 za) on A and 1s(2 zb) on B
    (plus 2s/2p that change nothing), so the densities chi_A^2 and chi_B^2 are fitted exactly."""
    R, za, zb = 1.6, 1.1, 0.8
    atoms = [(1, (0.0, 0.0, 0.0)), (1, (0.0, 0.0, R))]
    basis = [(0, 1, 0, za), (1, 1, 0, zb)]
    aux = [(0, 1, 0, 2 * za), (0, 2, 0, 1.7), (0, 2, 1, 1.9), (1, 1, 0, 2 * zb), (1, 2, 1, 1.3)]
    job = synth.Job("ri_pin", atoms, basis, aux, [COULOMB], oracle.J2 | oracle.J3)
    out = oracle.compute(job, mask=oracle.J2 | oracle.J3, with_abs=False)
    return R, za, zb, out


def test_exact_fit_one_centre_5zeta_over_8(exact_fit):
    """(aa|aa) of one normalised 1s function is 5 zeta / 8; with its density in the aux span
    eq 14 reproduces it."""
    R, za, zb, out = exact_fit
    eri = ri_oracle.ri_eri(out["J2"], out["J3"])
    assert abs(eri[0, 0] - 5 * za / 8) < 1e-12
    assert abs(eri[3, 3] - 5 * zb / 8) < 1e-12


def test_exact_fit_two_centre_repulsion(exact_fit):
    """(aa|bb) = c_a c_b (P|Q), chi^2 = c chi_P with c = zeta^1.5 / sqrt(8 pi) and (P|Q) the
    closed-form two-centre 1s-1s Coulomb integral of exponents 2 za, 2 zb."""
    R, za, zb, out = exact_fit
    eri = ri_oracle.ri_eri(out["J2"], out["J3"])
    c = lambda z: z ** 1.5 / math.sqrt(8 * math.pi)
    ref = c(za) * c(zb) * 0.5 * (cf.coulomb_2c(R, 2 * za, 2 * zb) + cf.coulomb_2c(R, 2 * zb, 2 * za))
    assert abs(eri[0, 3] - ref) < 1e-12
    assert abs(eri[3, 0] - ref) < 1e-12


def test_fitted_overlap_density_below_exact(exact_fit):
    """Coulomb-metric fitting never overestimates: (ab|ab)_RI <= (ab|ab) <= sqrt((aa|aa)(bb|bb))
    (Schwarz), the RI value of the diagonal a Gram norm >= 0."""
    R, za, zb, out = exact_fit
    eri = ri_oracle.ri_eri(out["J2"], out["J3"])
    ab = 0 * 2 + 1
    assert 0 < eri[ab, ab] <= math.sqrt((5 * za / 8) * (5 * zb / 8)) + 1e-12


def test_symmetry_psd_schwarz_h2():
    job = synth.h2_fp64(0, mask=oracle.J2 | oracle.J3)
    out = oracle.compute(job, mask=oracle.J2 | oracle.J3, with_abs=False)
    nb = job.n_bf
    eri = ri_oracle.ri_eri(out["J2"], out["J3"])
    np.testing.assert_allclose(eri, eri.T, rtol=0, atol=1e-10 * np.abs(eri).max())
    e4 = eri.reshape(nb, nb, nb, nb)
    np.testing.assert_allclose(e4, e4.transpose(1, 0, 2, 3), rtol=0, atol=1e-10 * np.abs(eri).max())
    ev = np.linalg.eigvalsh(0.5 * (eri + eri.T))
    assert ev.min() > -1e-10 * ev.max()
    d = np.sqrt(np.clip(np.diag(eri), 0, None))
    assert (np.abs(eri) <= np.outer(d, d) * (1 + 1e-10) + 1e-12).all()
