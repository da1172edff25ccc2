"""Parity of the RI 4-index assembly (Section 3, eq 14) on the GPU with the oracle.

The library factors (P|Q) = L L^T, solves B = L^-1 (P|ij) and forms (ij|kl) = sum_R B B; the
oracle writes eq 14 with a linear solve.  All FP64: on metrics of condition number kappa the
two routes agree to a few kappa * 2^-52 of the largest element, the bound written below.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import ri_oracle
import synth
import closed_forms as cf

pytestmark = pytest.mark.gpu

COULOMB = (48, 24, 8, 6, 6, 6, 3)
EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "the CUDA path needs a GPU"
    import paper_2510_15204_gb300 as P
    from paper_2510_15204_gb300 import build
    build.build()
    return P


def _random_spd(rng, n, cond=100.0):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.exp(rng.uniform(0.0, math.log(cond), n))
    return (Q * ev) @ Q.T


def _gpu_ri(P, J2, J3):
    import torch
    n = J2.shape[0]
    dJ2 = torch.tensor(J2, dtype=torch.float64, device="cuda")
    dB = torch.tensor(np.asarray(J3).reshape(n, -1), dtype=torch.float64, device="cuda")
    L, info = P.ri_factor(dJ2)
    P.ri_solve(L, dB)
    m = dB.shape[1]
    eri = P.ri_eri(dB, 0, m, 0, m)
    torch.cuda.synchronize()
    return L.cpu().numpy(), dB.cpu().numpy(), eri.cpu().numpy(), int(info.item())


@pytest.mark.parametrize("n,m", [(1, 1), (5, 7), (31, 63), (32, 64), (33, 65), (95, 130), (130, 700)])
def test_factor_solve_eri_random(P, n, m):
    rng = np.random.default_rng(n * 1000 + m)
    J2 = _random_spd(rng, n)
    X = rng.standard_normal((n, m))
    L, B, eri, info = _gpu_ri(P, J2, X)
    assert info == 0
    Lo = ri_oracle.cholesky(J2)
    assert np.abs(L - Lo).max() <= 1e3 * EPS * np.abs(Lo).max()
    Bo = ri_oracle.forward(Lo, X)
    assert np.abs(B - Bo).max() <= 1e3 * EPS * np.abs(Bo).max()
    Eo = ri_oracle.ri_eri(J2, X)
    assert np.abs(eri - Eo).max() <= 1e3 * EPS * np.abs(Eo).max()


def test_factor_in_place_and_empty(P):
    import torch
    rng = np.random.default_rng(7)
    J2 = _random_spd(rng, 40)
    d = torch.tensor(J2, device="cuda")
    L, info = P.ri_factor(d, L=d)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    np.testing.assert_allclose(d.cpu().numpy(), ri_oracle.cholesky(J2), rtol=0, atol=1e3 * EPS * 10)
    e = torch.empty((0, 0), dtype=torch.float64, device="cuda")
    L0, info0 = P.ri_factor(e)
    torch.cuda.synchronize()
    assert int(info0.item()) == 0
    B = torch.zeros((3, 0), dtype=torch.float64, device="cuda")
    P.ri_solve(torch.eye(3, dtype=torch.float64, device="cuda"), B)
    out = P.ri_eri(torch.zeros((3, 5), dtype=torch.float64, device="cuda"), 1, 0, 2, 3)
    assert out.shape == (0, 3)


def test_not_positive_definite_reports_the_pivot(P):
    import torch
    J2 = np.diag([1.0, 2.0, -1.0, 3.0])
    _, info = P.ri_factor(torch.tensor(J2, device="cuda"))
    torch.cuda.synchronize()
    assert int(info.item()) == 3
    rng = np.random.default_rng(8)
    A = _random_spd(rng, 70)
    A[50, 50] = -5.0  # leading minors up to 50 stay positive definite
    _, info = P.ri_factor(torch.tensor(A, device="cuda"))
    torch.cuda.synchronize()
    assert 1 <= int(info.item()) <= 51


def test_blocks_and_ranges(P):
    import torch
    rng = np.random.default_rng(9)
    n, m = 37, 150
    B = torch.tensor(rng.standard_normal((n, m)), device="cuda")
    full = P.ri_eri(B, 0, m, 0, m)
    blk = P.ri_eri(B, 17, 70, 90, 60)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(blk.cpu().numpy(), full.cpu().numpy()[17:87, 90:150])
    with pytest.raises(P.PsqError):
        P.ri_eri(B, 100, 60, 0, 5)
    with pytest.raises(P.PsqError):
        P.ri_eri(B, -1, 2, 0, 5)


def test_exact_fit_closed_forms_through_the_library(P):
    """The FP64 library path end to end: J2 and J3 from psq_compute, then eq 14 on the GPU;
    densities chi^2 of 1s functions lie in the aux span, so (aa|aa) = 5 zeta / 8 and (aa|bb)
    is the closed-form two-centre repulsion."""
    import torch
    R, za, zb = 1.6, 1.1, 0.8
    atoms = [(1, (0.0, 0.0, 0.0)), (1, (0.0, 0.0, R))]
    basis = [(0, 1, 0, za), (1, 1, 0, zb)]
    aux = [(0, 1, 0, 2 * za), (0, 2, 0, 1.7), (0, 2, 1, 1.9), (1, 1, 0, 2 * zb), (1, 2, 1, 1.3)]
    job = synth.Job("ri_pin", atoms, basis, aux, [COULOMB], oracle.J2 | oracle.J3)
    ctx = P.Context(0)
    J = P.Job.from_synth(ctx, job, P.FP64)
    out = J.compute(oracle.J2 | oracle.J3)
    torch.cuda.synchronize()
    _, _, eri, info = _gpu_ri(P, out["J2"].cpu().numpy(), out["J3"].cpu().numpy())
    assert info == 0
    c = lambda z: z ** 1.5 / math.sqrt(8 * math.pi)
    ref = c(za) * c(zb) * 0.5 * (cf.coulomb_2c(R, 2 * za, 2 * zb) + cf.coulomb_2c(R, 2 * zb, 2 * za))
    assert abs(eri[0, 0] - 5 * za / 8) < 1e-11
    assert abs(eri[3, 3] - 5 * zb / 8) < 1e-11
    assert abs(eri[0, 3] - ref) < 1e-11


def test_triatomic_eri_parity(P):
    """Triatomic J2 / J3 from the FP64 library path; eq 14 on the GPU against the oracle's
    solve on the same matrices, within a few kappa(J2) * 2^-52 of the largest element."""
    import torch
    job = synth.triatomic_oh2(0)
    ctx = P.Context(0)
    J = P.Job.from_synth(ctx, job, P.FP64)
    out = J.compute(oracle.J2 | oracle.J3)
    torch.cuda.synchronize()
    J2, J3 = out["J2"].cpu().numpy(), out["J3"].cpu().numpy()
    _, _, eri, info = _gpu_ri(P, J2, J3)
    assert info == 0
    ref = ri_oracle.ri_eri(J2, J3)
    kappa = np.linalg.cond(J2)
    err = np.abs(eri - ref).max() / np.abs(ref).max()
    assert err <= 50 * kappa * EPS, (err, kappa)
    nb = job.n_bf
    e4 = eri.reshape(nb, nb, nb, nb)
    assert np.abs(e4 - e4.transpose(2, 3, 0, 1)).max() <= 50 * kappa * EPS * np.abs(eri).max()


def window_bound(Ba, Bb):
    """sum over 128-row aux windows of (rows in the window) x (window max |a|) x (window max |b|)
    per element: the scale the digits resolve to about 2^-38 (each value keeps 39 bits relative
    to its window's largest: five 8-bit digits of its double-float split)."""
    out = 0.0
    for w0 in range(0, Ba.shape[0], 128):
        ma = np.abs(Ba[w0:w0 + 128]).max(axis=0)
        mb = np.abs(Bb[w0:w0 + 128]).max(axis=0)
        out = out + min(128, Ba.shape[0] - w0) * np.outer(ma, mb)
    return out


@pytest.mark.parametrize("n,m,blk", [(1, 9, (0, 9, 0, 9)), (37, 150, (17, 70, 90, 60)), (82, 676, (0, 676, 0, 676)),
                                     (200, 3000, (100, 1300, 500, 700))])
def test_eri_mixed_within_stated_error(P, n, m, blk):
    """Tensor-core (ij|kl) against the FP64 product: within 2e-9 of the window bound (a loose
    bound, kept from a four-digit version; five digits give about 2^-38); ragged aux counts,
    pair ranges and blocks, aux rows of scales e^-3..e^3."""
    import torch
    rng = np.random.default_rng(n + m)
    B = rng.standard_normal((n, m)) * np.exp(rng.uniform(-3, 3, (n, 1)))
    c0, nc, d0, nd = blk
    ref = B[:, c0:c0 + nc].T @ B[:, d0:d0 + nd]
    got = P.ri_eri_mixed(torch.tensor(B, device="cuda"), c0, nc, d0, nd)
    torch.cuda.synchronize()
    err = np.abs(got.cpu().numpy() - ref) / window_bound(B[:, c0:c0 + nc], B[:, d0:d0 + nd])
    assert err.max() < 2e-9, err.max()


def test_eri_mixed_on_the_triatomic_assembly(P):
    """The RI product of the triatomic job's FP64 (P|Q), (P|ij) on the tensor cores against the
    FP64 kernel: within 2e-9 of the window bound."""
    import torch
    job = synth.triatomic_oh2(0)
    J = P.Job.from_synth(P.Context(0), job, P.FP64)
    out = J.compute(oracle.J2 | oracle.J3)
    n = out["J2"].shape[0]
    L, info = P.ri_factor(out["J2"])
    B = P.ri_solve(L, out["J3"].reshape(n, -1).clone())
    m = B.shape[1]
    e64 = P.ri_eri(B, 0, m, 0, m)
    emx = P.ri_eri_mixed(B, 0, m, 0, m)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    Bh = B.cpu().numpy()
    err = np.abs(emx.cpu().numpy() - e64.cpu().numpy()) / window_bound(Bh, Bh)
    assert err.max() < 2e-9, err.max()
