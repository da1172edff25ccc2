"""Pins of the oracle's one-centre overlap and kinetic closed forms (the reading under which
Table 1's kinetic RMSE for SO2 is reproduced): symbolic radial integrals (sympy, the
Laplacian differentiated by sympy rather than written out), normalisation, the textbook
1s kinetic energy zeta^2 / 2, and the same elements integrated numerically on a fine PS grid."""
import math

import numpy as np
import pytest

import oracle
from oracle import psq_oracle as O

SHELLS = [(0, 1, 0, 1.3), (0, 2, 0, 0.8), (0, 2, 0, 2.1), (0, 2, 1, 1.1), (0, 3, 1, 0.7), (0, 3, 2, 2.0),
          (0, 4, 3, 1.6)]


def _fns(shells):
    return [(n, l, m, z) for (_, n, l, z) in shells for m in range(-l, l + 1)]


def test_symbolic_radial_integrals():
    sp = pytest.importorskip("sympy")
    r = sp.symbols("r", positive=True)
    S, T = O.one_centre_st(SHELLS)
    fns = _fns(SHELLS)
    for a, (na, la, ma, za) in enumerate(fns):
        for b, (nb, lb, mb, zb) in enumerate(fns):
            if la != lb or ma != mb:
                assert S[a, b] == 0.0 and T[a, b] == 0.0
                continue
            if b < a:
                continue
            za_, zb_ = sp.nsimplify(za), sp.nsimplify(zb)
            Na = (2 * za_) ** (na + sp.Rational(1, 2)) / sp.sqrt(sp.factorial(2 * na))
            Nb = (2 * zb_) ** (nb + sp.Rational(1, 2)) / sp.sqrt(sp.factorial(2 * nb))
            Ra = Na * r ** (na - 1) * sp.exp(-za_ * r)
            Rb = Nb * r ** (nb - 1) * sp.exp(-zb_ * r)
            lap_b = sp.diff(r ** 2 * sp.diff(Rb, r), r) / r ** 2 - lb * (lb + 1) * Rb / r ** 2
            s_ex = float(sp.integrate(Ra * Rb * r ** 2, (r, 0, sp.oo)))
            t_ex = float(sp.integrate(-sp.Rational(1, 2) * Ra * lap_b * r ** 2, (r, 0, sp.oo)))
            assert abs(S[a, b] - s_ex) <= 1e-13 * max(1.0, abs(s_ex)), (a, b)
            assert abs(T[a, b] - t_ex) <= 1e-12 * max(1.0, abs(t_ex)), (a, b)


def test_normalisation_and_1s_kinetic():
    S, T = O.one_centre_st(SHELLS)
    assert np.allclose(np.diag(S), 1.0, atol=1e-14, rtol=0)
    assert abs(T[0, 0] - 1.3 ** 2 / 2) < 1e-14
    assert np.allclose(S, S.T) and np.allclose(T, T.T)


def test_matches_pair_grid_quadrature():
    """The same block integrated on a fine PS pair grid of the atom and a neighbour 2.5 bohr
    away (eq 9 with the Laplacian form of the kinetic operand)."""
    atoms = [(8, (0.0, 0.0, 0.0)), (1, (0.0, 0.0, 2.5))]
    g = O.build_grid(atoms, (40, 40, 12, 6, 6, 4, 1), 0, 1)
    F, L = O.sto_values(SHELLS, g["rA"], g["dA"], with_laplacian=True)
    Sq = (F * g["w"]) @ F.T
    Tq = -0.25 * ((F * g["w"]) @ L.T + (L * g["w"]) @ F.T)
    S, T = O.one_centre_st(SHELLS)
    assert np.abs(Sq - S).max() < 1e-9, np.abs(Sq - S).max()
    assert np.abs(Tq - T).max() < 1e-7 * max(1.0, np.abs(T).max()), np.abs(Tq - T).max()


def test_compute_uses_the_closed_forms_for_one_centre_blocks():
    import synth
    job = synth.triatomic_oh2(0)
    job.specs = [(8, 6, 4, 4, 4, 4, 1)]
    out = oracle.compute(job, mask=oracle.S | oracle.T)
    start = 0
    for X in range(job.n_atoms):
        sh = [s for s in job.basis if s[0] == X]
        n = sum(2 * s[2] + 1 for s in sh)
        S, T = O.one_centre_st(sh)
        assert np.array_equal(out["S"][start:start + n, start:start + n], S)
        assert np.array_equal(out["T"][start:start + n, start:start + n], T)
        assert np.array_equal(out["absS"][start:start + n, start:start + n], np.abs(S))
        start += n
