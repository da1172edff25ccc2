"""Plain FP64 CPU oracle of the RI 4-index assembly (Section 3, eq 14).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this module; the library never calls it.

Eq 14 approximates a 4-index Coulomb integral through the 3-index ones and the inverse of
the 2-index metric: (ij|kl) ~ sum_PQ (ij|P) [(PQ)^-1] (Q|kl).  ``ri_eri`` writes exactly
that sum, with a linear solve for (PQ)^-1 (Q|kl); the library factors the metric instead
(Cholesky) and never forms the inverse, so the two routes share no arithmetic.
``cholesky`` and ``forward`` are the textbook factor and triangular solve (numpy/scipy
library primitives), kept for step-by-step parity of the library's intermediate outputs.
Pins (``tests/test_oracle_ri.py``): exact fits of one-centre 1s densities reproduce the
closed-form Coulomb integrals 5 zeta / 8 and the two-centre 1s-1s repulsion; a metric
built as J2 X gives X^T J2 X exactly; symmetry, positive semidefiniteness and the Schwarz
bound of the assembled matrix.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def ri_eri(J2, J3):
    """(ij|kl) of eq 14 for all pairs: J2 (n_aux, n_aux), J3 (n_aux, n_bf, n_bf) ->
    (n_bf^2, n_bf^2), row ij = i * n_bf + j, column kl = k * n_bf + l."""
    J2 = np.asarray(J2, dtype=np.float64)
    X = np.asarray(J3, dtype=np.float64).reshape(J2.shape[0], -1)
    return X.T @ np.linalg.solve(J2, X)


def cholesky(J2):
    """Lower-triangular L with L L^T = J2."""
    return np.linalg.cholesky(np.asarray(J2, dtype=np.float64))


def forward(L, X):
    """L^-1 X for lower-triangular L."""
    return scipy.linalg.solve_triangular(L, np.asarray(X, dtype=np.float64), lower=True)
