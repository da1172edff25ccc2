"""The paper's own basis sets and geometries, as inputs for paper-shaped workloads.

Transcribed from the supporting information of Stark et al., arXiv 2510.15204:

* ``TZ``: Table S1, TZ column (Slater exponents; every s shell is 1s, p shell 2p, d shell
  3d, f shell 4f, i.e. n = l + 1).  Elements H, C, N, O, F, Si, S, Cl.
* ``GEOMETRIES``: Table S2, in Angstrom, converted to bohr by ``bohr()``.  The table's page
  break before SO2 drops its first atom label and shifts the others down one row: the rows are
  read as S, O, O (both S-O distances are then 1.429 Angstrom).

This module holds input data only (no quadrature arithmetic).  The auxiliary exponents are
not printed; ``paper_job`` builds them with the combinatorial recipe of Section 3
(``combinatorial_aux``) and the per-l counts below, a reading of this repository.
"""
from __future__ import annotations

ANGSTROM = 1.0 / 0.529177210903  # bohr per Angstrom (CODATA 2018)

Z = {"H": 1, "C": 6, "N": 7, "O": 8, "F": 9, "Si": 14, "S": 16, "Cl": 17}

# Table S1, TZ: {element: {l: [exponents]}}
TZ = {
    "H": {0: [2.280, 1.520, 1.013], 1: [2.100, 1.500]},
    "C": {0: [8.689, 5.323, 3.261, 1.998, 1.224, 0.750], 1: [4.000, 2.051, 1.052], 2: [3.400, 1.900]},
    "N": {0: [10.820, 6.345, 3.720, 2.181, 1.279, 0.750], 1: [4.400, 2.588, 1.522], 2: [4.000, 2.000]},
    "O": {0: [13.351, 7.506, 4.220, 2.373, 1.334, 0.750], 1: [5.700, 2.850, 1.425], 2: [4.000, 2.000]},
    "F": {0: [15.520, 8.466, 4.619, 2.520, 1.375, 0.750], 1: [5.667, 3.063, 1.656], 2: [4.000, 2.000]},
    "Si": {0: [19.317, 12.870, 8.575, 5.713, 3.806, 2.536, 1.690, 1.126, 0.750],
           1: [11.333, 6.869, 4.163, 2.523, 1.529, 0.927], 2: [3.400, 2.000]},
    "S": {0: [23.379, 15.209, 9.894, 6.437, 4.187, 2.724, 1.772, 1.153, 0.750],
          1: [12.800, 8.000, 5.000, 3.125, 1.953, 1.221], 2: [3.700, 2.000]},
    "Cl": {0: [21.825, 15.156, 10.525, 7.309, 5.076, 3.525, 2.448, 1.700, 1.180],
           1: [22.000, 12.571, 7.184, 4.105, 2.346, 1.340], 2: [3.7, 2.0]},
}

# Table S2 (Angstrom): {molecule: [(element, (x, y, z))]}
GEOMETRIES = {
    "HF": [("H", (0.0, 0.0, 0.0)), ("F", (0.0, 0.0, 0.9170))],
    "CO": [("C", (0.0, 0.0, 0.0)), ("O", (0.0, 0.0, 1.128))],
    "N2": [("N", (0.0, 0.0, 0.0)), ("N", (0.0, 0.0, 1.098))],
    "ClF": [("Cl", (0.0, 0.0, 1.628)), ("F", (0.0, 0.0, 0.0))],
    "H2O": [("H", (0.03662, 0.2867, -0.7420)), ("H", (0.006501, 1.1120, 0.5315)),
            ("O", (-0.003118, 0.2113, 0.2105))],
    "OF2": [("O", (-0.01081, 0.06083, 0.3100)), ("F", (0.004032, 1.367, 0.7531)),
            ("F", (0.04678, 0.1819, -1.063))],
    "OF2_long": [("O", (0.0, 0.0, 0.0)), ("F", (0.0, 0.0, 1.380)), ("F", (0.0, 40.23, -9.810))],
    "SO2": [("S", (-0.01091, -0.06565, 0.2156)), ("O", (0.001496, 1.134, 0.9929)),
            ("O", (0.04941, 0.04196, -1.208))],
}

# Aux counts per L (a reading: Section 3 fixes the recipe, not the counts).  About three aux
# functions per basis function, up to L = 4 (g) for atoms with d shells ("the auxiliary basis
# contains up to g functions", Section 4), L = 2 for H.
AUX_COUNTS = {"H": (4, 3, 2), "C": (7, 6, 4, 3, 1), "N": (7, 6, 4, 3, 1), "O": (7, 6, 4, 3, 1),
              "F": (7, 6, 4, 3, 1), "Si": (9, 7, 5, 3, 1), "S": (9, 7, 5, 3, 1), "Cl": (9, 7, 5, 3, 1)}


def bohr(xyz):
    return tuple(float(c) * ANGSTROM for c in xyz)


def atoms_of(molecule):
    """[(Z, (x, y, z) in bohr)] of a Table S2 molecule."""
    return [(Z[e], bohr(p)) for e, p in GEOMETRIES[molecule]]


def basis_of(molecule, table=None):
    """Basis shells [(atom, n, l, zeta)] of a Table S2 molecule from Table S1 (TZ)."""
    table = TZ if table is None else table
    shells = []
    for a, (e, _) in enumerate(GEOMETRIES[molecule]):
        for l in sorted(table[e]):
            for z in table[e][l]:
                shells.append((a, l + 1, l, float(z)))
    return shells
