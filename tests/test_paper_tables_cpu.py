"""Pins of the transcribed paper inputs (synth/paper_tables.py): Section 3 says the bases are
even tempered (zeta = alpha beta^n), so each (element, l) list of Table S1 must be geometric;
Table S2's geometries must give the molecules' known bond lengths and angles."""
import math

import numpy as np
import pytest

import synth
from synth import paper_tables as pt


@pytest.mark.parametrize("col", ["TZ", "QZ", "5Z"])
@pytest.mark.parametrize("el", sorted(pt.TZ))
def test_exponents_are_even_tempered(col, el):
    for l, zs in pt.TABLES[col][el].items():
        if len(zs) < 3:
            continue
        r = np.array(zs[:-1]) / np.array(zs[1:])
        assert np.abs(r / r.mean() - 1).max() < 2e-3, (col, el, l, r)


def _dist(mol, i, j):
    p = np.array([a[1] for a in pt.GEOMETRIES[mol]])
    return float(np.linalg.norm(p[i] - p[j]))


def _angle(mol, c, i, j):
    p = np.array([a[1] for a in pt.GEOMETRIES[mol]])
    u, v = p[i] - p[c], p[j] - p[c]
    return math.degrees(math.acos(u @ v / np.linalg.norm(u) / np.linalg.norm(v)))


def test_geometries_match_known_structures():
    assert abs(_dist("ClF", 0, 1) - 1.628) < 1e-9
    assert abs(_dist("OF2", 0, 1) - 1.39) < 0.03 and abs(_dist("OF2", 0, 2) - 1.39) < 0.03  # DFT-optimised
    assert abs(_angle("OF2", 0, 1, 2) - 103.0) < 1.5
    assert abs(_dist("H2O", 2, 0) - 0.96) < 0.01 and abs(_angle("H2O", 2, 0, 1) - 104.5) < 1.5
    assert abs(_dist("SO2", 0, 1) - 1.429) < 2e-3 and abs(_dist("SO2", 0, 2) - 1.429) < 2e-3
    assert abs(_dist("OF2_long", 0, 2) - 41.41) < 0.01  # Figure S1's 41.41 Angstrom bond


def test_paper_jobs_sizes():
    j = synth.clf_tz()
    assert (j.n_atoms, j.n_bf) == (2, 37 + 25)
    assert max(s[2] for s in j.aux) == 4  # aux up to g (Section 4)
    assert abs(j.atoms[0][1][2] - 1.628 * pt.ANGSTROM) < 1e-12
    assert synth.of2_tz().n_bf == 75


def test_qz_5z_sizes():
    """Shell counts per column as Table S1 lists them (e.g. C: QZ 8s4p3d1f, 5Z 9s5p4d2f)."""
    count = lambda col, el: tuple(len(pt.TABLES[col][el].get(l, [])) for l in range(4))
    assert count("QZ", "C") == (8, 4, 3, 1) and count("5Z", "C") == (9, 5, 4, 2)
    assert count("QZ", "Cl") == (12, 8, 3, 1) and count("5Z", "Cl") == (12, 10, 4, 2)
    assert count("QZ", "H") == (4, 3, 1, 0) and count("5Z", "H") == (5, 4, 2, 0)
    j = synth.paper_job("CO", basis="5Z")
    assert j.n_bf == 2 * (9 + 15 + 20 + 14) and max(s[2] for s in j.aux) == 6
