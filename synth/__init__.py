"""Seeded synthetic inputs: molecules, STO basis shells, RI auxiliary shells, PS grid specs.

This module draws random numbers and lays out shells; it holds none of the quadrature's
arithmetic (no grids, no function values, no integrals).  Both the CPU oracle and the CUDA
path take their inputs from here, nothing else is shared between them.

Units are atomic units (bohr).  Shell tuples are ``(atom, n, l, zeta)`` with ``n = l + 1``
except where a workload names 2s shells explicitly.  Function order everywhere is: atom
order, then shell order as listed, then ``m = -l..l``.

Workloads (the shapes follow the paper's molecules and basis sets, Table S1/S2, and the
even-tempered / combinatorial auxiliary recipe of Section 3):

* ``h2_fp64``            two H 1.4 bohr apart, 1s2s2p basis, 1s2s2p3d aux, grid 15/10/6 Q4
* ``triatomic_oh2``      bent OH2, O 3s2p1d / H 3s1p basis, O 5s4p3d2f / H 4s3p1d aux,
                         grid 20/15/8 Q4 N_SP 3
* ``c3h6``               propanediyl-shaped C3H6, QZ-sized basis (C 4s3p2d1f, H 4s3p2d),
                         aux C 6s5p4d3f3g / H 6s5p4d3f1g, per-pair grids N_mu 15..30,
                         N_nu 10..20, N_phi 8
* ``fivez_diatomic`` / ``fivez_triatomic``  5s4p3d2f1g basis, 8s7p6d5f4g3h aux,
                         grid 30/25/16 with Q = (5,4,4)
* ``serving_stream``     Poisson-arriving random molecules of 2..9 atoms
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

S, T, V, J2, J3 = 1, 2, 4, 8, 16
ALL = S | T | V | J2 | J3
CLASS_NAMES = {S: "S", T: "T", V: "V", J2: "J2", J3: "J3"}


@dataclass
class Job:
    """One integral job: geometry, basis, aux basis, grid specs, class mask."""

    name: str
    atoms: list  # [(Z, (x, y, z))] in bohr
    basis: list  # [(atom, n, l, zeta)]
    aux: list  # [(atom, n, l, zeta)]
    specs: list  # [(n_mu, n_nu, n_phi, q_mu, q_nu, q_phi, n_sp)]: one, or one per pair A<B
    mask: int = ALL
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return len(self.atoms)

    @property
    def n_bf(self) -> int:
        return sum(2 * l + 1 for (_, _, l, _) in self.basis)

    @property
    def n_aux(self) -> int:
        return sum(2 * l + 1 for (_, _, l, _) in self.aux)

    def spec_for_pair(self, a: int, b: int):
        """Grid spec of pair (a, b), a < b; pairs are enumerated (0,1),(0,2),..,(1,2),.."""
        if len(self.specs) == 1:
            return self.specs[0]
        if a > b:
            a, b = b, a
        n = self.n_atoms
        idx = a * n - a * (a + 1) // 2 + (b - a - 1)
        return self.specs[idx]


def _log_uniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
        ]
    )


def _shells_from_pattern(atom, pattern, rng, lo, hi):
    """pattern: counts per l, e.g. (3, 2, 1) = 3s2p1d with n = l + 1, exponents log-uniform."""
    out = []
    for l, count in enumerate(pattern):
        for z in sorted(_log_uniform(rng, lo, hi, count), reverse=True):
            out.append((atom, l + 1, l, float(z)))
    return out


def combinatorial_aux(atom, basis_shells, counts):
    """Auxiliary shells of one atom, built the way Section 3 of the paper describes.

    For each aux angular momentum L the basis pairs (f, g) on the atom with l_f + l_g = L
    give summed exponents zeta_f + zeta_g; their min and max bound an even-tempered
    sequence of ``counts[L]`` exponents.  Every aux shell has n = L + 1.
    """
    mine = [(l, z) for (a, _, l, z) in basis_shells if a == atom]
    out = []
    for L, k in enumerate(counts):
        if k == 0:
            continue
        sums = [z1 + z2 for i, (l1, z1) in enumerate(mine) for (l2, z2) in mine[i:] if l1 + l2 == L]
        if not sums:  # no pair reaches L: span the whole summed range instead
            sums = [z1 + z2 for i, (_, z1) in enumerate(mine) for (_, z2) in mine[i:]]
        zmin, zmax = min(sums), max(sums)
        if k == 1:
            zs = [math.sqrt(zmin * zmax)]
        else:
            if zmax <= zmin * (1 + 1e-12):  # a single summed exponent: widen it
                zmin, zmax = zmin / 1.5, zmax * 1.5
            zs = list(np.geomspace(zmax, zmin, k))
        for z in zs:
            out.append((atom, L + 1, L, float(z)))
    return out


# ----------------------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------------------

def h2_fp64(seed: int = 0, spec=(15, 10, 6, 4, 4, 4, 3), mask: int = S | T | V | J2) -> Job:
    """Two H atoms 1.4 bohr apart on z; per atom 1s, 2s, 2p (xi ~ logU[0.5,3]) and aux
    1s, 2s, 2p, 3d (xi ~ logU[0.8,6]); grid n = (60, 40, 24) points = N (15,10,6) x Q 4."""
    rng = np.random.default_rng(seed)
    atoms = [(1, (0.0, 0.0, 0.0)), (1, (0.0, 0.0, 1.4))]
    basis, aux = [], []
    for a in range(2):
        z = _log_uniform(rng, 0.5, 3.0, 3)
        basis += [(a, 1, 0, float(z[0])), (a, 2, 0, float(z[1])), (a, 2, 1, float(z[2]))]
        za = _log_uniform(rng, 0.8, 6.0, 4)
        aux += [(a, 1, 0, float(za[0])), (a, 2, 0, float(za[1])), (a, 2, 1, float(za[2])),
                (a, 3, 2, float(za[3]))]
    return Job("h2_fp64", atoms, basis, aux, [tuple(spec)], mask, {"seed": seed})


def _bent_triatomic(rng, Zs, r_lo, r_hi):
    d1, d2 = rng.uniform(r_lo, r_hi, 2)
    ang = math.radians(rng.uniform(95.0, 115.0))
    pos = np.array([[0.0, 0.0, 0.0], [d1, 0.0, 0.0], [d2 * math.cos(ang), d2 * math.sin(ang), 0.0]])
    pos = pos @ _random_rotation(rng).T + rng.normal(scale=0.3, size=3)
    return [(int(Z), tuple(float(c) for c in p)) for Z, p in zip(Zs, pos)]


def triatomic_oh2(seed: int = 0, spec=(20, 15, 8, 4, 4, 4, 3), mask: int = ALL) -> Job:
    """Bent Z=(8,1,1), O-H ~ U[1.6,2.0] bohr, angle ~ U[95,115] deg, random orientation.
    O 3s2p1d, H 3s1p, xi ~ logU[0.3,12]; aux O 5s4p3d2f (46), H 4s3p1d (18)."""
    rng = np.random.default_rng(seed)
    atoms = _bent_triatomic(rng, (8, 1, 1), 1.6, 2.0)
    basis = _shells_from_pattern(0, (3, 2, 1), rng, 0.3, 12.0)
    for a in (1, 2):
        basis += _shells_from_pattern(a, (3, 1), rng, 0.3, 12.0)
    aux = combinatorial_aux(0, basis, (5, 4, 3, 2))
    for a in (1, 2):
        aux += combinatorial_aux(a, basis, (4, 3, 1))
    return Job("triatomic_oh2", atoms, basis, aux, [tuple(spec)], mask, {"seed": seed})


def c3h6(seed: int = 0, mask: int = ALL) -> Job:
    """Propanediyl-shaped C3H6: C-C 2.9 bohr, C-C-C 110 deg, C-H 2.05 bohr.
    C 4s3p2d1f (30), H 4s3p2d (23), xi ~ logU[0.2,15]; aux C 6s5p4d3f3g (89),
    H 6s5p4d3f1g (71); per-pair grids N_mu ~ U{15..30}, N_nu ~ U{10..20}, N_phi = 8."""
    rng = np.random.default_rng(seed)
    half = math.radians(110.0) / 2
    c2 = np.zeros(3)
    c1 = 2.9 * np.array([math.sin(half), 0.0, math.cos(half)])
    c3 = 2.9 * np.array([-math.sin(half), 0.0, math.cos(half)])
    ey = np.array([0.0, 1.0, 0.0])
    hs = []
    alpha = math.radians(58.0)
    for c, nbr in ((c1, [c2]), (c2, [c1, c3]), (c3, [c2])):
        out = sum((c - n) / np.linalg.norm(c - n) for n in nbr)
        out = out / np.linalg.norm(out)
        for s in (+1, -1):
            hs.append(c + 2.05 * (math.cos(alpha) * out + s * math.sin(alpha) * ey))
    pos = np.array([c1, c2, c3] + hs)
    Zs = [6, 6, 6] + [1] * 6
    atoms = [(Z, tuple(float(x) for x in p)) for Z, p in zip(Zs, pos)]
    basis = []
    for a, Z in enumerate(Zs):
        basis += _shells_from_pattern(a, (4, 3, 2, 1) if Z == 6 else (4, 3, 2), rng, 0.2, 15.0)
    aux = []
    for a, Z in enumerate(Zs):
        aux += combinatorial_aux(a, basis, (6, 5, 4, 3, 3) if Z == 6 else (6, 5, 4, 3, 1))
    n = len(atoms)
    specs = []
    for i in range(n):
        for j in range(i + 1, n):
            specs.append((int(rng.integers(15, 31)), int(rng.integers(10, 21)), 8, 4, 4, 4, 3))
    _check_min_distance(atoms, 1.8)
    return Job("c3h6", atoms, basis, aux, specs, mask, {"seed": seed})


def _fivez(seed, n_atoms, mask):
    rng = np.random.default_rng(seed)
    Zs = [int(z) for z in rng.choice([6, 7, 8], n_atoms)]
    if n_atoms == 2:
        d = rng.uniform(2.0, 2.6)
        pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, d]]) @ _random_rotation(rng).T
        atoms = [(Z, tuple(float(c) for c in p)) for Z, p in zip(Zs, pos)]
    else:
        atoms = _bent_triatomic(rng, Zs, 2.0, 2.6)
    basis, aux = [], []
    for a in range(n_atoms):
        basis += _shells_from_pattern(a, (5, 4, 3, 2, 1), rng, 0.15, 20.0)
    for a in range(n_atoms):
        aux += combinatorial_aux(a, basis, (8, 7, 6, 5, 4, 3))
    return atoms, basis, aux


def fivez_diatomic(seed: int = 0, spec=(30, 25, 16, 5, 4, 4, 3), mask: int = ALL) -> Job:
    atoms, basis, aux = _fivez(seed, 2, mask)
    return Job("fivez_diatomic", atoms, basis, aux, [tuple(spec)], mask, {"seed": seed})


def fivez_triatomic(seed: int = 0, spec=(30, 25, 16, 5, 4, 4, 3), mask: int = ALL) -> Job:
    atoms, basis, aux = _fivez(seed, 3, mask)
    return Job("fivez_triatomic", atoms, basis, aux, [tuple(spec)], mask, {"seed": seed})


def paper_job(molecule: str, spec=(26, 20, 8, 4, 4, 4, 3), mask: int = ALL, basis: str = "TZ") -> Job:
    """A molecule of the paper's Table S2 in one of its Slater bases (Table S1: "TZ", "QZ",
    "5Z"), aux by the combinatorial recipe of Section 3 with the per-l counts of
    ``paper_tables.AUX_COUNTS`` (TZ) / ``AUX_COUNTS_HIGH`` (QZ, 5Z), a reading: the paper does
    not print them.  Default grid: the smallest of Table S3 (26 / 20 / 8, Q 4, N_SP 3)."""
    from . import paper_tables as pt
    atoms = pt.atoms_of(molecule)
    shells = pt.basis_of(molecule, basis)
    counts = pt.AUX_COUNTS if basis == "TZ" else pt.AUX_COUNTS_HIGH
    aux = []
    for a, (e, _) in enumerate(pt.GEOMETRIES[molecule]):
        aux += combinatorial_aux(a, shells, counts[e])
    name = molecule.lower() + "_" + basis.lower()
    return Job(name, atoms, shells, aux, [tuple(spec)], mask, {"molecule": molecule, "basis": basis})


def clf_tz(seed: int = 0, spec=(26, 20, 8, 4, 4, 4, 3), mask: int = ALL) -> Job:
    """ClF in the paper's TZ basis, Table S2 geometry (Figs. 3-4); seed unused."""
    return paper_job("ClF", spec, mask)


def of2_tz(seed: int = 0, spec=(26, 20, 8, 4, 4, 4, 3), mask: int = ALL) -> Job:
    """OF2 in the paper's TZ basis, Table S2 geometry (Figs. 3-5); seed unused."""
    return paper_job("OF2", spec, mask)


SCAN_PAIRS = ((0, 0), (1, 1), (2, 2), (1, 3), (3, 3), (3, 5))


def scan_directions(k: int = 16):
    """k unit vectors spread over the sphere (Fibonacci lattice): the displacement directions
    of the Fig. 6 scans (the paper's 16 directions are not listed)."""
    g = math.pi * (3.0 - math.sqrt(5.0))
    out = []
    for i in range(k):
        z = 1.0 - (2 * i + 1) / k
        r = math.sqrt(1.0 - z * z)
        out.append((r * math.cos(g * i), r * math.sin(g * i), z))
    return out


def displacement_scan(pairs=SCAN_PAIRS, directions=None, distances=None, spec=(80, 70, 50, 4, 4, 4, 3),
                      mask: int = J2):
    """The Fig. 6 workload: one aux function of angular momentum l1 (zeta = 1, n = l1 + 1) at
    the origin, one of l2 at R d for each direction d and distance R (1.0 to 6.0 bohr in steps
    of 0.1), on the paper's large PS grid (80 / 70 / 50, Q 4); (P|Q) of their m = 0 components
    along each path.  Below about 1 bohr the truncated spheroid of eq 17 (mu_max = C1
    atanh(N/(N+1)), C1 = 2.3 a^(1/4)) no longer holds zeta = 1 functions.  Each point is its
    own diatomic job (a 1s basis function, zeta = 1, on each centre).  Returns [(meta, Job)],
    meta = (l1, l2, direction index, R, row of P, column of Q in (P|Q))."""
    directions = scan_directions() if directions is None else directions
    distances = [round(1.0 + 0.1 * i, 10) for i in range(51)] if distances is None else distances
    out = []
    for (l1, l2) in pairs:
        for di, d in enumerate(directions):
            for R in distances:
                atoms = [(1, (0.0, 0.0, 0.0)), (1, (R * d[0], R * d[1], R * d[2]))]
                basis = [(0, 1, 0, 1.0), (1, 1, 0, 1.0)]
                aux = [(0, l1 + 1, l1, 1.0), (1, l2 + 1, l2, 1.0)]
                job = Job("scan", atoms, basis, aux, [tuple(spec)], mask, {"R": R, "dir": di})
                out.append(((l1, l2, di, R, l1, 2 * l1 + 1 + l2), job))
    return out


def _check_min_distance(atoms, dmin):
    p = np.array([a[1] for a in atoms])
    for i in range(len(p)):
        for j in range(i + 1, len(p)):
            if np.linalg.norm(p[i] - p[j]) < dmin:
                raise ValueError("atoms %d,%d closer than %.2f bohr" % (i, j, dmin))


# Basis patterns per element for the serving mix: (basis counts per l, aux counts per l, xi range)
_PATTERNS = {
    "DZ": {"heavy": ((2, 1), (1, 1, 1, 1)), "H": ((2, 1), (1, 1, 1, 1)), "xi": (0.5, 3.0)},
    "TZ": {"heavy": ((3, 2, 1), (5, 4, 3, 2)), "H": ((3, 1), (4, 3, 1)), "xi": (0.3, 12.0)},
    "QZ": {"heavy": ((4, 3, 2, 1), (6, 5, 4, 3, 3)), "H": ((4, 3, 2), (6, 5, 4, 3, 1)),
           "xi": (0.2, 15.0)},
}


def random_molecule(rng, name="serve", spec=(20, 15, 8, 4, 4, 4, 3), mask=ALL,
                    n_bf_range=(8, 300), max_tries=1000) -> Job:
    """Random molecule of 2..9 atoms with Z in {1,6,7,8}; atoms are placed one by one
    1.8..3.0 bohr from a random earlier atom, rejecting any pair closer than 1.8 bohr and
    any nearly collinear triple; basis pattern DZ/TZ/QZ, kept if 8 <= n_bf <= 300."""
    for _ in range(max_tries):
        n = int(rng.integers(2, 10))
        Zs = [int(z) for z in rng.choice([1, 6, 7, 8], n)]
        pos = [np.zeros(3)]
        ok = True
        while len(pos) < n and ok:
            for _try in range(200):
                base = pos[int(rng.integers(0, len(pos)))]
                d = rng.normal(size=3)
                d /= np.linalg.norm(d)
                cand = base + rng.uniform(1.8, 3.0) * d
                if min(np.linalg.norm(cand - p) for p in pos) < 1.8:
                    continue
                if _nearly_collinear(pos + [cand]):
                    continue
                pos.append(cand)
                break
            else:
                ok = False
        if not ok:
            continue
        pat = _PATTERNS[["DZ", "TZ", "QZ"][int(rng.integers(0, 3))]]
        lo, hi = pat["xi"]
        basis = []
        for a, Z in enumerate(Zs):
            basis += _shells_from_pattern(a, pat["H" if Z == 1 else "heavy"][0], rng, lo, hi)
        job_nbf = sum(2 * l + 1 for (_, _, l, _) in basis)
        if not (n_bf_range[0] <= job_nbf <= n_bf_range[1]):
            continue
        aux = []
        for a, Z in enumerate(Zs):
            aux += combinatorial_aux(a, basis, pat["H" if Z == 1 else "heavy"][1])
        atoms = [(Z, tuple(float(c) for c in p)) for Z, p in zip(Zs, pos)]
        return Job(name, atoms, basis, aux, [tuple(spec)], mask, {})
    raise RuntimeError("could not draw a molecule")


def _nearly_collinear(pos, tol=1e-3):
    """True if some atom lies within sin(angle) < tol of the axis through two others."""
    p = np.array(pos)
    n = len(p)
    for i in range(n):
        for j in range(i + 1, n):
            ax = p[j] - p[i]
            ax = ax / np.linalg.norm(ax)
            for k in range(n):
                if k in (i, j):
                    continue
                v = p[k] - 0.5 * (p[i] + p[j])
                perp = v - np.dot(v, ax) * ax
                if np.linalg.norm(perp) < tol * np.linalg.norm(v):
                    return True
    return False


def serving_stream(seed: int = 0, rate: float = 100.0, n_jobs: int = 100, **kw):
    """Poisson arrivals: returns [(t_arrival_seconds, Job)] with exponential gaps of mean 1/rate."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_jobs):
        t += float(rng.exponential(1.0 / rate))
        out.append((t, random_molecule(rng, name="serve%d" % i, **kw)))
    return out


def sub_molecule(job: Job, keep, name: str = None) -> Job:
    """The sub-molecule of the atoms `keep` (in the given order): their shells and the grid
    specs of their pairs, renumbered; the same classes."""
    keep = list(keep)
    idx = {a: i for i, a in enumerate(keep)}
    atoms = [job.atoms[a] for a in keep]
    basis = [(idx[s[0]],) + tuple(s[1:]) for s in job.basis if s[0] in idx]
    aux = [(idx[s[0]],) + tuple(s[1:]) for s in job.aux if s[0] in idx]
    basis.sort(key=lambda s: s[0])
    aux.sort(key=lambda s: s[0])
    specs = [job.spec_for_pair(keep[i], keep[j]) for i in range(len(keep)) for j in range(i + 1, len(keep))]
    return Job(name or "%s_atoms%s" % (job.name, "".join(str(a) for a in keep)), atoms, basis, aux, specs, job.mask)


WORKLOADS = {
    "h2_fp64": h2_fp64,
    "triatomic_oh2": triatomic_oh2,
    "c3h6": c3h6,
    "fivez_diatomic": fivez_diatomic,
    "fivez_triatomic": fivez_triatomic,
    "clf_tz": clf_tz,
    "of2_tz": of2_tz,
}
