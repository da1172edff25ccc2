"""The paper's own molecules and bases on the GPU path (Table S1 TZ exponents, Table S2
geometries; aux by the combinatorial recipe of Section 3).

* ClF, TZ: FP64 parity with the oracle (1e-12 of each element's absolute-term sum), the mixed
  path within 1e-9 absolute.
* Figs. 3-4: convergence with grid size over Table S3's grids against a larger PS grid
  (RMSE of eq 13): every class falls monotonically; overlap, 2- and 3-centre Coulomb reach
  ~1e-10 on the largest Table S3 grid, kinetic and nuclear attraction (the nuclear cusps)
  ~1e-7.
* Fig. 5: for OF2 at equilibrium N_SP = 2 lowers the electron-nuclear RMSE on a fine grid
  and N_SP > 2 adds little.
Thresholds are the measured values with a margin of about 3-5x.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

CLASSES = ("S", "T", "V", "J2", "J3")
BIT = {"S": 1, "T": 2, "V": 4, "J2": 8, "J3": 16}
REF = (60, 50, 36, 4, 4, 4, 3)
S3 = [(26, 20, 8), (29, 26, 11), (32, 32, 14), (37, 42, 19)]  # rows of Table S3 (left)


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "the CUDA path needs a GPU"
    import paper_2510_15204_gb300 as P
    from paper_2510_15204_gb300 import build
    build.build()
    return P


@pytest.fixture(scope="module")
def ctx(P):
    return P.Context(0)


def run(P, ctx, job, mask, precision):
    import torch
    J = P.Job.from_synth(ctx, job, precision)
    out = J.compute(mask)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    del out, J
    torch.cuda.empty_cache()
    return res


def rmse(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2)))


@pytest.fixture(scope="module")
def clf_oracle():
    job = synth.clf_tz()
    ref = oracle.compute(job, mask=oracle.S | oracle.T | oracle.V | oracle.J2, with_abs=True)
    j3 = oracle.compute(job, mask=oracle.J3, with_abs=True, j3_triples=[(0, 0, 1)])
    ref["J3"], ref["absJ3"] = j3["J3"], j3["absJ3"]
    return job, ref


def _block(job, k, M):
    if k != "J3":
        return M
    na0 = sum(2 * s[2] + 1 for s in job.aux if s[0] == 0)
    nb0 = sum(2 * s[2] + 1 for s in job.basis if s[0] == 0)
    return M[:na0, :nb0, nb0:]


def test_clf_tz_fp64_parity(P, ctx, clf_oracle):
    job, ref = clf_oracle
    got = run(P, ctx, job, oracle.ALL, P.FP64)
    for k in CLASSES:
        g, o, c = (_block(job, k, M) for M in (got[k], ref[k], ref["abs" + k]))
        e = np.abs(g - o) / np.where(np.maximum(np.abs(o), c) > 0, np.maximum(np.abs(o), c), 1.0)
        assert e.max() <= 1e-12, (k, float(e.max()))


def test_clf_tz_mixed_within_1e9(P, ctx, clf_oracle):
    job, ref = clf_oracle
    got = run(P, ctx, job, oracle.ALL, P.MIXED)
    for k in CLASSES:
        g, o = (_block(job, k, M) for M in (got[k], ref[k]))
        assert np.abs(g - o).max() <= 1e-9, (k, float(np.abs(g - o).max()))


@pytest.mark.parametrize("cls", CLASSES)
def test_clf_convergence_with_grid_figs_3_4(P, ctx, cls):
    m = BIT[cls]
    ref = run(P, ctx, synth.clf_tz(spec=REF, mask=m), m, P.FP64)[cls]
    errs = [rmse(run(P, ctx, synth.clf_tz(spec=g + (4, 4, 4, 3), mask=m), m, P.FP64)[cls], ref) for g in S3]
    print("\nClF %s RMSE over the Table S3 rows:" % cls, " ".join("%.1e" % e for e in errs))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    bar = {"S": 3e-10, "J2": 2e-10, "J3": 3e-10, "T": 1e-6, "V": 3e-7}[cls]
    assert errs[-1] < bar, errs


def test_of2_third_centre_split_fig_5(P, ctx):
    ref = run(P, ctx, synth.of2_tz(spec=REF, mask=oracle.V), oracle.V, P.FP64)["V"]
    e = [rmse(run(P, ctx, synth.of2_tz(spec=(37, 42, 19, 4, 4, 4, nsp), mask=oracle.V), oracle.V, P.FP64)["V"], ref)
         for nsp in (1, 2, 3, 4)]
    assert e[1] < 0.6 * e[0], e
    assert max(e[2], e[3]) < 2.0 * e[1], e


def test_so2_tz_smallest_overlap_eigenvalue_on_the_gpu(P, ctx):
    """The one value this path's paper prints for a whole matrix: the smallest eigenvalue of
    SO2's TZ overlap matrix, 1.3e-5 (Section 4), on the PS grid 26/32/14, Q 4 (Table 1's
    BP-sized grid), through the FP64 CUDA path (and the mixed path to its error)."""
    job = synth.paper_job("SO2", spec=(26, 32, 14, 4, 4, 4, 3), mask=oracle.S)
    for prec in (P.FP64, P.MIXED):
        S = run(P, ctx, job, oracle.S, prec)["S"]
        ev = np.linalg.eigvalsh(0.5 * (S + S.T))[0]
        assert float("%.1e" % ev) == 1.3e-5, (prec, ev)


@pytest.mark.parametrize("basis,printed", [("TZ", {"S": 8.0e-12, "T": 9.6e-11, "V": 3.0e-7}),
                                           ("QZ", {"S": 5.4e-12, "T": 3.0e-10, "V": 3.1e-7}),
                                           ("5Z", {"S": 8.9e-12, "T": 2.8e-10, "V": 3.2e-7})])
def test_so2_table1_ps_rmse(P, ctx, basis, printed):
    """Table 1's PS column: RMSE of the 26/32/14 grid against 80/70/50 for SO2, all elements.
    One-centre S and T take their closed forms on both grids (the reading this repository
    takes), under which the kinetic RMSE is the printed one within 15% for TZ, QZ and 5Z; the
    overlap RMSE is below the printed one (7-14x here); V_ne (integrated on grids as before)
    within 3x."""
    lo = run(P, ctx, synth.paper_job("SO2", spec=(26, 32, 14, 4, 4, 4, 3), mask=7, basis=basis), 7, P.FP64)
    hi = run(P, ctx, synth.paper_job("SO2", spec=(80, 70, 50, 4, 4, 4, 3), mask=7, basis=basis), 7, P.FP64)
    job = synth.paper_job("SO2", basis=basis)
    atom = np.repeat([a for (a, _, l, _) in job.basis], [2 * l + 1 for (_, _, l, _) in job.basis])
    two = atom[:, None] != atom[None, :]
    rv = rmse(lo["V"], hi["V"])
    print("\nSO2 %s PS RMSE: V %.2e (printed %.1e)" % (basis, rv, printed["V"]))
    assert printed["V"] / 3 < rv < 3 * printed["V"], rv
    for k in ("S", "T"):
        d = lo[k] - hi[k]
        assert np.abs(d[~two]).max() < 1e-14, k  # one-centre: the same closed forms on both grids
        r = rmse(lo[k], hi[k])
        print("SO2 %s PS RMSE %s: all elements %.2e, two-centre %.2e (printed %.1e)"
              % (basis, k, r, float(np.sqrt(np.mean(d[two] ** 2))), printed[k]))
        if k == "T":
            assert abs(r / printed[k] - 1.0) < 0.15, (k, r)
        else:
            assert r < printed[k], (k, r)