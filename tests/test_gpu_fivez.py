"""The pentuple-zeta stress workload at full size: triatomic of Z in {6,7,8}, 5s4p3d2f1g basis
(55 per atom), 8s7p6d5f4g3h aux (163 per atom), grids 30/25/16 with Q = (5,4,4) (960,000 points
per pair grid, refined grids more).  GPU vs oracle on sampled blocks the oracle computes one
by one: FP64 path to 1e-12 of C, mixed path to 1e-9 absolute (its target)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

PAIRS = [(0, 0), (0, 1), (1, 2)]
AUX_PAIRS = [(0, 2)]
TRIPLES = [(2, 0, 1), (1, 1, 2)]


@pytest.fixture(scope="module")
def ref():
    job = synth.fivez_triatomic(0)
    return job, oracle.compute(job, mask=oracle.ALL, j3_triples=TRIPLES, pairs=PAIRS, aux_pairs=AUX_PAIRS)


def _fn_slices(shells, nat):
    out, off = [], 0
    for X in range(nat):
        n = sum(2 * s[2] + 1 for s in shells if s[0] == X)
        out.append(slice(off, off + n))
        off += n
    return out


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_fivez_sampled_blocks(ref, precision, tol):
    import torch
    import paper_2510_15204_gb300 as P
    from paper_2510_15204_gb300 import build
    build.build()
    job, R = ref
    ctx = P.Context(0)
    J = P.Job.from_synth(ctx, job, precision)
    ws, out = J.alloc(oracle.ALL)
    J.compute(oracle.ALL, ws, out)
    J.check(oracle.ALL, ws)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    for k, v in got.items():  # every element, not only the sampled blocks
        assert np.isfinite(v).all(), (k, int((~np.isfinite(v)).sum()))
    del ws
    torch.cuda.empty_cache()
    bs, ax = _fn_slices(job.basis, job.n_atoms), _fn_slices(job.aux, job.n_atoms)
    worst, absw = {}, {}

    def check(k, idx):
        scale = np.maximum(np.abs(R[k][idx]), R["abs" + k][idx])
        d = np.abs(got[k][idx] - R[k][idx])
        worst[k] = max(worst.get(k, 0.0), float((d / np.where(scale > 0, scale, 1.0)).max()))
        absw[k] = max(absw.get(k, 0.0), float(d.max()))

    for (A, B) in PAIRS:
        for k in ("S", "T", "V"):
            check(k, (bs[A], bs[B]))
    for (C, D) in AUX_PAIRS:
        check("J2", (ax[C], ax[D]))
    for (C, A, B) in TRIPLES:
        check("J3", (ax[C], bs[A], bs[B]))
    print("\nfivez precision %d worst rel / abs:" % precision,
          {k: "%.2e / %.2e" % (worst[k], absw[k]) for k in worst})
    for k in worst:
        # FP64: relative to C; mixed: absolute
        assert (worst[k] if precision == 0 else absw[k]) <= tol, (k, worst[k], absw[k])
