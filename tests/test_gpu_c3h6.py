"""The propanediyl-shaped C3H6 workload at full size (9 atoms, 228 basis / 693 aux functions,
36 pair grids with N_mu 15..30 and N_nu 10..20, 252 refined grids, 55.8 M points): every
class on the GPU, compared with the oracle on sampled blocks it can compute one by one
(one-, two- and three-centre S/T/V, (P|Q) and (P|ij) blocks, C-C, C-H and H-H).
FP64 path: 1e-12 of each element's absolute-term sum C.  Mixed path: 1e-9 absolute (its
target), relative errors printed."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

PAIRS = [(0, 0), (0, 1), (0, 3), (1, 5), (3, 4), (4, 8)]
AUX_PAIRS = [(0, 1), (2, 7), (5, 5)]
TRIPLES = [(0, 0, 0), (1, 0, 1), (3, 0, 1), (0, 3, 4), (6, 1, 5), (8, 2, 8)]


@pytest.fixture(scope="module")
def ref():
    job = synth.c3h6(0)
    return job, oracle.compute(job, mask=oracle.ALL, j3_triples=TRIPLES, pairs=PAIRS, aux_pairs=AUX_PAIRS)


def _fn_slices(shells, nat):
    out, off = [], 0
    for X in range(nat):
        n = sum(2 * s[2] + 1 for s in shells if s[0] == X)
        out.append(slice(off, off + n))
        off += n
    return out


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-9)])
def test_c3h6_sampled_blocks(ref, precision, tol):
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
    bs = _fn_slices(job.basis, job.n_atoms)
    ax = _fn_slices(job.aux, job.n_atoms)
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
    print("\nc3h6 precision %d worst rel / abs:" % precision,
          {k: "%.2e / %.2e" % (worst[k], absw[k]) for k in worst})
    for k in worst:
        # FP64: relative to C; mixed: absolute
        assert (worst[k] if precision == 0 else absw[k]) <= tol, (k, worst[k], absw[k])
