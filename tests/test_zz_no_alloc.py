"""psq_compute_noalloc, the entry point for callers that cannot allocate device memory (a host
application whose memory manager owns the GPU, a loop that must not pay cudaMalloc's
synchronisation): it runs on the library's own fixed device scratch array.  Its results must
match psq_compute's on a caller-allocated workspace, on two calls in a row (the scratch keeps
the previous call's contents), for the FP64 path and then for the mixed path on the same
scratch (node tables, packed operands and the status word left over from other calls); after
each call psq_check reads the status word through the scratch.  This file is collected last
on purpose."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the plain FP64 path's parity tolerance


def _rel(a, b, absref):
    scale = np.maximum(np.abs(b), absref)
    return float((np.abs(a - b) / np.where(scale > 0, scale, 1.0)).max())


def test_noalloc_matches_compute_twice():
    import torch
    assert torch.cuda.is_available()
    import paper_2510_15204_gb300 as P
    from paper_2510_15204_gb300 import build
    build.build()
    ctx = P.Context(0)
    job = synth.h2_fp64(1)
    J = P.Job.from_synth(ctx, job, P.FP64)
    mask = oracle.ALL
    need = J.workspace_bytes(mask)  # plans mask; the no-alloc call plans nothing
    assert need <= 64 << 20
    ws, ref_out = J.alloc(mask)
    J.compute(mask, ws, ref_out)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref_out.items()}
    absref = oracle.compute(job, mask=mask)  # only for the element scale of the tolerance
    for call in range(2):
        out = {k: torch.full_like(v, float("nan")) for k, v in ref_out.items()}
        J.compute_noalloc(mask, out)
        J.check(mask, None)  # the status word in the scratch
        torch.cuda.synchronize()
        for k in out:
            got = out[k].cpu().numpy()
            assert np.isfinite(got).all(), (call, k)
            assert _rel(got, ref[k], absref["abs" + k]) <= TOL, (call, k)


def test_noalloc_mixed_on_reused_scratch():
    """The mixed path after the FP64 calls on the same scratch, twice: bit for bit the results of
    psq_compute on a fresh workspace (same plan, same arithmetic)."""
    import torch
    import paper_2510_15204_gb300 as P
    ctx = P.Context(0)
    job = synth.h2_fp64(1)
    job.specs = [(12, 8, 6, 4, 4, 4, 3)]  # 36,864 points: the mixed workspace within the 64 MiB scratch
    J = P.Job.from_synth(ctx, job, P.MIXED)
    mask = oracle.ALL
    assert J.workspace_bytes(mask) <= 64 << 20
    ws, ref_out = J.alloc(mask)
    J.compute(mask, ws, ref_out)
    J.check(mask, ws)
    ref = {k: v.cpu().numpy() for k, v in ref_out.items()}
    for call in range(2):
        out = {k: torch.full_like(v, float("nan")) for k, v in ref_out.items()}
        J.compute_noalloc(mask, out)
        J.check(mask, None)
        for k in out:
            assert np.array_equal(out[k].cpu().numpy(), ref[k]), (call, k)


def test_noalloc_rejects_unplanned_and_oversized():
    import torch
    import paper_2510_15204_gb300 as P
    ctx = P.Context(0)
    J = P.Job.from_synth(ctx, synth.h2_fp64(0), P.FP64)
    out = {k: torch.empty(s, dtype=torch.float64, device="cuda") for k, s in J.out_shapes(oracle.S).items()}
    with pytest.raises(P.PsqError) as e:
        J.compute_noalloc(oracle.S, out)  # never planned
    assert e.value.status == 1
    big = P.Job.from_synth(ctx, synth.triatomic_oh2(0), P.FP64)
    assert big.workspace_bytes(oracle.ALL) > 64 << 20
    out = {k: torch.empty(s, dtype=torch.float64, device="cuda") for k, s in big.out_shapes(oracle.ALL).items()}
    with pytest.raises(P.PsqError) as e:
        big.compute_noalloc(oracle.ALL, out)
    assert e.value.status == 2
