"""psq_job_autotune: the candidate work splits give the same matrices (up to the order of the
range sums), the chosen plan is the one later computes and graph replays use."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _run(J, mask, ws, out):
    import torch
    J.compute(mask, ws, out)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().copy() for k, v in out.items()}


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_keeps_results_and_plan(precision):
    import torch
    import paper_2510_15204_gb300 as P
    from paper_2510_15204_gb300 import build
    build.build()
    ctx = P.Context(0)
    job = synth.triatomic_oh2(0)
    mask = oracle.ALL
    J = P.Job.from_synth(ctx, job, precision)
    need = J.workspace_bytes(mask)
    # room for every candidate's partial sums
    ws = torch.empty(4 * need + (64 << 20), dtype=torch.uint8, device="cuda")
    out = {k: torch.empty(s, dtype=torch.float64, device="cuda") for k, s in J.out_shapes(mask).items()}
    before = _run(J, mask, ws, out)
    split, ms = J.autotune(mask, ws, out)
    assert split in ((2, 4, 6, 8, 16, 32) if precision == 1 else (2, 4, 8, 16))
    assert ms > 0
    assert J.workspace_bytes(mask) <= ws.numel()
    after = _run(J, mask, ws, out)
    # another split sums the same points in other ranges: FP64 partials agree to rounding;
    # the mixed path's double-float window folds agree to its error (1e-9 absolute)
    tol = 1e-12 if precision == 0 else 1e-9
    for k in before:
        scale = np.abs(before[k]).max() if precision == 0 else 1.0  # mixed: absolute
        np.testing.assert_allclose(after[k], before[k], rtol=0, atol=tol * scale, err_msg=k)
    # a graph captured after tuning replays the tuned plan
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        J.compute_graph(mask, ws, out, stream)
        J.compute_graph(mask, ws, out, stream)
    torch.cuda.synchronize()
    for k in after:
        assert np.array_equal(out[k].cpu().numpy(), after[k]), k


def test_autotune_refuses_a_workspace_no_candidate_fits():
    import torch
    import paper_2510_15204_gb300 as P
    ctx = P.Context(0)
    job = synth.h2_fp64(0)
    J = P.Job.from_synth(ctx, job, P.FP64)
    ws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    out = {k: torch.empty(s, dtype=torch.float64, device="cuda") for k, s in J.out_shapes(job.mask).items()}
    with pytest.raises(P.PsqError) as e:
        J.autotune(job.mask, ws, out)
    assert e.value.status == 2
