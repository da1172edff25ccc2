"""The mixed path's grid waves (a bounded workspace): a job planned with a small wave budget
runs its grids in several waves on shared operand / packed / partial regions and gives the
results of the single-wave plan (to rounding: other waves cut the point ranges differently)
and the oracle's to 1e-9 absolute; the workspace shrinks accordingly."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_waves_match_single_wave_and_oracle():
    import torch
    import paper_2510_15204_gb300 as P
    from paper_2510_15204_gb300 import build
    build.build()
    ctx = P.Context(0)
    job = synth.triatomic_oh2(2)
    job.specs = [(12, 9, 6, 4, 4, 4, 3)]
    mask = oracle.ALL
    ref = oracle.compute(job, mask=mask)
    J = P.Job.from_synth(ctx, job, P.MIXED)
    one = J.workspace_bytes(mask)
    assert J.stats(mask)["launches"] == 1 + 4 + 5  # nodes, one wave, assembly
    a = J.compute(mask)
    J.set_wave_budget(1)  # every grid a wave of its own
    many = J.workspace_bytes(mask)
    st = J.stats(mask)
    assert st["launches"] == 1 + 4 * st["grids"] + 5
    assert many < one
    ws, out = J.alloc(mask)
    J.compute(mask, ws, out)
    J.check(mask, ws)
    torch.cuda.synchronize()
    for k in P.CLASSES:
        b = out[k].cpu().numpy()
        aa = a[k].cpu().numpy()
        assert np.abs(b - ref[k]).max() <= 1e-9, (k, float(np.abs(b - ref[k]).max()))
        assert np.abs(b - aa).max() <= 1e-12 * max(1.0, float(np.abs(aa).max())), k
