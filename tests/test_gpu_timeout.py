"""Failure detection on the GPU without a fault: every wait of the tensor-core contraction is
bounded.  With the test hook on, the compute raises a flag that nothing clears and the
contraction's loader waits for it; with a 2 ms wait limit that wait runs out, the kernel
records PSQ_ERR_TIMEOUT in the workspace's status word (read by psq_check), every role leaves
its loop, the copies and MMAs in flight are drained and the tensor memory released.  The
context stays usable: the next compute with the hook off and the default limit, on the same
workspace, matches the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_wait_timeout_is_reported_and_the_context_recovers():
    import torch
    import paper_2510_15204_gb300 as P
    from paper_2510_15204_gb300 import build
    build.build()
    ctx = P.Context(0)
    job = synth.h2_fp64(0)
    job.specs = [(20, 14, 8, 4, 4, 4, 3)]  # enough windows per work item for many waits
    mask = oracle.ALL
    J = P.Job.from_synth(ctx, job, P.MIXED)
    ws, out = J.alloc(mask)
    J.set_wait_limit(2 * 10 ** 6)
    J.test_stall(True)
    J.compute(mask, ws, out)
    with pytest.raises(P.PsqError) as e:
        J.check(mask, ws)
    assert e.value.status == 4  # PSQ_ERR_TIMEOUT
    torch.cuda.synchronize()  # the context still answers
    J.test_stall(False)
    J.set_wait_limit(4 * 10 ** 9)
    J.compute(mask, ws, out)
    J.check(mask, ws)
    ref = oracle.compute(job, mask=mask)
    for k in P.CLASSES:
        d = np.abs(out[k].cpu().numpy() - ref[k]).max()
        assert d <= 1e-9, (k, float(d))
