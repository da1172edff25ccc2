"""The serving loop: jobs of different sizes submitted together run concurrently on their own
streams out of one device arena; each result must equal the same job computed alone (the
kernels are deterministic, so equality is exact up to the stated tolerance)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SPEC = (10, 8, 4, 4, 4, 4, 2)


def _jobs(n, seed):
    rng = np.random.default_rng(seed)
    out = [synth.h2_fp64(0, spec=SPEC, mask=oracle.ALL)]
    while len(out) < n:
        out.append(synth.random_molecule(rng, spec=SPEC, n_bf_range=(8, 120)))
    return out


def _host_out(P, J, mask):
    import torch
    return {k: torch.empty(s, dtype=torch.float64).pin_memory() for k, s in J.out_shapes(mask).items()}


@pytest.mark.parametrize("precision", [0, 1])
def test_results_equal_alone_and_in_the_mix(precision):
    import torch
    import paper_2510_15204_gb300 as P
    from paper_2510_15204_gb300 import build
    build.build()
    ctx = P.Context(0)
    mask = oracle.ALL
    jobs = [P.Job.from_synth(ctx, j, precision) for j in _jobs(8, 11)]
    alone = []
    for J in jobs:
        ws, out = J.alloc(mask)
        J.compute(mask, ws, out)
        torch.cuda.synchronize()
        alone.append({k: v.cpu() for k, v in out.items()})
        del ws, out
    need = max(J.workspace_bytes(mask) for J in jobs)
    server = P.Server(ctx, arena_bytes=int(2.5 * need) + (64 << 20), max_inflight=4)
    outs = [_host_out(P, J, mask) for J in jobs]
    tickets = [server.submit(J, mask, o) for J, o in zip(jobs, outs)]
    lat = [server.wait(t) for t in tickets]
    server.close()
    assert all(x > 0 for x in lat)
    for a, b in zip(alone, outs):
        for k in a:
            assert torch.equal(a[k], b[k]), k


def test_job_larger_than_arena_is_refused():
    import paper_2510_15204_gb300 as P
    ctx = P.Context(0)
    J = P.Job.from_synth(ctx, synth.triatomic_oh2(0), P.FP64)
    server = P.Server(ctx, arena_bytes=64 << 20, max_inflight=2)
    with pytest.raises(P.PsqError) as e:
        server.submit(J, oracle.ALL, _host_out(P, J, oracle.ALL))
    assert e.value.status == 2
    server.close()
