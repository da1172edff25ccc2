"""Parity of the mixed-precision CUDA path (FP32 function values, tcgen05 contraction of
exact 8-bit integer slices with FP32 accumulation, double-float and FP64 sums) with the
FP64 CPU oracle.

Reported per class: the largest absolute error and the largest error relative to
max(C, 1e-4 x the class's largest C), C = the element's absolute-term sum (function values are
FP32, so elements far below the class scale carry FP32-level absolute error).  Bars: the
relative bar MIXED_REL holds for every class; the absolute errors are printed (the target
for them is 1e-9, which FP32 function values do not reach).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

CLASSES = ("S", "T", "V", "J2", "J3")
MIXED_REL = 2e-6


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
    ws, out = J.alloc(mask)
    J.compute(mask, ws, out)
    J.check(mask, ws)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def errors(got, ref, mask):
    """(largest absolute error, largest error relative to max(C, 1e-4 x the class's largest C))."""
    rep = {}
    for i, k in enumerate(CLASSES):
        if not (mask >> i) & 1:
            continue
        d = np.abs(got[k] - ref[k])
        scale = np.maximum(np.abs(ref[k]), ref["abs" + k])
        scale = np.maximum(scale, 1e-4 * ref["abs" + k].max())
        rel = d / np.where(scale > 0, scale, 1.0)
        rep[k] = (float(d.max()), float(rel.max()))
    return rep


@pytest.mark.parametrize("make", [lambda: synth.h2_fp64(0), lambda: synth.triatomic_oh2(0)])
def test_mixed_matches_oracle(P, ctx, make):
    job = make()
    mask = oracle.ALL
    ref = oracle.compute(job, mask=mask)
    got = run(P, ctx, job, mask, P.MIXED)
    rep = errors(got, ref, mask)
    print("\n%s mixed errors (abs, rel-to-C):" % job.name, {k: "%.2e %.2e" % v for k, v in rep.items()})
    for k, (ab, rel) in rep.items():
        assert rel < MIXED_REL, (k, ab, rel)


def test_mixed_small_blocks_and_ragged_tail(P, ctx):
    """Grids whose point counts are not multiples of the 64-point chunk, N_SP = 1, Q = 4
    (cell-aligned chunks; chunks that straddle coarse cells are covered below), blocks
    narrower than one MMA tile."""
    job = synth.triatomic_oh2(3)
    job.specs = [(7, 5, 3, 4, 4, 4, 1)]
    mask = oracle.ALL
    ref = oracle.compute(job, mask=mask)
    got = run(P, ctx, job, mask, P.MIXED)
    rep = errors(got, ref, mask)
    print("\nragged mixed errors:", {k: "%.2e %.2e" % v for k, v in rep.items()})
    for k, (ab, rel) in rep.items():
        assert rel < MIXED_REL, (k, ab, rel)


def test_mixed_wide_blocks(P, ctx):
    """More than 128 pair rows and more than 64 aux columns: several M and N tiles."""
    job = synth.fivez_diatomic(0)
    job.specs = [(8, 6, 4, 4, 4, 4, 2)]
    mask = oracle.J3 | oracle.J2 | oracle.S
    ref = oracle.compute(job, mask=mask)
    got = run(P, ctx, job, mask, P.MIXED)
    rep = errors(got, ref, mask)
    print("\nwide mixed errors:", {k: "%.2e %.2e" % v for k, v in rep.items()})
    for k, (ab, rel) in rep.items():
        assert rel < MIXED_REL, (k, ab, rel)


def test_mixed_agrees_with_fp64_path(P, ctx):
    job = synth.triatomic_oh2(1)
    job.specs = [(10, 8, 4, 4, 4, 4, 3)]
    a = run(P, ctx, job, oracle.ALL, P.FP64)
    b = run(P, ctx, job, oracle.ALL, P.MIXED)
    for k in CLASSES:
        scale = max(1.0, float(np.abs(a[k]).max()))
        assert np.abs(a[k] - b[k]).max() < 1e-5 * scale, k


def test_mixed_chunks_straddling_coarse_cells(P, ctx):
    """Q = (3,5,3): 45-point cells, so 64-point scale chunks straddle cells of very different
    magnitude on this deliberately coarse grid.  Known weak spot: the kinetic class reaches
    ~3e-5 of C here (1e-7 on the production grids); bar 1e-4."""
    job = synth.triatomic_oh2(3)
    job.specs = [(7, 5, 3, 3, 5, 3, 1)]
    mask = oracle.ALL
    ref = oracle.compute(job, mask=mask)
    got = run(P, ctx, job, mask, P.MIXED)
    rep = errors(got, ref, mask)
    print("\nstraddling mixed errors:", {k: "%.2e %.2e" % v for k, v in rep.items()})
    for k, (ab, rel) in rep.items():
        assert rel < 1e-4, (k, ab, rel)
