"""Parity of the mixed-precision CUDA path (double-float function values and weights, tcgen05
contraction of five exact 8-bit integer slices with FP32 accumulation, double-float and FP64
sums) with the FP64 CPU oracle.

The bar is the mixed path's target: every element of every class within MIXED_ABS = 1e-9
absolute of the oracle.  Reported per class: the largest absolute error and the largest
error relative to max(|value|, C), C = the element's absolute-term sum.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

CLASSES = ("S", "T", "V", "J2", "J3")
MIXED_ABS = 1e-9


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
    """(largest absolute error, largest error relative to max(|value|, C)) per class."""
    rep = {}
    for i, k in enumerate(CLASSES):
        if not (mask >> i) & 1:
            continue
        d = np.abs(got[k] - ref[k])
        scale = np.maximum(np.abs(ref[k]), ref["abs" + k])
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
        assert ab <= MIXED_ABS, (k, ab, rel)


def test_mixed_small_blocks_and_ragged_tail(P, ctx):
    """Grids whose point counts are not multiples of the 32-point chunk or the 128-point
    window, N_SP = 1, Q = 4, blocks narrower than one MMA tile."""
    job = synth.triatomic_oh2(3)
    job.specs = [(7, 5, 3, 4, 4, 4, 1)]
    mask = oracle.ALL
    ref = oracle.compute(job, mask=mask)
    got = run(P, ctx, job, mask, P.MIXED)
    rep = errors(got, ref, mask)
    print("\nragged mixed errors:", {k: "%.2e %.2e" % v for k, v in rep.items()})
    for k, (ab, rel) in rep.items():
        assert ab <= MIXED_ABS, (k, ab, rel)


def test_mixed_wide_blocks(P, ctx):
    """More than 128 pair rows and more than 48 aux columns: several M and N tiles."""
    job = synth.fivez_diatomic(0)
    job.specs = [(8, 6, 4, 4, 4, 4, 2)]
    mask = oracle.J3 | oracle.J2 | oracle.S
    ref = oracle.compute(job, mask=mask)
    got = run(P, ctx, job, mask, P.MIXED)
    rep = errors(got, ref, mask)
    print("\nwide mixed errors:", {k: "%.2e %.2e" % v for k, v in rep.items()})
    for k, (ab, rel) in rep.items():
        assert ab <= MIXED_ABS, (k, ab, rel)


def test_mixed_agrees_with_fp64_path(P, ctx):
    job = synth.triatomic_oh2(1)
    job.specs = [(10, 8, 4, 4, 4, 4, 3)]
    a = run(P, ctx, job, oracle.ALL, P.FP64)
    b = run(P, ctx, job, oracle.ALL, P.MIXED)
    for k in CLASSES:
        assert np.abs(a[k] - b[k]).max() <= MIXED_ABS, k


def test_mixed_chunks_straddling_coarse_cells(P, ctx):
    """Q = (3,5,3): 45-point cells, so 128-point scale windows straddle cells of very different
    magnitude on this deliberately coarse grid (each value keeps 39 bits of its window's
    largest, so the relative error of small elements grows; the absolute bar holds)."""
    job = synth.triatomic_oh2(3)
    job.specs = [(7, 5, 3, 3, 5, 3, 1)]
    mask = oracle.ALL
    ref = oracle.compute(job, mask=mask)
    got = run(P, ctx, job, mask, P.MIXED)
    rep = errors(got, ref, mask)
    print("\nstraddling mixed errors:", {k: "%.2e %.2e" % v for k, v in rep.items()})
    for k, (ab, rel) in rep.items():
        assert ab <= MIXED_ABS, (k, ab, rel)
