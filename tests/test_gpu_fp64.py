"""Parity of the plain FP64 CUDA path with the CPU oracle, element by element.

Tolerance (FP64 plain path, 1e-12 relative per element): for every element,
|gpu - oracle| <= 1e-12 * max(|oracle|, C), where C is the sum of the absolute values of the
terms of that element's quadrature sum (the oracle's "abs" matrices).  Elements that vanish
by symmetry are sums of cancelling terms; C is the scale their rounding lives on.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12
CLASSES = ("S", "T", "V", "J2", "J3")


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


def run_gpu(P, ctx, job, mask=None, precision=0):
    import torch
    mask = job.mask if mask is None else mask
    J = P.Job.from_synth(ctx, job, precision)
    out = J.compute(mask)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}, J


def rel_err(gpu, ref, absref):
    scale = np.maximum(np.abs(ref), absref)
    scale = np.where(scale > 0, scale, 1.0)
    return np.abs(gpu - ref) / scale


def assert_parity(got, ref, mask, tol=TOL):
    worst = {}
    for i, k in enumerate(CLASSES):
        if not (mask >> i) & 1:
            continue
        e = rel_err(got[k], ref[k], ref["abs" + k])
        worst[k] = float(e.max()) if e.size else 0.0
        assert worst[k] <= tol, (k, worst[k], np.unravel_index(int(np.argmax(e)), e.shape))
    return worst


# ------------------------------------------------------------------ step parity: grid (a1-a4)

def _gpu_points(J, g):
    import torch
    pts = J.grid_points(g)
    torch.cuda.synchronize()
    return pts.cpu().numpy()


@pytest.mark.parametrize("make", [lambda: synth.h2_fp64(0), lambda: synth.triatomic_oh2(0)])
def test_grid_points_match_oracle(P, ctx, make):
    job = make()
    J = P.Job.from_synth(ctx, job)
    for g in range(J.n_grids()):
        A, B, C, K = J.grid_info(g)
        pts = _gpu_points(J, g)
        live = pts[3] != 0.0
        ref = oracle.build_grid(job.atoms, job.spec_for_pair(A, B), A, B, C)
        assert live.sum() == len(ref["w"])
        np.testing.assert_allclose(pts[0:3, live].T, ref["P"], rtol=0, atol=1e-13 * max(1.0, np.abs(ref["P"]).max()))
        np.testing.assert_allclose(pts[3, live], ref["w"], rtol=1e-13, atol=0)
        np.testing.assert_allclose(pts[4, live], ref["rA"], rtol=1e-13, atol=0)
        np.testing.assert_allclose(pts[5, live], ref["rB"], rtol=1e-13, atol=0)


def test_grid_points_collinear_and_outside(P, ctx):
    atoms = [(1, (0.0, 0.0, 0.0)), (8, (0.0, 0.0, 1.5)), (1, (0.0, 0.0, 3.4)), (6, (300.0, 0.0, 0.7))]
    basis = [(a, 1, 0, 1.0) for a in range(4)]
    job = synth.Job("collinear", atoms, basis, [], [(10, 8, 5, 3, 3, 3, 2)])
    J = P.Job.from_synth(ctx, job)
    for g in range(J.n_grids()):
        A, B, C, K = J.grid_info(g)
        pts = _gpu_points(J, g)
        live = pts[3] != 0.0
        ref = oracle.build_grid(job.atoms, job.spec_for_pair(A, B), A, B, C)
        assert live.sum() == len(ref["w"]), (A, B, C)
        # a 300-bohr pair next to a 1.5-bohr one: the frame and third-centre coordinates carry
        # cancellation of order 300/1.5 ulps, and the split cells beside a moved line are thin
        np.testing.assert_allclose(pts[3, live], ref["w"], rtol=5e-12, atol=0)
        np.testing.assert_allclose(pts[0:3, live].T, ref["P"], rtol=0, atol=1e-12 * np.abs(ref["P"]).max())


# ------------------------------------------------------------------ step parity: functions (a5-a6)

@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 4e-12)])
@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_function_values_match_oracle(P, ctx, kind, precision, tol):
    """STO values, kinetic operands, aux functions and aux potentials (eq 1, eq 16) on every
    grid of the triatomic job.  The mixed path (precision 1) evaluates double-float values
    (about 48 bits) of x = zeta r and the direction, times FP64 row constants; its bar is a
    few times the FP64 one (its points come from double-float node tables)."""
    import torch
    job = synth.triatomic_oh2(0)
    J = P.Job.from_synth(ctx, job, precision)
    for g in range(J.n_grids()):
        A, B, C, K = J.grid_info(g)
        vals = J.grid_functions(g, kind)
        pts = J.grid_points(g)
        torch.cuda.synchronize()
        vals, pts = vals.cpu().numpy(), pts.cpu().numpy()
        live = pts[3] != 0.0
        ref = oracle.build_grid(job.atoms, job.spec_for_pair(A, B), A, B, C)
        rows, shells, lscale = [], [], []
        if kind in (0, 1):
            for X, key in ((A, "A"), (B, "B")):
                sh = [s for s in job.basis if s[0] == X]
                shells += sh
                r = ref["r" + key]
                F, L = oracle.sto_values(sh, r, ref["d" + key], with_laplacian=True)
                rows.append(F if kind == 0 else L)
                for (_, n, l, z) in sh:  # size of the terms of lap chi's radial factor
                    lscale.append(np.repeat((abs(n * (n - 1) - l * (l + 1)) / r ** 2 + 2 * n * z / r + z * z)[None, :],
                                            2 * l + 1, axis=0))
        else:
            centres = [A, B] if C is None else [C]
            for X in centres:
                sh = [s for s in job.aux if s[0] == X]
                shells += sh
                if X == A:
                    r, d = ref["rA"], ref["dA"]
                elif X == B:
                    r, d = ref["rB"], ref["dB"]
                else:
                    d = ref["P"] - np.array(job.atoms[X][1])
                    r = np.linalg.norm(d, axis=1)
                rows.append(oracle.sto_values(sh, r, d) if kind == 2 else oracle.aux_potential_values(sh, r, d))
        R = np.concatenate(rows)
        got = vals[:, live]
        assert got.shape == R.shape
        # scale of each value: the largest |value| over m of its shell at that point
        # (harmonics have nodal planes; their direction error is relative to the shell)
        scale = np.empty_like(R)
        base = np.concatenate(rows) if kind != 1 else None
        if kind == 1:  # lap chi = f(r) chi: scale by |chi| times the size of f's terms
            F = []
            for X, key in ((A, "A"), (B, "B")):
                sh = [s for s in job.basis if s[0] == X]
                F.append(oracle.sto_values(sh, ref["r" + key], ref["d" + key]))
            base = np.concatenate(F) * np.concatenate(lscale)
        r0 = 0
        for sh in shells:
            nf = 2 * sh[2] + 1
            scale[r0:r0 + nf] = np.abs(base[r0:r0 + nf]).max(axis=0)[None, :]
            r0 += nf
        if precision == 1:
            # double-float e^-x keeps its relative precision while e^-x > ~1e-31 and is 0 past
            # x = 87 (values ~1e-32 of their row's largest): values below 1e-18 of their row's
            # largest are compared absolutely, against that
            scale = np.maximum(scale, 1e-18 * np.abs(R).max(axis=1, keepdims=True))
        err = np.abs(got - R) / np.maximum(scale, 1e-290)
        r, q = np.unravel_index(int(err.argmax()), err.shape)
        assert err.max() < tol, (g, kind, float(err.max()), int(r), int(q), float(got[r, q]), float(R[r, q]),
                                 float(scale[r, q]), shells)


# ------------------------------------------------------------------ full path parity (a1-a9)

@pytest.mark.parametrize("seed", [0, 1])
def test_h2_all_classes(P, ctx, seed):
    job = synth.h2_fp64(seed)
    ref = oracle.compute(job, mask=oracle.ALL)
    got, _ = run_gpu(P, ctx, job, oracle.ALL)
    assert_parity(got, ref, oracle.ALL)


def test_triatomic_full_size_all_classes(P, ctx):
    """The triatomic workload at its full size (grids 20/15/8 Q4 N_SP 3, 963k points)."""
    job = synth.triatomic_oh2(0)
    ref = oracle.compute(job, mask=oracle.ALL)
    got, _ = run_gpu(P, ctx, job, oracle.ALL)
    assert_parity(got, ref, oracle.ALL)


@pytest.mark.parametrize("mask", [oracle.S, oracle.T | oracle.J2, oracle.V, oracle.J3, oracle.V | oracle.J3])
def test_class_subsets(P, ctx, mask):
    job = synth.triatomic_oh2(1)
    job.specs = [(9, 7, 4, 3, 3, 3, 2)]
    ref = oracle.compute(job, mask=mask)
    got, _ = run_gpu(P, ctx, job, mask)
    assert_parity(got, ref, mask)


def test_ragged_grids_and_edge_cases(P, ctx):
    """Collinear third centre (every phi cell split), a third centre outside mu_max, N_SP = 1,
    Q = (5,3,2), an atom with no aux functions, per-pair specs, 4 atoms."""
    atoms = [(1, (0.0, 0.0, 0.0)), (8, (0.0, 0.0, 1.5)), (1, (0.0, 0.0, 3.4)), (6, (60.0, 0.0, 0.7))]
    basis = [(0, 1, 0, 1.1), (0, 2, 1, 0.9), (1, 1, 0, 3.0), (1, 2, 1, 1.4), (1, 3, 2, 1.2),
             (2, 1, 0, 0.8), (3, 1, 0, 1.6), (3, 2, 1, 1.0)]
    aux = [(0, 1, 0, 1.5), (0, 2, 1, 2.0), (1, 1, 0, 4.0), (1, 3, 2, 2.5), (1, 4, 3, 3.0),
           (3, 2, 1, 2.2)]
    specs = [(6, 5, 3, 5, 3, 2, 1), (7, 4, 4, 3, 3, 3, 2), (5, 6, 3, 4, 4, 2, 3),
             (6, 5, 4, 3, 3, 3, 2), (4, 4, 2, 3, 3, 3, 1), (5, 5, 3, 2, 3, 4, 2)]
    job = synth.Job("edge", atoms, basis, aux, specs)
    ref = oracle.compute(job, mask=oracle.ALL)
    got, _ = run_gpu(P, ctx, job, oracle.ALL)
    assert_parity(got, ref, oracle.ALL)


def test_bitwise_reproducible(P, ctx):
    import torch
    job = synth.triatomic_oh2(2)
    job.specs = [(8, 6, 4, 3, 3, 3, 2)]
    J = P.Job.from_synth(ctx, job)
    ws, out = J.alloc(oracle.ALL)
    a = {k: v.clone() for k, v in J.compute(oracle.ALL, ws, out).items()}
    torch.cuda.synchronize()
    b = J.compute(oracle.ALL, ws, out)
    torch.cuda.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_compute_host_matches_device(P, ctx):
    import torch
    job = synth.h2_fp64(0)
    J = P.Job.from_synth(ctx, job)
    ws, out = J.alloc(oracle.ALL)
    host = {k: torch.empty(v.shape, dtype=torch.float64).pin_memory() for k, v in out.items()}
    J.compute_host(oracle.ALL, ws, out, host)
    for k in out:
        assert torch.equal(host[k], out[k].cpu()), k


def test_workspace_too_small_is_an_error(P, ctx):
    import torch
    job = synth.h2_fp64(0)
    J = P.Job.from_synth(ctx, job)
    ws, out = J.alloc(oracle.ALL)
    with pytest.raises(P.PsqError) as e:
        J.compute(oracle.ALL, ws[: ws.numel() // 2], out)
    assert e.value.status == 2
