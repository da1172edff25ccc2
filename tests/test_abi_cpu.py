"""C ABI checks that need no GPU: the library loads and exports every entry point of
include/psq.h; job validation; the host planner's grids, point counts and work counts agree
with the oracle's (planning-only context, no device)."""
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_2510_15204_gb300 as P
    if not os.path.exists(P.LIB_PATH):
        from paper_2510_15204_gb300 import build
        build.build()
    P.lib()
    return P


@pytest.fixture(scope="module")
def ctx(P):
    return P.Context(-1)


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "psq.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(psq_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(P):
    import ctypes
    L = ctypes.CDLL(P.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == {s[0] for s in P.SIGNATURES}


def test_planning_only_context_refuses_compute(P, ctx):
    j = P.Job.from_synth(ctx, synth.h2_fp64(0))
    import ctypes
    ptrs = (ctypes.c_void_p * 5)()
    st = P.lib().psq_compute(j.handle, 1, ctypes.c_void_p(256), 1 << 30, ptrs, None)
    assert st == 1 and b"planning only" in P.lib().psq_last_error()


@pytest.mark.parametrize("case,status", [
    ("l_ge_n", 1), ("zeta0", 1), ("coincident", 5), ("one_atom", 6), ("unsorted", 1),
    ("nspecs", 1), ("q17", 6), ("l7", 6), ("bad_atom", 1),
])
def test_job_validation(P, ctx, case, status):
    j = synth.triatomic_oh2(0)
    atoms, basis, aux, specs = list(j.atoms), list(j.basis), list(j.aux), list(j.specs)
    if case == "l_ge_n":
        basis[0] = (0, 1, 1, 1.0)
    elif case == "zeta0":
        aux[0] = (0, 1, 0, 0.0)
    elif case == "coincident":
        atoms[2] = (1, atoms[1][1])
    elif case == "one_atom":
        atoms = atoms[:1]
        basis = [s for s in basis if s[0] == 0]
        aux = [s for s in aux if s[0] == 0]
    elif case == "unsorted":
        basis = basis[::-1]
    elif case == "nspecs":
        specs = specs * 2
    elif case == "q17":
        specs = [(20, 15, 8, 17, 4, 4, 3)]
    elif case == "l7":
        aux.append((2, 8, 7, 1.0))
    elif case == "bad_atom":
        basis.append((5, 1, 0, 1.0))
    with pytest.raises(P.PsqError) as e:
        P.Job(ctx, atoms, basis, aux, specs)
    assert e.value.status == status


def _oracle_grid_sizes(job):
    sizes = {}
    nat = job.n_atoms
    for A in range(nat):
        for B in range(A + 1, nat):
            spec = job.spec_for_pair(A, B)
            sizes[(A, B, None)] = spec[0] * spec[1] * spec[2] * spec[3] * spec[4] * spec[5]
            for C in range(nat):
                if C in (A, B):
                    continue
                RA, RB, RC = (np.array(job.atoms[i][1]) for i in (A, B, C))
                a, M, Rm = oracle.pair_frame(RA, RB, RC)
                sizes[(A, B, C)] = len(oracle.grid_cells(spec, a, Rm.T @ (RC - M))) * spec[3] * spec[4] * spec[5]
    return sizes


def _collinear_job():
    atoms = [(1, (0.0, 0.0, 0.0)), (8, (0.0, 0.0, 1.5)), (1, (0.0, 0.0, 3.4)), (6, (300.0, 0.0, 0.7))]
    basis = [(a, 1, 0, 1.0 + 0.1 * a) for a in range(4)]
    aux = [(a, 2, 1, 1.2) for a in range(4)]
    return synth.Job("collinear", atoms, basis, aux, [(10, 8, 5, 3, 3, 3, 2)])


@pytest.mark.parametrize("make", [lambda: synth.triatomic_oh2(0), lambda: synth.c3h6(0), _collinear_job])
def test_grid_point_counts_match_oracle(P, ctx, make):
    job = make()
    J = P.Job.from_synth(ctx, job)
    ref = _oracle_grid_sizes(job)
    n = J.n_grids()
    assert n == len(ref)
    for g in range(n):
        A, B, C, K = J.grid_info(g)
        dead = 0
        if C is not None:
            dead = K - ref[(A, B, C)]  # w = 0 points at the unsplit touching cells
            spec = job.spec_for_pair(A, B)
            q3 = spec[3] * spec[4] * spec[5]
            assert dead % q3 == 0 and dead // q3 in (0, 8, 2 * 1 * spec[2])
        else:
            assert K == ref[(A, B, None)]


@pytest.mark.parametrize("make", [synth.h2_fp64, synth.triatomic_oh2, synth.c3h6, synth.fivez_triatomic])
def test_contraction_count_matches_oracle(P, ctx, make):
    job = make(0)
    J = P.Job.from_synth(ctx, job)
    for mask in (job.mask, oracle.S | oracle.J2, oracle.V | oracle.J3):
        assert J.stats(mask)["contractions"] == oracle.contractions(job, mask)


def test_launch_count_and_workspace(P, ctx):
    J = P.Job.from_synth(ctx, synth.triatomic_oh2(0))
    assert J.stats(oracle.ALL)["launches"] == 3 + 5
    assert J.stats(oracle.S)["launches"] == 3 + 1
    assert J.workspace_bytes(oracle.S) < J.workspace_bytes(oracle.ALL)
    assert J.stats(oracle.S)["grids"] == 3 and J.stats(oracle.ALL)["grids"] == 6


@pytest.mark.parametrize("make", [synth.h2_fp64, synth.triatomic_oh2, synth.c3h6])
def test_issued_flops_bound_the_useful_work(P, ctx, make):
    """The tensor-pipe roofline counts issued MMAs: fifteen slice products (orders 0..4 of
    five 8-bit slices) per useful product, plus tile padding and the duplicated triangle of
    symmetric blocks, so never less than 30 FLOPs per useful contraction; on the large blocks
    of C3H6 padding stays under 1.9x (its 3-index A tiles hold 72 or 90 aux rows of 128, and
    the one-centre pair tiles that a base grid's rows of one atom do not use are left out:
    55.7 FLOPs per contraction, 60.6 with them).  The FP64 path issues at least the useful 2
    FLOPs per contraction and at most 15% more on the triatomic and C3H6 (a pair grid's blocks
    hold only what an element reads; the symmetrised T and (P|Q) elements add their mirror
    blocks: 1.11x and 1.02x)."""
    job = make(0)
    for prec, lo in ((P.MIXED, 30.0), (P.FP64, 2.0)):
        J = P.Job.from_synth(ctx, job, prec)
        st = J.stats(job.mask)
        assert st["issued_flops"] >= lo * st["contractions"]
        if make is synth.c3h6 and prec == P.MIXED:
            assert st["issued_flops"] <= 1.9 * lo * st["contractions"]
        if make is not synth.h2_fp64 and prec == P.FP64:
            assert st["issued_flops"] <= 1.15 * lo * st["contractions"]


def test_noalloc_and_wait_limit_refuse_without_a_device(P, ctx):
    """The allocation-free entry point refuses a planning-only context (its job's device is
    not a device); the wait limit refuses a NULL job and out-of-range limits."""
    import ctypes
    J = P.Job.from_synth(ctx, synth.h2_fp64(0))
    J.workspace_bytes(oracle.ALL)
    ptrs = (ctypes.c_void_p * 5)()
    L = P.lib()
    assert L.psq_compute_noalloc(J.handle, oracle.ALL, ptrs, None) != 0
    assert L.psq_job_set_wait_limit(None, 1000) == 1
    assert L.psq_job_set_wait_limit(J.handle, 0) == 1
    assert L.psq_job_set_wait_limit(J.handle, 61 * 10 ** 9) == 1
    assert L.psq_job_set_wait_limit(J.handle, 2000) == 0


def test_autotune_needs_a_device(P, ctx):
    import ctypes
    J = P.Job.from_synth(ctx, synth.h2_fp64(0))
    ptrs = (ctypes.c_void_p * 5)()
    st = P.lib().psq_job_autotune(J.handle, oracle.ALL, None, 0, ptrs, None, None, None)
    assert st == 1  # PSQ_ERR_ARG: planning-only context


def test_ri_entry_points_validate_arguments_without_a_gpu(P):
    """psq_ri_* refuse bad sizes, ranges and pointers before touching the device."""
    import ctypes
    L = P.lib()
    dummy = ctypes.c_void_p(64)  # never dereferenced: every call below fails its checks first
    info = ctypes.c_void_p(64)
    assert L.psq_ri_factor(-1, dummy, dummy, info, None) == 1
    assert L.psq_ri_factor(4, None, dummy, info, None) == 1
    assert L.psq_ri_factor(4, dummy, dummy, None, None) == 1
    assert L.psq_ri_factor(4, ctypes.c_void_p(65), dummy, info, None) == 1  # misaligned
    assert L.psq_ri_solve(-2, 5, dummy, dummy, None) == 1
    assert L.psq_ri_solve(3, 5, None, dummy, None) == 1
    assert L.psq_ri_solve(0, 5, None, None, None) == 0  # nothing to do
    assert L.psq_ri_eri(3, 10, dummy, 8, 5, 0, 2, dummy, None) == 1  # c0 + nc > m
    assert L.psq_ri_eri(3, 10, dummy, 0, 2, -1, 2, dummy, None) == 1
    assert L.psq_ri_eri(3, 10, dummy, 0, 0, 0, 4, None, None) == 0  # empty block
    nbytes = ctypes.c_size_t()
    assert L.psq_ri_eri_mixed_workspace(-1, 4, 4, ctypes.byref(nbytes)) == 1
    assert L.psq_ri_eri_mixed_workspace(82, 676, 676, None) == 1
    assert L.psq_ri_eri_mixed_workspace(82, 676, 676, ctypes.byref(nbytes)) == 0 and nbytes.value > 676 * 676 * 8
    assert L.psq_ri_eri_mixed(3, 10, dummy, 8, 5, 0, 2, dummy, dummy, 1 << 20, None) == 1  # c0 + nc > m
    assert L.psq_ri_eri_mixed(3, 10, dummy, 0, 2, 0, 2, dummy, ctypes.c_void_p(64 + 8), 1 << 20, None) == 1  # ws align
    assert L.psq_ri_eri_mixed(3, 10, dummy, 0, 0, 0, 2, None, None, 0, None) == 0  # empty block


def test_measure_peaks_refuses_without_a_device(P):
    """The pipe-rate probe returns PSQ_ERR_CUDA with a message where no CUDA device exists."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    L = P.lib()
    assert L.psq_measure_peaks(None, None, None, None) == 3
    assert b"no CUDA device" in L.psq_last_error()
