/*
 * psq.h - C ABI of the GB300 prolate-spheroidal (PS) quadrature library for Slater-type
 * orbital (STO) integrals.
 *
 * Method: Stark et al., "Numerical Integration of Slater Basis Functions Over Prolate
 * Spheroidal Grids" (arXiv 2510.15204).  For every atom pair a PS grid (Section 2.1,
 * eqs 2-7, 10-12, 17; Algorithms 1-2) is built, refined around a third centre where a
 * 3-centre term needs it (Section 2.2, Fig. 2, parameter N_SP).  STOs (eq 1) and the
 * Coulomb potentials of RI auxiliary functions (eqs 15-16) are evaluated on its points and
 * contracted by eq 9 into overlap S, kinetic T, nuclear attraction V, 2-centre (P|Q) and
 * 3-centre (P|ij) matrices.  Polyatomics are assembled from grids over at most three atoms
 * (Section 4): every matrix element is integrated on exactly one grid, picked by the
 * distinct centres of its integrand (one centre: the pair grid of that atom and its nearest
 * neighbour, ties to the lower index; two: their pair grid; three: the pair grid of the two
 * basis-function atoms refined around the third).  One-centre overlap and kinetic elements
 * are not integrated: they take their closed forms (the reading under which Table 1's
 * kinetic RMSE is reproduced).
 *
 * Conventions.  Atomic units (bohr).  Shells must be listed grouped by atom in ascending
 * atom order.  Function order: atom, then shell as listed, then m = -l..l of real
 * orthonormal spherical harmonics (no Condon-Shortley phase).  Radial normalisation
 * N = (2 zeta)^(n+1/2) / sqrt((2n)!).  Pair (A,B) puts the lower atom index A at (0,0,+a).
 * Kinetic integrals use -1/2 chi_a lap chi_b symmetrised, (P|Q) is symmetrised.
 *
 * Errors.  Every call returns a psq_status; no call throws or aborts.  psq_last_error()
 * gives a message for the calling thread's last failure.  On a failed call no output has
 * been written unless the status is PSQ_ERR_CUDA / PSQ_ERR_TIMEOUT raised by a kernel, in
 * which case outputs are undefined.
 *
 * Memory.  The library allocates no device memory of its own for a computation: the
 * caller passes a device workspace (size from psq_job_workspace) and device output
 * buffers.  Jobs copy their inputs at creation; the caller may free them afterwards.  A
 * job holds a small page-locked host staging buffer for its tables.
 */
#ifndef PSQ_H
#define PSQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PSQ_OK = 0,
  PSQ_ERR_ARG = 1,         /* invalid argument: bad Z, l >= n, zeta <= 0, sizes, pointers */
  PSQ_ERR_OOM = 2,         /* host allocation failed or workspace too small */
  PSQ_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  PSQ_ERR_TIMEOUT = 4,     /* a bounded device wait expired; the context stays usable */
  PSQ_ERR_GEOMETRY = 5,    /* coincident atoms or an unusable pair geometry */
  PSQ_ERR_UNSUPPORTED = 6  /* e.g. a single atom, l > 6, Q > 16 */
} psq_status;

typedef struct { int Z; double xyz[3]; } psq_atom;             /* Z >= 0, position in bohr */
typedef struct { int atom, n, l; double zeta; } psq_shell;      /* n > l >= 0, zeta > 0     */

/* The five grid variables of Section 3 (N_mu, N_nu, N_phi, Q, N_SP), with Q per dimension
 * as Algorithm 2 allows: n_mu x n_nu x n_phi volume elements, q_mu x q_nu x q_phi
 * Gauss-Legendre points in each, and each volume element touching a third centre split
 * n_sp times per dimension.  1 <= q <= 16; a refined grid needs n_mu, n_nu >= 2. */
typedef struct { int n_mu, n_nu, n_phi, q_mu, q_nu, q_phi, n_sp; } psq_grid_spec;

typedef enum {
  PSQ_FP64 = 0,  /* plain path: every step in FP64 */
  PSQ_MIXED = 1  /* FP64 node tables, third-centre offsets, row constants and range sums;
                    double-float (FP32 hi + lo, ~48 bits) weights, STO values and aux
                    potentials; contraction on tcgen05 tensor cores: five 8-bit integer slices
                    per value in BF16 under a power-of-two scale per row and 128-point window
                    (39 bits of the window's largest value), the slice products of orders
                    0..4 accumulated exactly in FP32 and folded into double-float sums */
} psq_precision;

enum { PSQ_S = 1, PSQ_T = 2, PSQ_V = 4, PSQ_J2 = 8, PSQ_J3 = 16, PSQ_ALL = 31 };

typedef struct psq_context psq_context;
typedef struct psq_job psq_job;

/* Binds a context to a CUDA device (makes it current on the calling thread).  device = -1
 * makes a planning-only context: its jobs can be created, sized and queried, not computed. */
psq_status psq_context_create(int device, psq_context** out);
psq_status psq_context_destroy(psq_context* ctx);

/* Plans a job: validates and copies atoms and shells, builds every pair frame, the cell
 * edges (eq 7, 12, 17), the third-centre line moves and splits (Section 2.2) and the
 * block assignment.  pair_specs holds n_atoms*(n_atoms-1)/2 specs in pair order
 * (0,1),(0,2)..(0,n-1),(1,2).. or a single spec for every pair (n_specs == 1). */
psq_status psq_job_create(psq_context* ctx, const psq_atom* atoms, int n_atoms,
                          const psq_shell* basis, int n_basis_shells,
                          const psq_shell* aux, int n_aux_shells,
                          const psq_grid_spec* pair_specs, int n_specs,
                          psq_precision precision, psq_job** out);
psq_status psq_job_destroy(psq_job* job);

/* Basis and aux function counts. */
psq_status psq_job_sizes(const psq_job* job, int* n_bf, int* n_aux);

/* Device workspace bytes psq_compute needs for the classes in mask. */
psq_status psq_job_workspace(const psq_job* job, unsigned mask, size_t* bytes);

/* Workspace bound of the PSQ_MIXED path (no paper counterpart).  Its grids are processed in
 * waves of consecutive grids whose double-float operand rows and packed panels together stay
 * within `bytes` (a wave holds at least one grid; 0 selects the default, 6 GiB); the operand,
 * packed and partial-sum regions of the workspace are shared by the waves, so the workspace is
 * about the largest wave plus the result blocks.  Plans (and captured graphs) made before are
 * dropped; later calls plan with the new bound.  No effect on PSQ_FP64 jobs.  Errors:
 * PSQ_ERR_ARG for a NULL job. */
psq_status psq_job_set_wave_budget(psq_job* job, size_t bytes);

/* Job statistics: number of grids, total quadrature points (over the grids mask needs),
 * useful contractions (sum over integrated blocks of rows x cols x points, each (P,i<=j)
 * once on a same-atom pair), and kernel launches psq_compute issues for mask. */
psq_status psq_job_stats(const psq_job* job, unsigned mask, int* n_grids, int64_t* n_points,
                         double* contractions, int* launches);

/* Autotuning (the batched launch's work split; no paper counterpart).  Plans mask with each
 * candidate work split (PSQ_MIXED: 2, 4, 6, 8, 16 or 32 contraction work items per SM;
 * PSQ_FP64: 2, 4, 8 or 16 waves of CTAs per SM), runs each candidate that fits ws_bytes once to warm up
 * and three times under CUDA events on stream, keeps the fastest as the job's plan for mask
 * (later psq_compute / psq_compute_graph / psq_job_workspace calls use it; graphs captured
 * before are dropped) and returns its split and mean milliseconds (either pointer may be
 * NULL).  Synchronises the stream.  d_out holds valid results afterwards (of the last
 * candidate run).  Errors: PSQ_ERR_ARG for a planning-only context, NULL or misaligned
 * arguments; PSQ_ERR_OOM when no candidate fits ws_bytes; PSQ_ERR_CUDA on a failed launch. */
psq_status psq_job_autotune(psq_job* job, unsigned mask, void* d_workspace, size_t ws_bytes, double* d_out[5],
                            void* stream, int* work_split, float* best_ms);

/* Floating-point operations the contraction kernel issues in one psq_compute for mask (the
 * measure a tensor-pipe roofline counts; no paper counterpart).  PSQ_MIXED: every tensor-core
 * MMA of the 8-bit slice products, tiles of 128 rows x 48 columns whatever their fill, 15
 * slice products per 32-point chunk, each M x N x K MMA counting 2MNK.  PSQ_FP64: 2 x rows x cols x
 * points summed over the computed blocks.  Errors: PSQ_ERR_ARG for NULL pointers or unknown
 * mask bits. */
psq_status psq_job_issued_flops(const psq_job* job, unsigned mask, double* flops);

/* Computes the classes in mask, asynchronously on `stream` (a cudaStream_t; NULL = legacy
 * default stream).  d_out[0..4] are device buffers for S, T, V (n_bf*n_bf doubles each,
 * row-major), J2 (n_aux*n_aux) and J3 (n_aux*n_bf*n_bf, [P][i][j]); entries for classes
 * not in mask may be NULL.  d_workspace: at least psq_job_workspace(mask) bytes of device
 * memory, 256-byte aligned.  The caller synchronises the stream before reading outputs. */
psq_status psq_compute(psq_job* job, unsigned mask, void* d_workspace, size_t ws_bytes,
                       double* d_out[5], void* stream);

/* psq_compute through a CUDA graph: the first call for a (mask, workspace, outputs) triple
 * plans the job, captures its launch sequence on `stream` (which must not be the legacy
 * default stream) and instantiates it; every call then launches that graph.  Graphs are
 * owned by the job and freed with it. */
psq_status psq_compute_graph(psq_job* job, unsigned mask, void* d_workspace, size_t ws_bytes,
                             double* d_out[5], void* stream);

/* psq_compute followed by device-to-host copies of the requested classes into h_out[0..4]
 * (page-locked memory recommended) and a synchronisation of the stream. */
psq_status psq_compute_host(psq_job* job, unsigned mask, void* d_workspace, size_t ws_bytes,
                            double* d_out[5], double* h_out[5], void* stream);

/* Bytes psq_compute copies host-to-device (the job's tables) and psq_compute_host copies
 * device-to-host (the requested matrices) per call. */
psq_status psq_job_io_bytes(const psq_job* job, unsigned mask, size_t* h2d, size_t* d2h);

/* Launch timing.  While enabled, psq_compute records a CUDA event on its stream before each
 * step: 0 table upload, 1 grid + function evaluation, 2 contraction, 3 chunk reduction,
 * 4 assembly (all classes), 5 operand packing (PSQ_MIXED only).  psq_profile_read waits for the recorded events, returns the
 * summed milliseconds and counts per step kind (8 slots) and clears the record. */
psq_status psq_profile_enable(psq_job* job, int on);
psq_status psq_profile_read(psq_job* job, double ms[8], int counts[8]);

/* Allocation-free compute (no counterpart in the paper; a service of this library).
 * Some callers cannot allocate device memory: a host application whose own memory manager
 * owns the GPU's memory and forbids direct cudaMalloc, or a latency-critical loop that must
 * not pay cudaMalloc's device-wide synchronisation.  psq_compute_noalloc runs psq_compute on
 * a scratch array of PSQ_NOALLOC_SCRATCH_BYTES compiled into the library (held by every
 * device that loads it until exit) and allocates nothing: no cudaMalloc or cudaFree, no host
 * allocation, no planning.  The caller still passes the job and the device outputs, and must
 * have planned mask on this job before (psq_job_workspace(job, mask, ...)); otherwise
 * PSQ_ERR_ARG.  A job whose workspace for mask exceeds PSQ_NOALLOC_SCRATCH_BYTES fails with
 * PSQ_ERR_OOM.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture.  Every call, on every stream, shares the one array and leaves its contents for the
 * next: calls whose work overlaps on the GPU race and give undefined results. */
#define PSQ_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
psq_status psq_compute_noalloc(psq_job* job, unsigned mask, double* d_out[5], void* stream);

/* Waits for `stream` and reports whether a kernel of the last psq_compute on this workspace
 * gave up a bounded wait (PSQ_ERR_TIMEOUT); psq_compute_host calls it itself.  d_workspace
 * NULL reads the status of the last psq_compute_noalloc on the current device. */
psq_status psq_check(psq_job* job, unsigned mask, void* d_workspace, void* stream);

/* Failure detection (no paper counterpart): the limit, in nanoseconds, of every bounded wait
 * in the main loops of the tensor-core contraction for this job's later psq_compute calls
 * (default 4e9; 1 <= ns <= 6e10).  A wait that runs out makes the kernel record a status
 * (psq_check then returns PSQ_ERR_TIMEOUT), stop its loops, wait (4 s at most) for its own
 * copies and MMAs in flight, release its tensor memory and return: the context stays usable
 * and the next psq_compute starts afresh.  Graphs captured before keep the limit they were
 * captured with.  Errors: PSQ_ERR_ARG for a NULL job or a limit out of range. */
psq_status psq_job_set_wait_limit(psq_job* job, uint64_t ns);

/* Failure-detection test hook (no paper counterpart): while `on`, every psq_compute of a
 * PSQ_MIXED job raises a flag in its workspace that nothing clears; the contraction's loader
 * waits for it to clear, gives up when the wait limit runs out and the compute ends with
 * PSQ_ERR_TIMEOUT in psq_check, exercising the timeout path without a GPU fault.  Errors:
 * PSQ_ERR_ARG for a NULL job. */
psq_status psq_job_test_stall(psq_job* job, int on);

/* Diagnostics for step-by-step parity tests. */
/* Grid g of the PSQ_ALL plan (0 <= g < n_grids; pair grids (A<B) first, then the refined
 * grids (A<B; C)): its atoms (C = -1 for an unrefined pair grid) and point count. */
psq_status psq_job_grid_info(const psq_job* job, int g, int* A, int* B, int* C, int64_t* n_points);
/* Writes the points of grid g (Section 2.1 eqs 2-6, 10-11; Algorithm 2) into d_out: 8 rows
 * of n_points doubles, x, y, z in the molecule frame, w, r_A, r_B, mu, nu.  Volume elements
 * split around a third centre keep their unsplit points with w = 0; the split sub-cells
 * follow the regular cells.  Uses the first psq_job_workspace(PSQ_ALL) bytes of d_workspace
 * for tables. */
psq_status psq_job_grid_points(psq_job* job, int g, void* d_workspace, size_t ws_bytes,
                               double* d_out, void* stream);
/* Evaluates on grid g: kind 0 = basis chi of the grid's two pair atoms (rows in function
 * order), 1 = their kinetic operand lap chi, 2 = aux chi, 3 = aux potentials V^P (aux of
 * both pair atoms for an unrefined grid, of the third centre for a refined one).  d_out
 * holds rows x n_points doubles; *rows receives the row count.  A PSQ_FP64 job evaluates in
 * FP64; a PSQ_MIXED job runs the mixed path's evaluation (double-float values of x = zeta r
 * and the direction) and returns them times their FP64 row constants. */
psq_status psq_job_grid_functions(psq_job* job, int g, int kind, void* d_workspace,
                                  size_t ws_bytes, double* d_out, int* rows, void* stream);

/* Serving: a request loop for jobs of different sizes arriving over time (continuous
 * batching).  The server owns max_inflight streams and a worker thread; device memory comes
 * from the caller's arena (d_arena, arena_bytes, 256-byte aligned), first-fit.  A submitted
 * job waits until its workspace and outputs fit in the arena and a stream is free; waiting
 * jobs are admitted in submission order, except that a later job that fits runs before an
 * earlier one that does not (backfilling).  Admitted jobs run concurrently, each on its own
 * stream, and their requested matrices are copied into h_out[0..4] (host buffers, page-locked
 * recommended, laid out as psq_compute's outputs).  submit plans the job on the calling
 * thread (psq_job_workspace) and returns a ticket; PSQ_ERR_OOM if the job can never fit.
 * poll reports whether the ticket is done and its latency so far (submit to completion);
 * wait blocks up to timeout_s seconds.  A job's status (e.g. PSQ_ERR_TIMEOUT) is returned by
 * poll/wait once it is done.  A job must not be destroyed while it has unfinished tickets.
 * destroy waits for the running jobs and frees the server's streams. */
typedef struct psq_server psq_server;
psq_status psq_server_create(psq_context* ctx, void* d_arena, size_t arena_bytes, int max_inflight,
                             psq_server** out);
psq_status psq_server_submit(psq_server* server, psq_job* job, unsigned mask, double* h_out[5],
                             uint64_t* ticket);
psq_status psq_server_poll(psq_server* server, uint64_t ticket, int* done, double* latency_s);
psq_status psq_server_wait(psq_server* server, uint64_t ticket, double timeout_s);
psq_status psq_server_destroy(psq_server* server);

/* Thread-local message describing the calling thread's last error. */
const char* psq_last_error(void);

/* RI 4-index assembly (Section 3, eq 14): (ij|kl) ~ sum_PQ (ij|P) [(PQ)^-1] (Q|kl), from the
 * (P|Q) and (P|ij) matrices that psq_compute writes.  With the Cholesky factor (P|Q) = L L^T
 * and B = L^-1 (P|ij), (ij|kl) = sum_R B[R][ij] B[R][kl].  FP64 throughout, on the device,
 * asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream), on the current
 * device.  Matrices are row-major; the pair index of (P|ij) is ij = i * n_bf + j, so its
 * n_aux x n_bf x n_bf layout is B's n x m layout with m = n_bf^2.  The caller owns every
 * buffer.  Errors: PSQ_ERR_ARG for negative sizes, NULL or non-8-byte-aligned pointers with
 * nonzero sizes, or column ranges outside [0, m); PSQ_ERR_CUDA on a failed launch. */

/* Cholesky factor of the symmetric positive definite n x n matrix d_J2 (its lower triangle is
 * read): d_L (n x n; may equal d_J2) receives L, lower triangular, zeros above the diagonal.
 * *d_info (device int) is set to 0, or to k + 1 when the k-th pivot is not positive (the
 * matrix is not positive definite; d_L is then undefined).  Read it after the stream. */
psq_status psq_ri_factor(int n, const double* d_J2, double* d_L, int* d_info, void* stream);

/* Forward substitution in place: d_B (n x m) <- L^-1 d_B, L from psq_ri_factor. */
psq_status psq_ri_solve(int n, int64_t m, const double* d_L, double* d_B, void* stream);

/* A block of 4-index integrals: d_out[c][d] = sum_R B[R][c0 + c] B[R][d0 + d] for
 * 0 <= c < nc, 0 <= d < nd (row-major nc x nd), B (n x m) from psq_ri_solve: with ij = c0 + c
 * and kl = d0 + d, the RI value of (ij|kl). */
psq_status psq_ri_eri(int n, int64_t m, const double* d_B, int64_t c0, int64_t nc, int64_t d0, int64_t nd,
                      double* d_out, void* stream);

/* The same block on the tensor cores (the mixed path's arithmetic, no paper counterpart): each
 * FP64 value of B's pair columns is split into a double-float pair and cut into five 8-bit
 * digits under a power-of-two scale per pair and 128 aux functions, the slice products of
 * orders 0..4 accumulate exactly in FP32 and the aux ranges add in FP64.  Error: each value
 * keeps 39 bits relative to its window's largest, so the block is within about 2^-38 of
 * sum_w n_w M_w(ij) M_w(kl) over the windows w of 128 aux functions (n_w of them), M_w(p) the
 * largest |B[R][p]| in w (the tests assert the looser 2e-9).  d_workspace (256-byte aligned)
 * needs psq_ri_eri_mixed_workspace(n, nc, nd) bytes on the current device; its first int is
 * the contraction's status word (nonzero: a bounded wait expired, d_out undefined).  Errors
 * as psq_ri_eri, and PSQ_ERR_OOM for a smaller workspace, PSQ_ERR_UNSUPPORTED for blocks of
 * more than 2^30 pairs a side. */
psq_status psq_ri_eri_mixed_workspace(int n, int64_t nc, int64_t nd, size_t* bytes);
psq_status psq_ri_eri_mixed(int n, int64_t m, const double* d_B, int64_t c0, int64_t nc, int64_t d0, int64_t nd,
                            double* d_out, void* d_workspace, size_t ws_bytes, void* stream);

/* Peak rates of the current device's arithmetic pipes, measured (no paper counterpart; the
 * denominators of the FP64- and FP32-bound rooflines): independent dependent-FMA chains in
 * FP64 and in FP32 and a chain of the special-function unit's ex2.approx, each launched as 4
 * CTAs x 256 threads per SM, 8 chains per thread, ~30 ms: the fastest of three launches timed
 * by CUDA events on `stream` after a warm-up launch.  Outputs (host doubles; any may be
 * NULL): FP64 and FP32 TFLOP/s (2 FLOPs per FMA), SFU operations in G/s.  Uses no device
 * memory of the caller; synchronises the stream.  Errors: PSQ_ERR_CUDA when there is no
 * device or a launch or event call fails. */
psq_status psq_measure_peaks(void* stream, double* fp64_tflops, double* fp32_tflops, double* sfu_gops);

#ifdef __cplusplus
}
#endif
#endif /* PSQ_H */
