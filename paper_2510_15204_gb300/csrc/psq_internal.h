// Internal structures shared by the host planner (psq_host.cpp) and the CUDA kernels
// (psq_kernels.cu, psq_mma.cu).  Everything here is plain data laid out for one H2D copy.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/psq.h"

namespace psq {

constexpr int kMaxL = 6;    // highest angular momentum of a basis or aux shell
constexpr int kMaxN = 12;   // highest principal quantum number
constexpr int kMaxQ = 16;   // Gauss-Legendre points per dimension

// One shell of STO or aux functions (eq 1), with its radial normalisation.
struct DevShell {
  int n, l, atom, fn0;   // fn0: first function index of the shell within its atom
  double zeta, norm;     // norm = (2 zeta)^(n+1/2) / sqrt((2n)!)
};

// One PS grid: a pair (A, B) with A at (0,0,+a) of its own frame, optionally refined around
// a third centre C (Section 2.2).  Points are numbered: regular cells (i, j, k) x Q^3 nodes,
// where cells touching C carry zero weight, then the N_SP^3 sub-cells of each touching cell.
struct DevGrid {
  double M[3];      // midpoint of A and B (molecule frame)
  double R[9];      // rotation pair frame -> molecule frame, R[i*3+j] = axis j, component i
  double RC[3];     // third-centre position (molecule frame), refined grids only
  double a;         // half the A-B distance
  int A, B, C;      // atoms; C = -1 for an unrefined grid
  int n_mu, n_nu, n_phi, q_mu, q_nu, q_phi, n_sp;
  int edge_off;     // edges: mu[n_mu+1], nu[n_nu+1], phi[n_phi+1] from this offset
  int t_mu0, t_mu1, t_nu0, t_nu1, t_phi_all, n_touch;  // cells touching C (n_touch = 0: none)
  int64_t K, K_reg; // points; points of the regular cell block
  // Operand matrices of this grid: rows of ld doubles (or floats) from op_off.
  int64_t op_off;
  int64_t ld;
  int row_F, row_L, row_G, row_U, row_W;  // first row per kind, -1 when absent
  int nFA, nFB;     // basis functions of A and of B (rows of F/L: A's then B's)
  int nG;           // aux rows in G/U (A's then B's on an unrefined grid, C's on a refined one)
  int shb_A0, shb_A1, shb_B0, shb_B1;     // basis shell ranges of A and B
  int sha_0, sha_1, sha_2, sha_3;         // aux shells: [0,1) first centre, [2,3) second
  int aux_c0, aux_c1;                     // atoms of the two aux ranges (-1 none)
  // mixed path: 1-D node tables (rows: the N volume-element rows, then N_SP sub-rows of each
  // touching row), and the third centre's pair-frame coordinates (xc, 0, zc)
  int nt_off, nt_mu, nt_nu, nt_phi;
  double xc, zc;
  float Rh[9], Rl[9];  // R as an FP32 pair
  int xi_off;          // FP32 (hi, lo) x-scales of the shells: basis A, basis B, aux c0, aux c1
  int rc_off;          // FP64 constant of every operand row (norms, zeta powers, a^3 ...)
};

// One Gauss-Legendre node of one dimension of one grid row: the coordinate v and its
// sine/cosine (sinh/cosh for mu) in FP64 (third-centre offsets), and as double-float (hi, lo)
// pairs the sine/cosine, sin^2(v/2) (sinh^2 for mu), cos^2(v/2) and the 1-D weight.
struct NodeEntry {
  double v, s, c;
  float2 fs, fc, fh2, fg2, fw;
};

// A contraction block of the tensor-core path: R[r][c] = sum_p A_r(p) B_c(p), row-major
// m x n, where every operand row is one of the grid's operand rows times an optional second
// one: A_r = src[a.x] * src[a.y] (a = rows[a_off + r], y = -1: no factor), B_c likewise from
// rows[b_off + c].  A always comes from a packed panel (a_panel); B from a packed panel
// (b_panel >= 0) or, for the 3-index operand chi_i chi_j, is formed in shared memory from
// the staged basis rows of the pair tiles [ptile_off, ptile_off + n_btiles).
struct MmaBlock {
  int grid;
  int m, n;
  int a_off, b_off;
  int n_ranges, win_per;  // point range split into n_ranges of win_per 128-point windows
  int a_panel, b_panel;
  int ptile_off, n_btiles;
  int64_t res_off, part_off;
};

// Tensor-core tiling of the mixed path (shared by the planner and the kernels).
constexpr int kMmaM = 128;     // tile rows
constexpr int kMmaN = 48;      // tile columns: 5 orders x 48 columns x 2 accumulator sets fill 480 of
                               // the 512 TMEM columns
constexpr int kChunkPts = 32;  // points per shared-memory stage (one 64-byte row of BF16 digits)
constexpr int kWinPts = 128;   // points per scale window (the exact FP32 accumulation bound)
constexpr int kSlices = 5;     // 8-bit integer slices per operand value; orders 0..4 are kept
constexpr int kPackRows = 16;  // operand rows per packing job

// A packed operand panel: nrows operand rows (rows[rows_off ...]) of one grid in tiles of tr
// rows (kMmaM for the A side of a tile, kMmaN for B); tile t holds rt = min(tr, nrows - t*tr)
// rows.  Every value is split into kSlices BF16 planes of 8-bit integers under a power-of-two
// scale per row and kWinPts-point window (exponent e: value = 2^(e-7) (s0 + s1/256 + ... +
// s4/256^4)).  The planes of tile t, 32-point chunk c start at pack_off + t*nch*5*tr*64 +
// c*5*rt*64 bytes, plane k rt*64 bytes after plane k-1, each exactly as the tcgen05
// shared-memory operand wants it: 64-byte rows (32 points), the four 16-byte groups of row r
// XOR-swizzled by (r / 2) % 4 (the 64-byte swizzle).  Rows past rt are not stored (their
// products only reach result rows or columns that are never read).  The exponents of tile t,
// window w are tr ints at exp_off + (t*nwin + w)*tr*4 bytes; a zero row (or padding row) has
// exponent kZeroExp.
struct Panel {
  int grid;
  int rows_off, nrows;
  int tr, n_tiles;
  int nch, nwin;
  int64_t pack_off, exp_off;
  int64_t job_begin;  // first packing job (tile, window, 16-row group) of this panel, prefix over panels
};
constexpr int kZeroExp = -100000;
constexpr int kPackHintJobs = 256;  // packing jobs per entry of a wave's panel hint table

// The formed B operand of one tile of a 3-index block: column c (< kMmaN) is the product of
// the staged basis rows dx[c] and dy[c] (indices into rows[], grid operand rows) and lands
// in column col[c] of the block's result.
constexpr int kPairTileRows = 16;
struct PairTile {
  int ncols, nrows;
  short rows[kPairTileRows];
  unsigned char dx[kMmaN], dy[kMmaN];
  int col[kMmaN];
};

// One output block of a contraction (eq 9): out[r][c] = sum_p A_r(p) d(p) B_c(p), where
// B_c is a row of the grid's operands (b_mode 0) or the product of two basis rows (b_mode 1,
// the 3-index operand chi_i chi_j of eq 16).
struct GemmBlock {
  int grid;
  int a_row, m;
  int b_row, n;
  int b_mode;
  int pair_off;     // into the pair table (b_mode 1): pairs of F rows
  int d_row;        // weight row (w, w/r_A, w/r_B or w/r_C)
  int n_chunks;     // point range split into n_chunks partial sums
  int tile_m, tile_n;  // output tile of one CTA (tile_m <= kFpTileRows, tile_n <= kFpTileCols, <= 1024 outputs)
  int64_t res_off;  // m x n FP64 result
  int64_t part_off; // n_chunks x m x n FP64 partial sums
};
constexpr int kFpTileRows = 64, kFpTileCols = 256, kFpTileOut = 1024;

struct GemmItem { int block, tm, tn, chunk; };

// Assembly sources (Section 4: each element from exactly one grid, V_ne summed over nuclei).
// Two-index element (a on X, b on Y, local indices la, lb) from block M = res + off:
//   mode 0: M[(rX+la)*ld + cY+lb], averaged with its mirror M2[(rY+lb)*ld2 + cX+la] where the
//           class is symmetrised (M2 = res + off2 with leading dimension ld2 when ld2 > 0,
//           else M and ld: the mirror in the same block);
//   mode 1: M[p*ld + cX*cs], p = packed index of the local pair (rX+la, cY+lb) over nloc;
//   mode 2: M[p*ld + cX*cs], p = la*nloc + lb (a rectangular pair list).
struct SrcEntry {
  int64_t off;
  int ld, rX, cY, rY, cX, mode, nloc, cs;
  double z;
  int64_t off2;
  int ld2;
};
// Three-index element (P on X, i on Y, j on W; Y <= W): res[off + p*s_pair + lP*s_aux] with
// p the packed (mode 1) index of (offY+li, offW+lj) over nloc or (mode 0) (offY+li)*nloc +
// offW+lj.
struct J3Src { int64_t off; int s_pair, s_aux, mode, nloc, offY, offW; };

struct PointBlock { int grid; int pad; int64_t p0; };  // evaluation: 128 points (one window) of one grid

}  // namespace psq

// Launchers (psq_kernels.cu).  Each returns the cudaError_t of its launch.
namespace psq {
struct LaunchTables {
  const DevGrid* grids;
  const double* edges;
  const DevShell* bshell;
  const DevShell* ashell;
  const double* atom_xyz;     // 3 * n_atoms
  const PointBlock* pblocks;
  int n_pblocks;
  const GemmBlock* gblocks;
  int n_gblocks;
  const GemmItem* items;
  int n_items;
  const short2* pairs;
  const int64_t* elem_begin;  // prefix sums of m*n over blocks (n_gblocks + 1)
  int64_t n_elems;
};
void upload_gl_tables(const double* x, const double* w, const double* klm);  // host constants
cudaError_t launch_eval_fp64(const LaunchTables& t, double* ops, int kinds, cudaStream_t s);
cudaError_t launch_contract_fp64(const LaunchTables& t, const double* ops, double* part, cudaStream_t s);
cudaError_t launch_reduce(const LaunchTables& t, const double* part, double* res, cudaStream_t s);
// shells / fn_shell (S and T only, else NULL): the basis shells and each function's shell,
// for the one-centre elements, which take their closed forms.
cudaError_t launch_assemble(int cls, int n_atoms, int nfn, int naux, const int* fn_atom,
                            const int* fn_local, const int* aux_atom, const int* aux_local,
                            const SrcEntry* src, const int* src_ptr, const J3Src* j3,
                            const DevShell* shells, const int* fn_shell, const double* res, double* out,
                            cudaStream_t s);
cudaError_t launch_grid_points(const LaunchTables& t, int g, double* out, cudaStream_t s);
void upload_mixed_tables(const double* x, const double* w, const double* klm);
cudaError_t launch_nodes(const DevGrid* grids, int n_grids, int max_entries, const double* edges, NodeEntry* tab,
                         cudaStream_t s);
cudaError_t launch_eval_mixed(const LaunchTables& t, const NodeEntry* tab, const float2* xi, float* ops,
                              float* ops_lo, cudaStream_t s);
cudaError_t launch_combine_rows(const float* h, const float* l, const double* rc, int nrows, int64_t K, int64_t ld,
                                double* out, cudaStream_t s);
size_t ws_smem_bytes();
cudaError_t prepare_kernels();  // per-device kernel attributes (context creation)
// hint: per block of kPackHintJobs jobs (numbered from 0 in panels[0]), the index of the panel
// holding the block's first job (or NULL: bisection).
cudaError_t launch_pack(const DevGrid* grids, const Panel* panels, int n_panels, const int* hint, int64_t n_jobs,
                        const short2* rows, const float* ops, const float* ops_lo, uint8_t* packed, cudaStream_t s);
// Packed panels of the RI 4-index product from FP64 rows (panels[0] from srcA, panels[1] from
// srcB, rows of n values); n_jobs covers both panels' packing jobs.
cudaError_t launch_ri_pack(const Panel* panels, int64_t n_jobs, const double* srcA, const double* srcB, int n,
                           uint8_t* packed, cudaStream_t s);
// CTA b of the persistent contraction works through items [cta_begin[b], cta_begin[b + 1]).
// wait_ns bounds every wait of the main loops (the drains after a timeout keep a fixed 4 s);
// hold (may be NULL): a device word that, while nonzero, holds the loader back (the
// failure-detection test raises it and nothing clears it).
cudaError_t launch_contract_ws(const DevGrid* grids, const MmaBlock* blocks, const GemmItem* items,
                               const int* cta_begin, int n_ctas, const Panel* panels, const PairTile* ptiles,
                               const float* ops, const float* ops_lo, const uint8_t* packed, float2* part, int* status,
                               uint64_t wait_ns, const int* hold, cudaStream_t s);
// Reduces the elements [e0, e1) of the blocks (prefix sums elem_begin).
cudaError_t launch_reduce_mixed(const DevGrid* grids, const MmaBlock* blocks, int n_blocks, const int64_t* elem_begin,
                                int64_t e0, int64_t e1, const short2* rows, const double* rowc, const float2* part,
                                double* res, cudaStream_t s);

// Host side (psq_host.cpp): psq_compute on a given workspace; with plan_must_exist the call
// plans nothing (no host or device allocation) and fails if mask was never planned.
psq_status compute_on(psq_job* job, unsigned mask, void* d_workspace, size_t ws_bytes, double* d_out[5],
                      void* stream, bool plan_must_exist);
psq_status set_error(psq_status s, const char* msg);
int context_device(const psq_context* ctx);           // -1 for a planning-only context
int job_device(const psq_job* job);                   // the device of the job's context
// Device address of the allocation-free entry point's scratch on the current device (looked
// up once per device).
psq_status noalloc_scratch(void** ptr);
size_t status_offset(psq_job* job, unsigned mask);     // workspace offset of the status word
}  // namespace psq
