// RI 4-index assembly (Section 3, eq 14): (ij|kl) ~ sum_PQ (ij|P) [(PQ)^-1] (Q|kl).  The metric
// (P|Q) is factored as L L^T (blocked right-looking Cholesky), B = L^-1 (P|ij) by blocked
// forward substitution, and (ij|kl) = sum_R B[R][ij] B[R][kl] by a tiled FP64 product or,
// for large blocks, on the tensor cores through the mixed path's packing and contraction.
// The factor and the solve stay FP64 on the CUDA cores: the metric is ill-conditioned enough
// to need it.  Blocks of 32 rows; every loop bound is a size argument (no waits outside the
// contraction's own bounded ones).
#include "psq_internal.h"

#include <algorithm>
#include <cstdint>

namespace psq {
namespace {

constexpr int kB = 32;  // block size of the factor and the solve

// Factor of the kb x kb diagonal block at (k0, k0), in place in shared memory (one CTA of
// 32 x 32 threads).  A pivot that is not positive records info = k0 + j + 1 (the first one
// wins) and continues with 1 so that nothing divides by zero.
__global__ void __launch_bounds__(1024) chol_diag_kernel(int n, int k0, int kb, double* __restrict__ L,
                                                         int* __restrict__ info) {
  __shared__ double a[kB][kB + 1];
  const int r = threadIdx.x >> 5, c = threadIdx.x & 31;
  if (r < kb && c <= r) a[r][c] = L[(int64_t)(k0 + r) * n + k0 + c];
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    if (threadIdx.x == 0) {
      double d = a[j][j];
      if (!(d > 0.0)) {
        atomicCAS(info, 0, k0 + j + 1);
        d = 1.0;
      }
      a[j][j] = sqrt(d);
    }
    __syncthreads();
    if (c == j && r > j && r < kb) a[r][j] /= a[j][j];
    __syncthreads();
    if (r > j && r < kb && c > j && c <= r) a[r][c] -= a[r][j] * a[c][j];
    __syncthreads();
  }
  if (r < kb && c <= r) L[(int64_t)(k0 + r) * n + k0 + c] = a[r][c];
}

// Panel below the diagonal block: row i >= k0 + kb gets x with x D^T = a (D the factored
// diagonal block), one thread per row.
__global__ void __launch_bounds__(128) chol_panel_kernel(int n, int k0, int kb, double* __restrict__ L) {
  __shared__ double d[kB][kB + 1];
  for (int t = threadIdx.x; t < kB * kB; t += blockDim.x) {
    const int r = t >> 5, c = t & 31;
    d[r][c] = (r < kb && c <= r) ? L[(int64_t)(k0 + r) * n + k0 + c] : 0.0;
  }
  __syncthreads();
  const int i = k0 + kb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double* row = L + (int64_t)i * n + k0;
  double x[kB];
#pragma unroll
  for (int j = 0; j < kB; ++j) {
    if (j < kb) {
      double s = row[j];
#pragma unroll
      for (int m = 0; m < j; ++m) s -= x[m] * d[j][m];
      x[j] = s / d[j][j];
      row[j] = x[j];
    }
  }
}

// Trailing update L[i][j] -= sum_m L[i][k0+m] L[j][k0+m] for k1 = k0 + kb <= j <= i < n, one
// CTA per 32 x 32 tile of the lower triangle (tile t -> (ti, tj), ti >= tj).
__global__ void __launch_bounds__(256) chol_update_kernel(int n, int k0, int kb, double* __restrict__ L) {
  __shared__ double pa[kB][kB + 1], pb[kB][kB + 1];
  const int k1 = k0 + kb;
  const int t = blockIdx.x;
  int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
  while (ti * (ti + 1) / 2 > t) --ti;
  const int tj = t - ti * (ti + 1) / 2;
  const int i0 = k1 + ti * kB, j0 = k1 + tj * kB;
  for (int q = threadIdx.x; q < kB * kB; q += blockDim.x) {
    const int r = q >> 5, m = q & 31;
    pa[r][m] = (i0 + r < n && m < kb) ? L[(int64_t)(i0 + r) * n + k0 + m] : 0.0;
    pb[r][m] = (j0 + r < n && m < kb) ? L[(int64_t)(j0 + r) * n + k0 + m] : 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x & 31, r0 = threadIdx.x >> 5;  // rows r0, r0 + 8, r0 + 16, r0 + 24
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int m = 0; m < kb; ++m) {
    const double b = pb[c][m];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fma(pa[r0 + 8 * q][m], b, acc[q]);
  }
  const int j = j0 + c;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + r0 + 8 * q;
    if (i < n && j < n && j <= i) L[(int64_t)i * n + j] -= acc[q];
  }
}

__global__ void zero_upper_kernel(int n, double* __restrict__ L) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  if (j > i) L[idx] = 0.0;
}

// Forward substitution on the diagonal block: B[k0 + r][col] for r < kb, one thread per
// column.
__global__ void __launch_bounds__(256) trsv_diag_kernel(int n, int64_t m, int k0, int kb,
                                                        const double* __restrict__ L, double* __restrict__ B) {
  __shared__ double d[kB][kB + 1];
  for (int t = threadIdx.x; t < kB * kB; t += blockDim.x) {
    const int r = t >> 5, c = t & 31;
    d[r][c] = (r < kb && c <= r) ? L[(int64_t)(k0 + r) * n + k0 + c] : 0.0;
  }
  __syncthreads();
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= m) return;
  double* b = B + (int64_t)k0 * m + col;
  double x[kB];
#pragma unroll
  for (int j = 0; j < kB; ++j) {
    if (j < kb) {
      double s = b[(int64_t)j * m];
#pragma unroll
      for (int q = 0; q < j; ++q) s -= d[j][q] * x[q];
      x[j] = s / d[j][j];
      b[(int64_t)j * m] = x[j];
    }
  }
}

// B[k1 + r][col] -= sum_q L[k1 + r][k0 + q] B[k0 + q][col]: 64 x 64 tiles, 256 threads with
// 4 x 4 outputs each.
__global__ void __launch_bounds__(256) trsv_update_kernel(int n, int64_t m, int k0, int kb,
                                                          const double* __restrict__ L, double* __restrict__ B) {
  __shared__ double ls[64][kB + 1];
  __shared__ double bs[kB][64];
  const int k1 = k0 + kb;
  const int i0 = k1 + blockIdx.y * 64;
  const int64_t c0 = (int64_t)blockIdx.x * 64;
  for (int t = threadIdx.x; t < 64 * kB; t += blockDim.x) {
    const int r = t / kB, q = t % kB;
    ls[r][q] = (i0 + r < n && q < kb) ? L[(int64_t)(i0 + r) * n + k0 + q] : 0.0;
  }
  for (int t = threadIdx.x; t < kB * 64; t += blockDim.x) {
    const int q = t / 64, c = t % 64;
    bs[q][c] = (q < kb && c0 + c < m) ? B[(int64_t)(k0 + q) * m + c0 + c] : 0.0;
  }
  __syncthreads();
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;  // rows tr + 16a, columns tc + 16b
  double acc[4][4] = {};
  for (int q = 0; q < kb; ++q) {
    double lv[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) lv[a] = ls[tr + 16 * a][q];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = bs[q][tc + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(lv[a], bv[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + tr + 16 * a;
    if (i >= n) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t c = c0 + tc + 16 * b;
      if (c < m) B[(int64_t)i * m + c] -= acc[a][b];
    }
  }
}

// out[c][d] = sum_R B[R][c0 + c] B[R][d0 + d]: 64 x 64 output tiles, R in steps of 16
// through shared memory, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256) eri_kernel(int n, int64_t m, const double* __restrict__ B, int64_t c0,
                                                  int64_t nc, int64_t d0, int64_t nd, double* __restrict__ out) {
  __shared__ double as[16][64];
  __shared__ double bs[16][64];
  const int64_t tc0 = (int64_t)blockIdx.y * 64, td0 = (int64_t)blockIdx.x * 64;
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  double acc[4][4] = {};
  for (int R0 = 0; R0 < n; R0 += 16) {
    for (int t = threadIdx.x; t < 16 * 64; t += blockDim.x) {
      const int q = t / 64, x = t % 64;
      const bool okr = R0 + q < n;
      as[q][x] = (okr && tc0 + x < nc) ? B[(int64_t)(R0 + q) * m + c0 + tc0 + x] : 0.0;
      bs[q][x] = (okr && td0 + x < nd) ? B[(int64_t)(R0 + q) * m + d0 + td0 + x] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = as[q][tr + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = bs[q][tc + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t c = tc0 + tr + 16 * a;
    if (c >= nc) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t d = td0 + tc + 16 * b;
      if (d < nd) out[c * nd + d] = acc[a][b];
    }
  }
}

// ---------------------------------------------------------------- tensor-core product
//
// (ij|kl) = sum_R B[R][ij] B[R][kl] is the contraction of eq 9 with the aux index R in the
// place of the points: the pair columns of B become operand rows (transposed into Bt), are
// packed as in the mixed path (five 8-bit slices per value under a power-of-two scale per
// row and 128 aux functions), and the tcgen05 contraction and its FP64 range reduction run
// unchanged on them (one block, A = the c pairs, B = the d pairs, all row constants 1).

constexpr size_t kAlign = 256;
size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct RiMixedLayout {
  int64_t nc, nd;
  int n, nch, nwin, tmA, tnB, n_ranges, win_per, n_ctas;
  int64_t n_items, jobsA, jobsB;
  size_t o_grid, o_pn, o_blk, o_items, o_cb, o_rows, o_rowc, o_eb, o_status, o_bt, o_pack, o_part, total;
  int64_t packA, expA, packB, expB;  // panel offsets within the packed area
};

RiMixedLayout ri_mixed_layout(int n, int64_t nc, int64_t nd, int sm_count) {
  RiMixedLayout L{};
  L.n = n; L.nc = nc; L.nd = nd;
  L.nch = (n + kChunkPts - 1) / kChunkPts;
  L.nwin = (n + kWinPts - 1) / kWinPts;
  L.tmA = (int)((nc + kMmaM - 1) / kMmaM);
  L.tnB = (int)((nd + kMmaN - 1) / kMmaN);
  const int64_t tiles = (int64_t)L.tmA * L.tnB;
  const int64_t want = 2LL * sm_count;  // at least two items per SM: ranges of aux windows
  int r = tiles >= want ? 1 : (int)std::min<int64_t>(L.nwin, (want + tiles - 1) / tiles);
  L.win_per = (L.nwin + r - 1) / r;
  L.n_ranges = (L.nwin + L.win_per - 1) / L.win_per;
  L.n_items = tiles * L.n_ranges;
  L.n_ctas = (int)std::min<int64_t>(L.n_items, sm_count);
  L.jobsA = (int64_t)L.tmA * L.nwin * (kMmaM / kPackRows);
  L.jobsB = (int64_t)L.tnB * L.nwin * (kMmaN / kPackRows);
  size_t o = 0;
  auto sec = [&](size_t bytes) { const size_t at = o; o = up(o + bytes); return at; };
  L.o_status = sec(sizeof(int));
  L.o_grid = sec(sizeof(DevGrid));
  L.o_pn = sec(2 * sizeof(Panel));
  L.o_blk = sec(sizeof(MmaBlock));
  L.o_items = sec(sizeof(GemmItem) * (size_t)L.n_items);
  L.o_cb = sec(sizeof(int) * (size_t)(L.n_ctas + 1));
  L.o_rows = sec(sizeof(short2) * (size_t)(nc + nd));
  L.o_rowc = sec(sizeof(double));
  L.o_eb = sec(2 * sizeof(int64_t));
  L.o_bt = sec(sizeof(double) * (size_t)(nc + nd) * n);
  size_t pk = 0;
  auto psec = [&](size_t bytes) { const size_t at = pk; pk = up(pk + bytes); return (int64_t)at; };
  L.packA = psec((size_t)nc * L.nch * kSlices * 2 * kChunkPts);
  L.expA = psec((size_t)L.tmA * L.nwin * kMmaM * 4);
  L.packB = psec((size_t)nd * L.nch * kSlices * 2 * kChunkPts);
  L.expB = psec((size_t)L.tnB * L.nwin * kMmaN * 4);
  L.o_pack = sec(pk);
  L.o_part = sec(sizeof(float2) * (size_t)L.n_ranges * nc * nd);
  L.total = o;
  return L;
}

// The tables of the one-block plan, written on the device (nothing to stage on the host, so
// the call can be captured in a CUDA graph).  Items dealt round-robin, stored per CTA.
__global__ void ri_setup_kernel(RiMixedLayout L, char* __restrict__ ws) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *reinterpret_cast<int*>(ws + L.o_status) = 0;
    DevGrid* g = reinterpret_cast<DevGrid*>(ws + L.o_grid);
    g->K = L.n;
    g->rc_off = 0;
    Panel* pn = reinterpret_cast<Panel*>(ws + L.o_pn);
    pn[0].grid = 0; pn[0].rows_off = 0; pn[0].nrows = (int)L.nc; pn[0].tr = kMmaM; pn[0].n_tiles = L.tmA;
    pn[0].nch = L.nch; pn[0].nwin = L.nwin; pn[0].pack_off = L.packA; pn[0].exp_off = L.expA; pn[0].job_begin = 0;
    pn[1].grid = 0; pn[1].rows_off = (int)L.nc; pn[1].nrows = (int)L.nd; pn[1].tr = kMmaN; pn[1].n_tiles = L.tnB;
    pn[1].nch = L.nch; pn[1].nwin = L.nwin; pn[1].pack_off = L.packB; pn[1].exp_off = L.expB; pn[1].job_begin = L.jobsA;
    MmaBlock* b = reinterpret_cast<MmaBlock*>(ws + L.o_blk);
    b->grid = 0; b->m = (int)L.nc; b->n = (int)L.nd; b->a_off = 0; b->b_off = (int)L.nc;
    b->n_ranges = L.n_ranges; b->win_per = L.win_per; b->a_panel = 0; b->b_panel = 1;
    b->ptile_off = 0; b->n_btiles = 0; b->res_off = 0; b->part_off = 0;
    *reinterpret_cast<double*>(ws + L.o_rowc) = 1.0;
    int64_t* eb = reinterpret_cast<int64_t*>(ws + L.o_eb);
    eb[0] = 0;
    eb[1] = L.nc * L.nd;
  }
  const int64_t q = L.n_items / L.n_ctas, rem = L.n_items % L.n_ctas;
  if (i <= L.n_ctas) reinterpret_cast<int*>(ws + L.o_cb)[i] = (int)(i * q + (i < rem ? i : rem));
  if (i < L.n_items) {
    const int64_t tiles = (int64_t)L.tmA * L.tnB;
    const int chunk = (int)(i / tiles), t = (int)(i % tiles);
    const int64_t bcta = i % L.n_ctas, j = i / L.n_ctas;
    const int64_t slot = bcta * q + (bcta < rem ? bcta : rem) + j;
    reinterpret_cast<GemmItem*>(ws + L.o_items)[slot] = GemmItem{0, t / L.tnB, t % L.tnB, chunk};
  }
  if (i < L.nc + L.nd) reinterpret_cast<short2*>(ws + L.o_rows)[i] = make_short2(0, -1);
}

// Bt[r][R] = B[R][col0 + r] for r < count: the pair columns as rows (32 x 32 tiles).
__global__ void ri_transpose_kernel(int n, int64_t m, const double* __restrict__ B, int64_t col0, int64_t count,
                                    double* __restrict__ Bt) {
  __shared__ double tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  const int R0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int R = R0 + k;
    const int64_t c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (R < n && c < count) ? B[(int64_t)R * m + col0 + c] : 0.0;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t c = c0 + k;
    const int R = R0 + threadIdx.x;
    if (c < count && R < n) Bt[c * n + R] = tile[threadIdx.x][k];
  }
}

bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

psq_status launched() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PSQ_OK : set_error(PSQ_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace
}  // namespace psq

using namespace psq;

extern "C" psq_status psq_ri_factor(int n, const double* d_J2, double* d_L, int* d_info, void* stream) {
  if (n < 0) return set_error(PSQ_ERR_ARG, "psq_ri_factor: n < 0");
  if (!d_info || ((uintptr_t)d_info & 3u)) return set_error(PSQ_ERR_ARG, "psq_ri_factor: d_info NULL or misaligned");
  if (n > 0 && (!d_J2 || !d_L || !aligned8(d_J2) || !aligned8(d_L)))
    return set_error(PSQ_ERR_ARG, "psq_ri_factor: NULL or misaligned matrix");
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_info, 0, sizeof(int), s) != cudaSuccess) return launched();
  if (n == 0) return PSQ_OK;
  if (d_L != d_J2 &&
      cudaMemcpyAsync(d_L, d_J2, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return launched();
  for (int k0 = 0; k0 < n; k0 += kB) {
    const int kb = n - k0 < kB ? n - k0 : kB;
    chol_diag_kernel<<<1, 1024, 0, s>>>(n, k0, kb, d_L, d_info);
    const int rest = n - k0 - kb;
    if (rest > 0) {
      chol_panel_kernel<<<(rest + 127) / 128, 128, 0, s>>>(n, k0, kb, d_L);
      const int T = (rest + kB - 1) / kB;
      chol_update_kernel<<<T * (T + 1) / 2, 256, 0, s>>>(n, k0, kb, d_L);
    }
  }
  const int64_t nn = (int64_t)n * n;
  zero_upper_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(n, d_L);
  return launched();
}

extern "C" psq_status psq_ri_solve(int n, int64_t m, const double* d_L, double* d_B, void* stream) {
  if (n < 0 || m < 0) return set_error(PSQ_ERR_ARG, "psq_ri_solve: negative size");
  if (n == 0 || m == 0) return PSQ_OK;
  if (!d_L || !d_B || !aligned8(d_L) || !aligned8(d_B))
    return set_error(PSQ_ERR_ARG, "psq_ri_solve: NULL or misaligned matrix");
  if ((m + 63) / 64 > 0x7fffffff) return set_error(PSQ_ERR_ARG, "psq_ri_solve: m too large");
  cudaStream_t s = (cudaStream_t)stream;
  for (int k0 = 0; k0 < n; k0 += kB) {
    const int kb = n - k0 < kB ? n - k0 : kB;
    trsv_diag_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(n, m, k0, kb, d_L, d_B);
    const int rest = n - k0 - kb;
    if (rest > 0) trsv_update_kernel<<<dim3((unsigned)((m + 63) / 64), (rest + 63) / 64), 256, 0, s>>>(n, m, k0, kb, d_L, d_B);
  }
  return launched();
}

extern "C" psq_status psq_ri_eri(int n, int64_t m, const double* d_B, int64_t c0, int64_t nc, int64_t d0, int64_t nd,
                                 double* d_out, void* stream) {
  if (n < 0 || m < 0 || nc < 0 || nd < 0) return set_error(PSQ_ERR_ARG, "psq_ri_eri: negative size");
  if (c0 < 0 || d0 < 0 || c0 + nc > m || d0 + nd > m) return set_error(PSQ_ERR_ARG, "psq_ri_eri: range outside [0, m)");
  if (nc == 0 || nd == 0) return PSQ_OK;
  if (!d_out || !aligned8(d_out) || (n > 0 && (!d_B || !aligned8(d_B))))
    return set_error(PSQ_ERR_ARG, "psq_ri_eri: NULL or misaligned pointer");
  if ((nc + 63) / 64 > 65535 || (nd + 63) / 64 > 0x7fffffff) return set_error(PSQ_ERR_ARG, "psq_ri_eri: block too large");
  eri_kernel<<<dim3((unsigned)((nd + 63) / 64), (unsigned)((nc + 63) / 64)), 256, 0, (cudaStream_t)stream>>>(
      n, m, d_B, c0, nc, d0, nd, d_out);
  return launched();
}

extern "C" psq_status psq_ri_eri_mixed_workspace(int n, int64_t nc, int64_t nd, size_t* bytes) {
  if (!bytes) return set_error(PSQ_ERR_ARG, "psq_ri_eri_mixed_workspace: bytes is NULL");
  if (n < 0 || nc < 0 || nd < 0) return set_error(PSQ_ERR_ARG, "psq_ri_eri_mixed_workspace: negative size");
  if (nc > (1 << 30) || nd > (1 << 30)) return set_error(PSQ_ERR_UNSUPPORTED, "psq_ri_eri_mixed_workspace: block too large");
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *bytes = ri_mixed_layout(n, nc, nd, sms).total;
  return PSQ_OK;
}

extern "C" psq_status psq_ri_eri_mixed(int n, int64_t m, const double* d_B, int64_t c0, int64_t nc, int64_t d0,
                                       int64_t nd, double* d_out, void* d_workspace, size_t ws_bytes, void* stream) {
  if (n < 0 || m < 0 || nc < 0 || nd < 0) return set_error(PSQ_ERR_ARG, "psq_ri_eri_mixed: negative size");
  if (c0 < 0 || d0 < 0 || c0 + nc > m || d0 + nd > m)
    return set_error(PSQ_ERR_ARG, "psq_ri_eri_mixed: range outside [0, m)");
  if (nc == 0 || nd == 0) return PSQ_OK;
  if (!d_out || !aligned8(d_out) || (n > 0 && (!d_B || !aligned8(d_B))))
    return set_error(PSQ_ERR_ARG, "psq_ri_eri_mixed: NULL or misaligned pointer");
  if (!d_workspace || (uintptr_t)d_workspace % kAlign)
    return set_error(PSQ_ERR_ARG, "psq_ri_eri_mixed: workspace NULL or not 256-byte aligned");
  if (nc > (1 << 30) || nd > (1 << 30)) return set_error(PSQ_ERR_UNSUPPORTED, "psq_ri_eri_mixed: block too large");
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    if (cudaMemsetAsync(d_out, 0, sizeof(double) * (size_t)nc * nd, s) != cudaSuccess) return launched();
    return PSQ_OK;
  }
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return launched();
  const RiMixedLayout L = ri_mixed_layout(n, nc, nd, sms);
  if (ws_bytes < L.total) return set_error(PSQ_ERR_OOM, "psq_ri_eri_mixed: workspace too small");
  if (prepare_kernels() != cudaSuccess) return launched();
  char* ws = (char*)d_workspace;
  if (cudaMemsetAsync(ws, 0, L.o_bt, s) != cudaSuccess) return launched();  // tables (zeroed, then set)
  const int64_t setup_n = std::max<int64_t>(std::max<int64_t>(L.n_items, nc + nd), L.n_ctas + 1);
  ri_setup_kernel<<<(unsigned)((setup_n + 255) / 256), 256, 0, s>>>(L, ws);
  double* btA = (double*)(ws + L.o_bt);
  double* btB = btA + (size_t)nc * n;
  ri_transpose_kernel<<<dim3((unsigned)((nc + 31) / 32), (n + 31) / 32), dim3(32, 8), 0, s>>>(n, m, d_B, c0, nc, btA);
  ri_transpose_kernel<<<dim3((unsigned)((nd + 31) / 32), (n + 31) / 32), dim3(32, 8), 0, s>>>(n, m, d_B, d0, nd, btB);
  uint8_t* packed = (uint8_t*)(ws + L.o_pack);
  const Panel* pn = (const Panel*)(ws + L.o_pn);
  if (launch_ri_pack(pn, L.jobsA + L.jobsB, btA, btB, n, packed, s) != cudaSuccess) return launched();
  if (launch_contract_ws((const DevGrid*)(ws + L.o_grid), (const MmaBlock*)(ws + L.o_blk),
                         (const GemmItem*)(ws + L.o_items), (const int*)(ws + L.o_cb), L.n_ctas, pn, nullptr, nullptr,
                         nullptr, packed, (float2*)(ws + L.o_part), (int*)(ws + L.o_status), 4000000000ull,
                         nullptr, s) != cudaSuccess)
    return launched();
  if (launch_reduce_mixed((const DevGrid*)(ws + L.o_grid), (const MmaBlock*)(ws + L.o_blk), 1,
                          (const int64_t*)(ws + L.o_eb), 0, nc * nd, (const short2*)(ws + L.o_rows),
                          (const double*)(ws + L.o_rowc), (const float2*)(ws + L.o_part), d_out, s) != cudaSuccess)
    return launched();
  return launched();
}
