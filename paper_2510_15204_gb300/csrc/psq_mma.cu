// Mixed-precision path of the PS quadrature on sm_103a:
//  * node tables: the PS grid is a tensor product in (mu, nu, phi) per volume element, so the
//    per-node trigonometric factors (Section 2.1, eqs 2-6, 10-11) are computed once per grid
//    row in FP64 (nodes_kernel) and stored with double-float (FP32 hi + lo) copies;
//  * eval_mixed_kernel: point weights, focal distances and offsets in double-float from the
//    node tables (the cancellation-free forms), the third-centre offset in FP64 (it cancels
//    near that centre), STOs (eq 1), their kinetic operand and the aux potentials (eq 16,
//    incomplete gamma by its positive series below x = k) as double-float functions of
//    x = zeta r and the direction (psq_df.cuh); every constant factor of a row is left to FP64;
//  * pack_kernel: every operand row that a contraction tile reads whole is scaled by a power
//    of two per 128-point window (from the window's maximum) and cut into five integer slices
//    of at most 8 bits (exact in BF16; 39 bits of the window's largest value), stored as the
//    tcgen05 shared-memory image (64-byte rows of 32 points, 64-byte swizzle);
//  * contract_ws_kernel: the weighted contraction of eq 9 on tcgen05 tensor cores.  Packed
//    tiles arrive by bulk copies; the 3-index operand chi_i chi_j is formed (double-float
//    products) and sliced in shared memory from staged basis rows.  Per K step of 16 points
//    five MMAs (A slice i against B slices 0..4-i, contiguous in shared memory) accumulate
//    the slice products of orders 0..4 into five FP32 TMEM accumulators; all partial sums are
//    integers below 2^24, so the FP32 accumulation is exact.  After each window the
//    accumulators are scaled back and added into double-float registers; each work item
//    writes its point range's (hi, lo) sums, and reduce_mixed_kernel adds the ranges in FP64
//    and applies the FP64 constants of each row and column (normalisations, powers of zeta,
//    a^3), which the values omit.
#include "psq_internal.h"
#include "psq_df.cuh"

#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

namespace psq {

// ------------------------------------------------------------------ node tables

__constant__ double c_glx2[kMaxQ + 1][kMaxQ];
__constant__ double c_glw2[kMaxQ + 1][kMaxQ];
__constant__ float c_rcpf[128];           // 1/n (FP32 tails of the incomplete-gamma series)
__constant__ float2 c_factd[2 * kMaxN + 4];  // k! as (hi, lo)
__constant__ float2 c_exp_tab[64];        // 2^(-j/64) as (hi, lo)
__constant__ dfa::ExpConsts c_expc;

__host__ __device__ __forceinline__ float2 split_f(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

void upload_mixed_tables(const double* x, const double* w, const double* klm) {
  (void)klm;
  cudaMemcpyToSymbol(c_glx2, x, sizeof(double) * (kMaxQ + 1) * kMaxQ);
  cudaMemcpyToSymbol(c_glw2, w, sizeof(double) * (kMaxQ + 1) * kMaxQ);
  float2 f[2 * kMaxN + 4];
  double fd = 1.0;
  f[0] = split_f(1.0);
  for (int i = 1; i < 2 * kMaxN + 4; ++i) {
    fd *= i;
    f[i] = split_f(fd);
  }
  cudaMemcpyToSymbol(c_factd, f, sizeof(f));
  float r[128];
  r[0] = 0.0f;
  for (int i = 1; i < 128; ++i) r[i] = (float)(1.0 / i);
  cudaMemcpyToSymbol(c_rcpf, r, sizeof(r));
  float2 t[64];
  for (int j = 0; j < 64; ++j) t[j] = split_f(std::exp2(-j / 64.0));
  cudaMemcpyToSymbol(c_exp_tab, t, sizeof(t));
  // ln2/64 = c1 + c2 + c3, c1 rounded to 10 significant bits
  const double l64 = 0.693147180559945309417232121458 / 64.0;
  int e2 = 0;
  std::frexp(l64, &e2);
  const double c1 = std::ldexp(std::nearbyint(std::ldexp(l64, 10 - e2)), e2 - 10);
  const float c2 = (float)(l64 - c1);
  const float c3 = (float)(l64 - c1 - (double)c2);
  dfa::ExpConsts ec{(float)(64.0 / 0.693147180559945309417232121458), (float)c1, c2, c3};
  cudaMemcpyToSymbol(c_expc, &ec, sizeof(ec));
}

// Entry (row, node) of one dimension: rows 0..N-1 are the volume-element rows, then
// N_SP sub-rows of each touching row.  dim 0 = mu, 1 = nu, 2 = phi.
__global__ void nodes_kernel(const DevGrid* __restrict__ grids, const double* __restrict__ edges,
                             NodeEntry* __restrict__ tab) {
  const DevGrid& g = grids[blockIdx.y];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int nmu = (g.n_mu + g.nt_mu * g.n_sp) * g.q_mu;
  const int nnu = (g.n_nu + g.nt_nu * g.n_sp) * g.q_nu;
  const int nph = (g.n_phi + g.nt_phi * g.n_sp) * g.q_phi;
  if (e >= nmu + nnu + nph) return;
  int dim, idx, N, Q, t0;
  const double* ed = edges + g.edge_off;
  if (e < nmu) {
    dim = 0; idx = e; N = g.n_mu; Q = g.q_mu; t0 = g.t_mu0;
  } else if (e < nmu + nnu) {
    dim = 1; idx = e - nmu; N = g.n_nu; Q = g.q_nu; t0 = g.t_nu0; ed += g.n_mu + 1;
  } else {
    dim = 2; idx = e - nmu - nnu; N = g.n_phi; Q = g.q_phi; t0 = 0; ed += g.n_mu + 1 + g.n_nu + 1;
  }
  const int row = idx / Q, q = idx % Q;
  double m0, m1;
  if (row < N) {
    m0 = ed[row];
    m1 = ed[row + 1];
  } else {
    const int t = (row - N) / g.n_sp, s = (row - N) % g.n_sp;
    int base;
    if (dim < 2) base = t0 + t;
    else base = g.t_phi_all ? t : (t == 0 ? 0 : g.n_phi - 1);
    const double M0 = ed[base], M1 = ed[base + 1];
    const int ns = g.n_sp;
    m0 = M0 + (M1 - M0) * s / ns;
    m1 = M0 + (M1 - M0) * (s + 1) / ns;
  }
  const double h = 0.5 * (m1 - m0);
  const double v = 0.5 * (m0 + m1) + h * c_glx2[Q][q];
  double s, c, h2, g2;
  if (dim == 0) {
    s = sinh(v);
    c = cosh(v);
    const double sh2 = sinh(0.5 * v);
    h2 = sh2 * sh2;
    g2 = 0.0;
  } else {
    sincos(v, &s, &c);
    double s2, c2;
    sincos(0.5 * v, &s2, &c2);
    h2 = s2 * s2;
    g2 = c2 * c2;
  }
  NodeEntry o;
  o.v = v;
  o.s = s;
  o.c = c;
  o.fs = split_f(s);
  o.fc = split_f(c);
  o.fh2 = split_f(h2);
  o.fg2 = split_f(g2);
  o.fw = split_f(h * c_glw2[Q][q]);
  tab[g.nt_off + e] = o;
}

// ------------------------------------------------------------------ mixed evaluation
//
// Every value is a double-float (hi, lo) pair (about 48 bits): the slices the contraction
// keeps reach 39 bits of each 128-point window's largest value, so the function values must
// carry more than that.

using dfa::df;

__device__ __forceinline__ df ld2(float2 v) { return df{v.x, v.y}; }

// Rows of the shells [s0, s1) of one centre for one or two row kinds (chi with lap chi, or
// chi with V^P: x, e^-x and 1/x are shared).  xi[k] is the (hi, lo) scale that turns rho into
// x for shell s0 + k.  Values go to the hi and lo planes.
__device__ __forceinline__ void eval_shells_df(const DevShell* __restrict__ sh, const float2* __restrict__ xi,
                                               int s0, int s1, df rho, const df* Y, float* __restrict__ oh,
                                               float* __restrict__ ol, int64_t ld, int64_t p, int row_a,
                                               int kind_a, int row_b, int kind_b, const float2* etab) {
#pragma unroll 1  // one shell at a time: unrolled copies only grow the code
  for (int s = s0; s < s1; ++s) {
    const DevShell q = sh[s];
    const df x = dfa::mul(ld2(xi[s - s0]), rho);
    const df ex = dfa::exp_neg(x, c_expc, etab);
    const df ix = (kind_a != 0 || (row_b >= 0 && kind_b != 0)) ? dfa::rcp(x) : dfa::mk(0.0f);
    const int base = q.l * q.l + q.l;
    if (row_a >= 0) {
      const df ra = dfa::radial(kind_a, q.n, q.l, x, ex, ix, c_factd, c_rcpf);
#pragma unroll 1
      for (int m = -q.l; m <= q.l; ++m) {
        const df v = dfa::mul(ra, Y[base + m]);
        const int64_t o = (int64_t)(row_a + q.fn0 + q.l + m) * ld + p;
        oh[o] = v.h;
        ol[o] = v.l;
      }
    }
    if (row_b >= 0) {
      const df rb = dfa::radial(kind_b, q.n, q.l, x, ex, ix, c_factd, c_rcpf);
#pragma unroll 1
      for (int m = -q.l; m <= q.l; ++m) {
        const df v = dfa::mul(rb, Y[base + m]);
        const int64_t o = (int64_t)(row_b + q.fn0 + q.l + m) * ld + p;
        oh[o] = v.h;
        ol[o] = v.l;
      }
    }
  }
}

__device__ __forceinline__ int shells_lmax_f(const DevShell* sh, int s0, int s1) {
  int l = 0;
  for (int s = s0; s < s1; ++s) l = max(l, sh[s].l);
  return l;
}

// u = R v / len (R as a double-float matrix), the unit vector of the offset v of length len.
__device__ __forceinline__ void rotate_unit_df(const DevGrid& g, df vx, df vy, df vz, df inv_len, df* u) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const df r0{g.Rh[c * 3], g.Rl[c * 3]}, r1{g.Rh[c * 3 + 1], g.Rl[c * 3 + 1]}, r2{g.Rh[c * 3 + 2], g.Rl[c * 3 + 2]};
    const df d = dfa::add(dfa::add(dfa::mul(r0, vx), dfa::mul(r1, vy)), dfa::mul(r2, vz));
    u[c] = dfa::mul(d, inv_len);
  }
}

__device__ __forceinline__ df split_d(double v) {
  const float hi = (float)v;
  return df{hi, (float)(v - (double)hi)};
}

// One thread per point.  The weight w = a^3 [G G G sinh mu sin nu (sinh^2 mu + sin^2 nu)]
// and r_A = 2a rho_A, r_B = 2a rho_B are written without their per-grid constants (a^3,
// a^2/2), which are applied in FP64 after the contraction; functions likewise.  The offsets
// from A and B (in units of a) are (sinh mu sin nu cos phi, sinh mu sin nu sin phi,
// 2(sinh^2(mu/2) cos nu -+ {sin^2, cos^2}(nu/2))), of length 2 rho; the offset from a third
// centre is formed in FP64 (it cancels near that centre).
__global__ void __launch_bounds__(128) eval_mixed_kernel(LaunchTables t, const NodeEntry* __restrict__ tab,
                                                         const float2* __restrict__ xi_tab,
                                                         float* __restrict__ ops, float* __restrict__ ops_lo) {
  __shared__ float2 etab[64];
  if (threadIdx.x < 64) etab[threadIdx.x] = c_exp_tab[threadIdx.x];
  __syncthreads();
  const PointBlock pb = t.pblocks[blockIdx.x];
  const DevGrid& g = t.grids[pb.grid];
  const int p = (int)pb.p0 + (int)threadIdx.x;  // K < 2^31 - 256 (the planner checks)
  if (p >= g.K) return;
  const int q3 = g.q_mu * g.q_nu * g.q_phi;
  int ri, rj, rk;
  bool dead = false;
  int pr;
  if (p < g.K_reg) {
    const int cell = p / q3;
    pr = p - cell * q3;
    const int cnp = cell / g.n_phi;
    rk = cell - cnp * g.n_phi;
    ri = cnp / g.n_nu;
    rj = cnp - ri * g.n_nu;
    if (g.n_touch > 0 && ri >= g.t_mu0 && ri <= g.t_mu1 && rj >= g.t_nu0 && rj <= g.t_nu1 &&
        (g.t_phi_all || rk == 0 || rk == g.n_phi - 1))
      dead = true;
  } else {
    const int pe = p - (int)g.K_reg;
    const int s = pe / q3;
    pr = pe - s * q3;
    const int ns = g.n_sp, ns3 = ns * ns * ns;
    const int tc = s / ns3, sub = s - tc * ns3;
    const int ntp = g.nt_phi, nnu = g.nt_nu;
    const int ti = tc / (nnu * ntp), tj = (tc / ntp) % nnu, tk = tc % ntp;
    const int si = sub / (ns * ns), sj = (sub / ns) % ns, sk = sub % ns;
    ri = g.n_mu + ti * ns + si;
    rj = g.n_nu + tj * ns + sj;
    rk = g.n_phi + tk * ns + sk;
  }
  const int qnp = pr / g.q_phi;
  const int qk = pr - qnp * g.q_phi;
  const int qi = qnp / g.q_nu;
  const int qj = qnp - qi * g.q_nu;
  const int nmu = (g.n_mu + g.nt_mu * g.n_sp) * g.q_mu;
  const int nnu = (g.n_nu + g.nt_nu * g.n_sp) * g.q_nu;
  const NodeEntry& Mu = tab[g.nt_off + ri * g.q_mu + qi];
  const NodeEntry& Nu = tab[g.nt_off + nmu + rj * g.q_nu + qj];
  const NodeEntry& Ph = tab[g.nt_off + nmu + nnu + rk * g.q_phi + qk];
  const df sh = ld2(Mu.fs), s2m = ld2(Mu.fh2);
  const df sn = ld2(Nu.fs), cs = ld2(Nu.fc), s2n = ld2(Nu.fh2), c2n = ld2(Nu.fg2);
  const df sp = ld2(Ph.fs), cp = ld2(Ph.fc);
  const df shsn = dfa::mul(sh, sn);
  df w = dfa::mk(0.0f);
  if (!dead) {
    const df gw = dfa::mul(dfa::mul(ld2(Mu.fw), ld2(Nu.fw)), ld2(Ph.fw));
    w = dfa::mul(dfa::mul(gw, shsn), dfa::add_same(dfa::mul(sh, sh), dfa::mul(sn, sn)));
  }
  const df rhoA = dfa::add_same(s2m, s2n), rhoB = dfa::add_same(s2m, c2n);
  const df xs = dfa::mul(shsn, cp), ys = dfa::mul(shsn, sp);
  const df s2mc = dfa::mul(s2m, cs);
  df uA[3], uB[3], uC[3] = {dfa::mk(0.f), dfa::mk(0.f), dfa::mk(1.f)};
  rotate_unit_df(g, xs, ys, dfa::scale2(dfa::sub(s2mc, s2n), 2.0f), dfa::rcp(dfa::scale2(rhoA, 2.0f)), uA);
  rotate_unit_df(g, xs, ys, dfa::scale2(dfa::add(s2mc, c2n), 2.0f), dfa::rcp(dfa::scale2(rhoB, 2.0f)), uB);
  df rC = dfa::mk(1.0f);
  if (g.C >= 0) {
    // offset from the third centre in the pair frame, FP64: it cancels near that centre
    const double X = g.a * Mu.s * Nu.s * Ph.c - g.xc;
    const double Yv = g.a * Mu.s * Nu.s * Ph.s;
    const double Z = g.a * Mu.c * Nu.c - g.zc;
    const df dX = split_d(X), dY = split_d(Yv), dZ = split_d(Z);
    rC = dfa::sqrt(dfa::add_same(dfa::add_same(dfa::mul(dX, dX), dfa::mul(dY, dY)), dfa::mul(dZ, dZ)));
    rotate_unit_df(g, dX, dY, dZ, dfa::rcp(rC), uC);
  }
  float* bh = ops + g.op_off;
  float* bl = ops_lo + g.op_off;
  const int64_t ld = g.ld;
  if (g.row_W >= 0) {
    const df wv[4] = {w, dfa::div(w, rhoA), dfa::div(w, rhoB), g.C >= 0 ? dfa::div(w, rC) : dfa::mk(0.0f)};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      bh[(int64_t)(g.row_W + k) * ld + p] = wv[k].h;
      bl[(int64_t)(g.row_W + k) * ld + p] = wv[k].l;
    }
  }
  const float2* xi = xi_tab + g.xi_off;  // basis A, basis B, aux c0, aux c1 shells
  const int nbA = g.shb_A1 - g.shb_A0, nbB = g.shb_B1 - g.shb_B0, na0 = g.sha_1 - g.sha_0;
  df Y[(kMaxL + 1) * (kMaxL + 1)];
  if (g.row_F >= 0 || g.row_L >= 0) {
    for (int c = 0; c < 2; ++c) {
      const int s0 = c == 0 ? g.shb_A0 : g.shb_B0, s1 = c == 0 ? g.shb_A1 : g.shb_B1;
      if (s1 <= s0) continue;
      const df* u = c == 0 ? uA : uB;
      dfa::real_ylm(shells_lmax_f(t.bshell, s0, s1), u[0], u[1], u[2], Y, c_rcpf);
      const int roff = c == 0 ? 0 : g.nFA;
      eval_shells_df(t.bshell, xi + (c == 0 ? 0 : nbA), s0, s1, c == 0 ? rhoA : rhoB, Y, bh, bl, ld, p,
                     g.row_F >= 0 ? g.row_F + roff : -1, 0, g.row_L >= 0 ? g.row_L + roff : -1, 1, etab);
    }
  }
  if (g.row_G >= 0 || g.row_U >= 0) {
    int roff = 0;
    for (int c = 0; c < 2; ++c) {
      const int s0 = c == 0 ? g.sha_0 : g.sha_2, s1 = c == 0 ? g.sha_1 : g.sha_3;
      const int atom = c == 0 ? g.aux_c0 : g.aux_c1;
      if (atom < 0 || s1 <= s0) continue;
      const df* u;
      df rho;
      if (atom == g.A) { u = uA; rho = rhoA; }
      else if (atom == g.B) { u = uB; rho = rhoB; }
      else { u = uC; rho = rC; }
      dfa::real_ylm(shells_lmax_f(t.ashell, s0, s1), u[0], u[1], u[2], Y, c_rcpf);
      eval_shells_df(t.ashell, xi + nbA + nbB + (c == 0 ? 0 : na0), s0, s1, rho, Y, bh, bl, ld, p,
                     g.row_G >= 0 ? g.row_G + roff : -1, 0, g.row_U >= 0 ? g.row_U + roff : -1, 2, etab);
      int nf = 0;
      for (int s = s0; s < s1; ++s) nf += 2 * t.ashell[s].l + 1;
      roff += nf;
    }
  }
}

// ------------------------------------------------------------------ tcgen05 contraction

namespace mma {

constexpr int kM = kMmaM;
constexpr int kTileN = kMmaN;
constexpr int kChunk = kChunkPts;
constexpr int kRowB = 2 * kChunkPts;            // bytes of one operand row of a stage (64)
constexpr int kStages = 3;                      // A ring depth (chunks, 40 KB each)
constexpr int kStagesB = 3;                     // B ring depth (chunks, 15 KB each)
constexpr int kChunksPerWin = kWinPts / kChunkPts;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512 bytes apart.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;    // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;             // descriptor version for sm_100 family
  d |= (uint64_t)4 << 61;             // SWIZZLE_64B
  return d;
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t make_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

// Non-blocking test of the phase of the given parity.
__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase of the given parity; gives up (false) after limit_ns nanoseconds, or
// early once *abort (if given) is set by another role of the CTA.
constexpr uint64_t kWaitNs = 4000000000ull;
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, const int* abort = nullptr,
                                          uint64_t limit_ns = kWaitNs) {
  if (mbar_try(mbar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(mbar, parity)) return true;
    if ((it & 255u) == 0) {
      if (abort && *(volatile const int*)abort) return false;
      if (global_ns() - t0 > limit_ns) return false;
    }
  }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ float pow2f(int k) {
  if (k < -126) return 0.0f;
  if (k > 127) k = 127;
  return __int_as_float((k + 127) << 23);
}

}  // namespace mma

// ------------------------------------------------------------------ operand packing
//
// Every operand row that a tile reads as a whole (weighted aux potentials, weighted kinetic
// operands, basis and aux functions) is sliced once per job into the tcgen05 shared-memory
// image by pack_kernel; the contraction then moves it with bulk copies.  Only the 3-index
// operand chi_i chi_j, whose rows are products of two basis rows, is formed inside the
// contraction, from basis rows staged in shared memory.
//
// Slicing.  A row's values in a 128-point window are scaled by 2^(7-e) (|v| < 2^e over the
// window) and cut into five digits v ~ s0 + s1/256 + ... + s4/256^4 of integers (each the
// nearest integer of what the previous digits left, times 256), exact in BF16: 39 bits of the
// window's largest value.  Values are double-float pairs, products of two pairs left
// unnormalised (|lo| <= 3 2^-24 |hi|); the first two digits come from the hi part (exactly),
// then the lo part joins the remainder, which rounds once, at 2^-17 of the third digit's unit
// (2^-40 of the window's largest value); s2 can reach 130.  Accumulation bound: the order-k
// sum sum_{i+j=k} s_i t_j over 128 points stays below 128 x 114688 < 2^24 for every k <= 4,
// so the FP32 tensor-core accumulators hold it exactly.

namespace mma {

// JOIN: the digit after which the lo parts join the remainder.  JOIN = 2 for normalised pairs
// (|lo| <= 2^-24 |hi|; s3 <= 256); JOIN = 1 for products left unnormalised (|lo| <= 3 2^-24
// |hi|: the join adds at most 1.5 to s2, which stays <= 130, and rounds at 2^-17 of s2's unit,
// 2^-40 of the window's largest value).
//
// Each digit takes three full-rate FP32 instructions.  With M = 1.5 x 2^23 and |x| < 2^22,
// t = x + M rounds x to its nearest integer s (ties to even): t lies in [2^23, 2^24), where the
// spacing is 1, so t = M + s exactly.  Then fma(t, -256, 256 M) = -256 s and
// fma(x, 256, -256 s) = 256 (x - s) are exact (|x - s| <= 1/2 is a multiple of x's spacing).
// The stored digit is -256 s, exact in BF16 like s (at most 8 significant bits); every operand
// is stored this way, so a slice product carries 2^16, which keeps the order sums exact in FP32
// (multiples of 2^16 below 2^40) and which the fold removes with the window scales.
constexpr float kRneMagic = 12582912.0f;         // 1.5 x 2^23
constexpr float kRneMagic256 = 3221225472.0f;    // 256 x 1.5 x 2^23 = 1.5 x 2^31
constexpr int kDigitScaleExp = 8;                // |stored digit| = 2^8 |s|

// BF16x2 bits of two floats that are exact in BF16 (at most 8 significant bits: their low 16
// bits are zero), first value in the low half.
__device__ __forceinline__ uint32_t pack_bf16_exact(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// The window scale of a row whose largest |value| is below 2^e, for the hi words (sc) and
// for the lo words joining after digit JOIN (sc 256^(JOIN + 1), capped at 2^127: rows below
// 2^-96, whose lo parts are below 2^-120, join them at a smaller weight).
template <int JOIN>
__device__ __forceinline__ void window_scales(int e, float& sc, float& scj) {
  sc = e == kZeroExp ? 0.0f : pow2f(7 - e);
  scj = e == kZeroExp ? 0.0f : pow2f(7 - e + 8 * (JOIN + 1));
}

template <int JOIN>
__device__ __forceinline__ void slice8_df(const float* vh, const float* vl, float sc, float scj, uint4* w) {
  uint32_t o[kSlices][4];
  const float sc256 = sc * 256.0f;  // at most 2^125
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float r0 = 0.0f, r1 = 0.0f;
    const float l0 = vl[2 * q] * scj, l1 = vl[2 * q + 1] * scj;
#pragma unroll
    for (int k = 0; k < kSlices; ++k) {
      // digit 0 rounds v sc (exact: sc is a power of two) inside its first FMA
      const float t0 = k == 0 ? __fmaf_rn(vh[2 * q], sc, kRneMagic) : __fadd_rn(r0, kRneMagic);
      const float t1 = k == 0 ? __fmaf_rn(vh[2 * q + 1], sc, kRneMagic) : __fadd_rn(r1, kRneMagic);
      const float d0 = __fmaf_rn(t0, -256.0f, kRneMagic256), d1 = __fmaf_rn(t1, -256.0f, kRneMagic256);
      o[k][q] = pack_bf16_exact(d0, d1);
      if (k + 1 < kSlices) {
        r0 = k == 0 ? __fmaf_rn(vh[2 * q], sc256, d0) : __fmaf_rn(r0, 256.0f, d0);
        r1 = k == 0 ? __fmaf_rn(vh[2 * q + 1], sc256, d1) : __fmaf_rn(r1, 256.0f, d1);
        if (k == JOIN) {
          r0 = __fadd_rn(r0, l0);
          r1 = __fadd_rn(r1, l1);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kSlices; ++k) w[k] = make_uint4(o[k][0], o[k][1], o[k][2], o[k][3]);
}

// Exponent e with mx < 2^e <= 2 mx (frexp's), read from the exponent bits, or kZeroExp for
// a row that is zero (or below 2^-110; subnormal maxima count as zero).
__device__ __forceinline__ int row_exponent(float mx) {
  const int e = (int)(__float_as_uint(mx) >> 23) - 126;  // mx >= 0
  return e < -110 ? kZeroExp : e;
}

// Byte offset of 16-byte group j (0..3) of row r in a 64-byte-row swizzled operand tile.
__device__ __forceinline__ uint32_t swz(int r, int j) { return (uint32_t)r * 64u + ((uint32_t)(j ^ ((r >> 1) & 3)) << 4); }

}  // namespace mma

// (xh + xl)(yh + yl) as hi = fl(xh yh) and the unnormalised lo = the exact error of that
// product plus the cross terms (|lo| <= 3 2^-24 |hi|; the lo lo term, below 2^-48, dropped).
__device__ __forceinline__ void prod_unnorm(float xh, float xl, float yh, float yl, float& h, float& l) {
  h = __fmul_rn(xh, yh);
  float e = __fmaf_rn(xh, yh, -h);
  e = __fmaf_rn(xh, yl, e);
  l = __fmaf_rn(xl, yh, e);
}

// Decodes packing job `job` (panel, tile, window, 16-row group) for this thread: 8 threads per
// row, thread qq holding points [16 qq, 16 qq + 16) of the window (chunk 4 w + qq/2, 16-byte
// groups 2 (qq % 2) and 2 (qq % 2) + 1 of its row).
struct PackPos {
  int pn, t, w, r, qq;
};

// The panel of a job: from hint[job / kPackHintJobs] (the panel of that block's first job) by
// a short forward scan, or by bisection when there is no hint.
__device__ __forceinline__ PackPos pack_pos(int64_t job, const Panel* __restrict__ panels, int n_panels,
                                            const int* __restrict__ hint) {
  int lo = 0;
  if (hint) {
    lo = __ldg(hint + (job / kPackHintJobs));
    while (lo + 1 < n_panels && panels[lo + 1].job_begin <= job) ++lo;
  } else {
    int hi = n_panels;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (panels[mid].job_begin <= job) lo = mid; else hi = mid;
    }
  }
  const Panel& pn = panels[lo];
  const int G = pn.tr / kPackRows;
  const int lj = (int)(job - pn.job_begin);  // jobs of one panel < 2^31 (one launch's grid)
  const int tw = lj / G, grp = lj - tw * G;
  PackPos P;
  P.pn = lo;
  P.t = tw / pn.nwin;
  P.w = tw - P.t * pn.nwin;
  P.r = kPackRows * grp + (threadIdx.x >> 3);
  P.qq = threadIdx.x & 7;
  return P;
}

// The row's window exponent (the eight threads of the row share it) and the five planes of
// this thread's 16 points.
__device__ __forceinline__ void pack_store(const PackPos& P, const Panel& pn, const float* h, const float* l,
                                           uint8_t* __restrict__ packed) {
  using namespace mma;
  float mx = 0.0f;
#pragma unroll
  for (int i = 0; i < 16; ++i) mx = fmaxf(mx, fabsf(h[i]));
  const unsigned m8 = 0xffu << ((threadIdx.x & 31) & ~7u);
  mx = fmaxf(mx, __shfl_xor_sync(m8, mx, 1));
  mx = fmaxf(mx, __shfl_xor_sync(m8, mx, 2));
  mx = fmaxf(mx, __shfl_xor_sync(m8, mx, 4));
  const int e = row_exponent(mx);
  if (P.qq == 0)
    *reinterpret_cast<int*>(packed + pn.exp_off + (((int64_t)P.t * pn.nwin + P.w) * pn.tr + P.r) * 4) = e;
  const int rt = min(pn.tr, pn.nrows - P.t * pn.tr);
  const int c = kChunksPerWin * P.w + (P.qq >> 1);
  if (c >= pn.nch || P.r >= rt) return;
  float sc, scj;
  window_scales<1>(e, sc, scj);
  uint8_t* dst = packed + pn.pack_off + (int64_t)P.t * pn.nch * (kSlices * pn.tr * kRowB) +
                 (int64_t)c * (kSlices * rt * kRowB);
  const int plane = rt * kRowB;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    uint4 wv[kSlices];
    slice8_df<1>(h + 8 * j, l + 8 * j, sc, scj, wv);
#pragma unroll
    for (int k = 0; k < kSlices; ++k) *reinterpret_cast<uint4*>(dst + k * plane + swz(P.r, 2 * (P.qq & 1) + j)) = wv[k];
  }
}

// One CTA of 128 threads per packing job.  Values: source row times its weight row
// (double-float products), zeros past K.
__global__ void __launch_bounds__(128) pack_kernel(const DevGrid* __restrict__ grids, const Panel* __restrict__ panels,
                                                   int n_panels, const int* __restrict__ hint, const short2* __restrict__ rows,
                                                   const float* __restrict__ ops, const float* __restrict__ ops_lo,
                                                   uint8_t* __restrict__ packed) {
  const PackPos P = pack_pos(blockIdx.x, panels, n_panels, hint);
  const Panel& pn = panels[P.pn];
  const DevGrid& g = grids[pn.grid];
  const int row = P.t * pn.tr + P.r;
  const int64_t k0 = (int64_t)kWinPts * P.w + 16 * P.qq;
  int64_t src = -1, mul = -1;
  if (row < pn.nrows) {
    const short2 q = rows[pn.rows_off + row];
    src = g.op_off + (int64_t)q.x * g.ld + k0;
    if (q.y >= 0) mul = g.op_off + (int64_t)q.y * g.ld + k0;
  }
  const int64_t left = src >= 0 ? g.K - k0 : 0;
  float h[16], l[16];
#pragma unroll
  for (int i4 = 0; i4 < 4; ++i4) {
    float4 ah = make_float4(0.f, 0.f, 0.f, 0.f), al = ah, bh = make_float4(1.f, 1.f, 1.f, 1.f), bl = al;
    if (left >= 4 * i4 + 4) {
      ah = __ldg(reinterpret_cast<const float4*>(ops + src) + i4);
      al = __ldg(reinterpret_cast<const float4*>(ops_lo + src) + i4);
      if (mul >= 0) {
        bh = __ldg(reinterpret_cast<const float4*>(ops + mul) + i4);
        bl = __ldg(reinterpret_cast<const float4*>(ops_lo + mul) + i4);
      }
    } else if (left > 4 * i4) {
      float* ph = &ah.x; float* pl = &al.x; float* qh = &bh.x; float* ql = &bl.x;
      for (int i = 0; i < 4 && 4 * i4 + i < left; ++i) {
        ph[i] = ops[src + 4 * i4 + i];
        pl[i] = ops_lo[src + 4 * i4 + i];
        if (mul >= 0) {
          qh[i] = ops[mul + 4 * i4 + i];
          ql[i] = ops_lo[mul + 4 * i4 + i];
        }
      }
    }
    const float xh[4] = {ah.x, ah.y, ah.z, ah.w}, xl[4] = {al.x, al.y, al.z, al.w};
    const float yh[4] = {bh.x, bh.y, bh.z, bh.w}, yl[4] = {bl.x, bl.y, bl.z, bl.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (mul >= 0) {
        prod_unnorm(xh[i], xl[i], yh[i], yl[i], h[4 * i4 + i], l[4 * i4 + i]);
      } else {
        h[4 * i4 + i] = xh[i];
        l[4 * i4 + i] = xl[i];
      }
    }
  }
  pack_store(P, pn, h, l, packed);
}

// The same packed-panel image from FP64 operand rows (row-major, stride n): used for the
// RI 4-index product, whose operand rows are the (P|ij) columns after the forward solve.
// Panel k's rows start at src[k]; jobs as in pack_kernel, both panels' jobs in one launch.
// Each FP64 value is split into a double-float pair first (48 bits, beyond the 39 that the
// digits keep).
__global__ void __launch_bounds__(128) ri_pack_kernel(const Panel* __restrict__ panels, const double* __restrict__ srcA,
                                                      const double* __restrict__ srcB, int n, uint8_t* __restrict__ packed) {
  const PackPos P = pack_pos(blockIdx.x, panels, 2, nullptr);
  const Panel& pn = panels[P.pn];
  const double* src = P.pn ? srcB : srcA;
  const int row = P.t * pn.tr + P.r;
  const int k0 = kWinPts * P.w + 16 * P.qq;
  float h[16], l[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    double v = 0.0;
    if (row < pn.nrows && k0 + i < n) v = src[(int64_t)row * n + k0 + i];
    h[i] = (float)v;
    l[i] = (float)(v - (double)h[i]);
  }
  pack_store(P, pn, h, l, packed);
}

// ------------------------------------------------------------------ warp-specialised contraction
//
// One persistent CTA per SM, 512 threads, working through tiles (128 A rows x <= 48 B
// columns x a range of 128-point windows):
//   warp 4       loader: two ordered streams of bulk copies, each served as soon as its next
//                buffer is free: the packed A tile of every 32-point chunk into a three-stage
//                A ring (and, for a packed B, its B tile into the B ring), and the staged basis
//                rows (hi and lo planes) of every formed window into two buffers;
//   warps 0-3, 6, 7  producers: for a formed B, column c of the tile = product of two staged
//                rows (a double-float product); each warp owns 8 columns, four lanes per
//                column, lane g the 16-byte group g of every chunk; per window they form the
//                products, find each column's scale, then slice chunk by chunk into the B ring,
//                so that the MMAs of one chunk overlap the slicing of the next (for a packed B
//                they only pass each chunk on);
//   warp 5       MMA issue: per chunk 2 K-steps x 5 MMAs (A plane i against B planes
//                0..4-i, contiguous in shared memory: one MMA of N = 48 (5 - i) whose columns
//                land on the order accumulators i..4) into the window's TMEM accumulator set
//                (5 orders x 48 columns; two sets);
//   warps 8-15   fold: per window, the five order sums of their TMEM lane quadrant and column
//                half, scaled by the window's row and column exponents, into double-float
//                registers (orders 0 and 1 join the sum exactly through TwoSums, orders 2-4
//                as one FP32 term); at the end of the tile, (hi, lo) partials to global memory.
// Every wait is bounded (wait_ns in the main loops, the fixed kWaitNs for the drains); a
// timeout sets *status and the CTA's abort flag, and each role leaves its loops at its next
// wait; the loader then waits for its copies in flight and the MMA lane for its MMAs before
// the TMEM is released.

namespace ws {

constexpr int kThreads = 512;
constexpr int kLoadWarp = 4, kMmaWarp = 5, kFoldWarp0 = 8;
constexpr int kRawStride = 132;  // floats per staged row: 128 points + 4 (bank spread)

struct Smem {
  alignas(1024) uint8_t a[mma::kStages][kSlices][mma::kM * mma::kRowB];
  alignas(1024) uint8_t b[mma::kStagesB][kSlices][mma::kTileN * mma::kRowB];
  alignas(16) float raw[2][2][kPairTileRows][kRawStride];  // [buffer][hi, lo][row][point]
  int eb[2][mma::kTileN];
  float sbw[8][mma::kTileN];  // fold warp k: the column scales of the current window
  alignas(8) uint64_t a_full[mma::kStages], a_free[mma::kStages], b_ready[mma::kStagesB], b_free[mma::kStagesB];
  uint64_t tmem_full[2], tmem_free[2], raw_full[2], raw_free[2], eb_free[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mma::smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(mma::smem_u32(b))
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   mma::smem_u32(b)),
               "r"(bytes)
               : "memory");
}

// Bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completing
// on mbarrier b.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   mma::smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(mma::smem_u32(b))
               : "memory");
}

__device__ __forceinline__ bool wait(uint64_t* b, uint32_t parity, const int* abort, uint64_t limit_ns) {
  return mma::mbar_wait(mma::smem_u32(b), parity, abort, limit_ns);
}

// Ring positions of chunk c: A stage c % kStages after c / kStages completed rounds, B stage
// c % kStagesB after c / kStagesB rounds.
__device__ __forceinline__ int stage_of(uint32_t c) { return (int)(c % mma::kStages); }
__device__ __forceinline__ uint32_t round_of(uint32_t c) { return c / mma::kStages; }
__device__ __forceinline__ int bstage_of(uint32_t c) { return (int)(c % mma::kStagesB); }
__device__ __forceinline__ uint32_t bround_of(uint32_t c) { return c / mma::kStagesB; }
// A stage of chunk c free again (its MMAs of chunk c - kStages complete)
__device__ __forceinline__ bool wait_a_free(Smem& sm, uint32_t c, uint64_t ns) {
  return c < (uint32_t)mma::kStages || mma::mbar_wait(mma::smem_u32(&sm.a_free[stage_of(c)]), (round_of(c) - 1) & 1, &sm.abort, ns);
}
// B stage of chunk c free again (its MMAs of chunk c - kStagesB complete)
__device__ __forceinline__ bool wait_b_free(Smem& sm, uint32_t c, uint64_t ns) {
  return c < (uint32_t)mma::kStagesB ||
         mma::mbar_wait(mma::smem_u32(&sm.b_free[bstage_of(c)]), (bround_of(c) - 1) & 1, &sm.abort, ns);
}

// What every role needs to know about an item.
struct Geo {
  const MmaBlock* blk;
  int64_t K;
  int nch, nwin, w0, w1;
  int nt;  // B columns of the tile
  bool formed;
  const PairTile* pt;
};

__device__ __forceinline__ Geo geo(const GemmItem& it, const MmaBlock* blocks, const DevGrid* grids,
                                   const PairTile* ptiles) {
  Geo q;
  q.blk = blocks + it.block;
  const MmaBlock& b = *q.blk;
  q.K = grids[b.grid].K;
  q.nch = (int)((q.K + mma::kChunk - 1) / mma::kChunk);
  q.nwin = (q.nch + mma::kChunksPerWin - 1) / mma::kChunksPerWin;
  q.w0 = it.chunk * b.win_per;
  q.w1 = min(q.nwin, q.w0 + b.win_per);
  q.formed = b.b_panel < 0;
  q.pt = q.formed ? ptiles + b.ptile_off + it.tn : nullptr;
  q.nt = q.formed ? q.pt->ncols : min(mma::kTileN, b.n - it.tn * mma::kTileN);
  return q;
}

__device__ __forceinline__ int chunks_in(const Geo& q, int win) { return min(mma::kChunksPerWin, q.nch - mma::kChunksPerWin * win); }

__device__ __forceinline__ void fail(Smem& sm, int* status, int code) {
  *(volatile int*)&sm.abort = 1;
  atomicCAS(status, 0, code);  // the first failure's code stays
}

__device__ __forceinline__ bool aborted(Smem& sm) { return *(volatile int*)&sm.abort != 0; }

// The loader's stream of staged-row requests: the formed windows of the CTA's items in the
// order the producers form them, with the current item's tile rows and grid offsets cached
// (one lookup per item, not per window).
struct RowStream {
  int ii, ie, win, w1;  // current item, end, next window, the item's window end
  int nr;               // staged rows of the item's pair tile (<= kPairTileRows)
  int64_t src;          // this lane's row (lane & 15) of plane (lane >> 4), window 0, in floats
  bool more;

  __device__ __forceinline__ void open(int i0, int i1, const GemmItem* items, const MmaBlock* blocks,
                                       const DevGrid* grids, const PairTile* ptiles, int lane) {
    ii = i0;
    ie = i1;
    win = -1;
    more = false;
    seek(items, blocks, grids, ptiles, lane, false);
  }
  // Advances to the next formed window (the next window of the current item when `step`).
  __device__ __forceinline__ void seek(const GemmItem* items, const MmaBlock* blocks, const DevGrid* grids,
                                       const PairTile* ptiles, int lane, bool step) {
    if (step && ++win < w1) return;
    if (step) ++ii;
    for (; ii < ie; ++ii) {
      const Geo q = geo(items[ii], blocks, grids, ptiles);
      if (!q.formed) continue;
      const DevGrid& g = grids[q.blk->grid];
      win = q.w0;
      w1 = q.w1;
      nr = q.pt->nrows;
      src = g.op_off + (int64_t)q.pt->rows[max(0, min(lane & 15, nr - 1))] * g.ld;
      more = win < w1;
      if (more) return;
    }
    more = false;
  }
  // Bulk copies of the current window's rows (hi and lo planes, 512 bytes per row and plane)
  // into raw buffer rb, completing on raw_full[rb]; one warp.
  __device__ __forceinline__ void request(Smem& sm, int rb, const float* ops, const float* ops_lo, int lane) const {
    if (lane == 0) mbar_expect_tx(&sm.raw_full[rb], (uint32_t)nr * 2u * 512u);
    __syncwarp();
    const int rr = lane & 15, pl = lane >> 4;
    if (rr < nr) bulk_g2s(sm.raw[rb][pl][rr], (pl ? ops_lo : ops) + src + (int64_t)kWinPts * win, 512u, &sm.raw_full[rb]);
  }
};

}  // namespace ws

__global__ void __launch_bounds__(ws::kThreads, 1)
    contract_ws_kernel(const DevGrid* __restrict__ grids, const MmaBlock* __restrict__ blocks,
                       const GemmItem* __restrict__ items, const int* __restrict__ cta_begin,
                       const Panel* __restrict__ panels, const PairTile* __restrict__ ptiles,
                       const float* __restrict__ ops, const float* __restrict__ ops_lo,
                       const uint8_t* __restrict__ packed, float2* __restrict__ part, int* __restrict__ status,
                       uint64_t wait_ns, const int* __restrict__ hold) {
  using namespace mma;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  ws::Smem& sm = *reinterpret_cast<ws::Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == ws::kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      ws::mbar_init(&sm.a_full[s], 1);
      ws::mbar_init(&sm.a_free[s], 1);
    }
    for (int s = 0; s < kStagesB; ++s) {
      ws::mbar_init(&sm.b_ready[s], 6);
      ws::mbar_init(&sm.b_free[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      ws::mbar_init(&sm.tmem_full[s], 1);
      ws::mbar_init(&sm.tmem_free[s], 8);
      ws::mbar_init(&sm.raw_full[s], 1);
      ws::mbar_init(&sm.raw_free[s], 6);
      ws::mbar_init(&sm.eb_free[s], 8);
    }
    ws::mbar_init(&sm.drain, 1);
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm.tmem_base;
  uint32_t c = 0, w = 0, rw = 0;  // chunks, windows and formed windows of this CTA so far

  constexpr unsigned kFull = 0xffffffffu;
  if (warp == ws::kLoadWarp) {
    // ------------------------------------------------------------------ loader
    bool run = true;  // warp-uniform
    int last_a = -1;  // last issued chunk (for the drain)
    if (hold) {
      // failure-detection test: a raised flag that nothing clears holds the first copy back
      // until the wait limit runs out
      int held = 0;
      if (lane == 0) {
        const uint64_t t0 = global_ns();
        while ((held = *(volatile const int*)hold) != 0 && global_ns() - t0 <= wait_ns) {
        }
      }
      if (__shfl_sync(kFull, held, 0) != 0) {
        ws::fail(sm, status, 8);
        run = false;
      }
    }
    // Two ordered streams: the packed A (and packed B) tiles of every chunk into the rings, and
    // the staged basis rows of every formed window into two buffers (the rows of formed window
    // k + 1 are in flight while the producers form window k).  The warp waits for the chunk
    // stream's buffers and, before each of those waits, requests every window of rows whose
    // buffer is already free.
    const int ie = cta_begin[blockIdx.x + 1];
    ws::RowStream rs;
    rs.open(cta_begin[blockIdx.x], ie, items, blocks, grids, ptiles, lane);
    uint32_t rq = 0;  // formed windows requested
    auto request_free = [&]() {
      while (rs.more) {
        // buffer rq & 1 last held formed window rq - 2, released after its products
        const int rb = (int)(rq & 1);
        int free_ = 1;
        if (lane == 0) free_ = rq < 2 || mbar_test(smem_u32(&sm.raw_free[rb]), ((rq - 2) >> 1) & 1);
        if (!__shfl_sync(kFull, free_, 0)) return;
        rs.request(sm, rb, ops, ops_lo, lane);
        ++rq;
        rs.seek(items, blocks, grids, ptiles, lane, true);
      }
    };
    for (int ii = cta_begin[blockIdx.x]; ii < ie && run; ++ii) {
      const GemmItem it = items[ii];
      const ws::Geo q = ws::geo(it, blocks, grids, ptiles);
      const MmaBlock& b = *q.blk;
      const Panel& pa = panels[b.a_panel];
      const Panel* pb = q.formed ? nullptr : panels + b.b_panel;
      for (int win = q.w0; win < q.w1 && run; ++win) {
        const int nck = ws::chunks_in(q, win);
        for (int j = 0; j < nck; ++j, ++c) {
          request_free();
          const int s = ws::stage_of(c), sb = ws::bstage_of(c), ch = kChunksPerWin * win + j;
          const bool ok = ws::wait_a_free(sm, c, wait_ns) && (!pb || ws::wait_b_free(sm, c, wait_ns));
          run = __all_sync(kFull, ok && !ws::aborted(sm));
          if (!run) { ws::fail(sm, status, 4); break; }
          // the stored rows of the tiles, one bulk copy per plane (lanes 0-4: A, 5-9: B)
          const int ra = min(kM, pa.nrows - it.tm * kM);
          const int rbw = pb ? min(kTileN, pb->nrows - it.tn * kTileN) : 0;
          if (lane == 0) ws::mbar_expect_tx(&sm.a_full[s], (uint32_t)(kSlices * kRowB * (ra + rbw)));
          __syncwarp();
          if (lane < kSlices) {
            const uint8_t* src = packed + pa.pack_off + (int64_t)it.tm * pa.nch * (kSlices * kM * kRowB) +
                                 (int64_t)ch * (kSlices * ra * kRowB) + (int64_t)lane * ra * kRowB;
            ws::bulk_g2s(sm.a[s][lane], src, (uint32_t)(kRowB * ra), &sm.a_full[s]);
          } else if (lane < 2 * kSlices && pb) {
            const int k = lane - kSlices;
            const uint8_t* src = packed + pb->pack_off + (int64_t)it.tn * pb->nch * (kSlices * kTileN * kRowB) +
                                 (int64_t)ch * (kSlices * rbw * kRowB) + (int64_t)k * rbw * kRowB;
            ws::bulk_g2s(sm.b[sb][k], src, (uint32_t)(kRowB * rbw), &sm.a_full[s]);
          }
          __syncwarp();
          last_a = (int)c;
        }
      }
    }
    // the rows of the last formed windows, as their buffers free up
    while (run && rs.more) {
      const int rb = (int)(rq & 1);
      const bool ok = rq < 2 || ws::wait(&sm.raw_free[rb], ((rq - 2) >> 1) & 1, &sm.abort, wait_ns);
      run = __all_sync(kFull, ok && !ws::aborted(sm));
      if (!run) { ws::fail(sm, status, 4); break; }
      request_free();
    }
    // drain: nothing may still be copying into shared memory when the CTA exits (another
    // role may have given up after this loop ended; the phases waited for here are the last
    // ones issued on each barrier, complete at once when the copies were consumed)
    for (int k = last_a; k >= 0 && k > last_a - kStages; --k)
      ws::wait(&sm.a_full[ws::stage_of(k)], ws::round_of(k) & 1, nullptr, kWaitNs);
    for (int k = (int)rq - 1; k >= 0 && k > (int)rq - 3; --k)
      ws::wait(&sm.raw_full[k & 1], (k >> 1) & 1, nullptr, kWaitNs);
  } else if (warp < 4 || warp == 6 || warp == 7) {
    // ------------------------------------------------------------------ producers
    const int pw = warp < 4 ? warp : warp - 2;  // 0..5
    const int col = 8 * pw + (lane >> 2);       // 0..47: this lane's column of the tile
    const int g = lane & 3;                     // 16-byte group of each chunk's row
    const unsigned col_mask = 0xfu << (lane & 28);
    bool run = true;  // warp-uniform
    for (int ii = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1]; ii < ie && run; ++ii) {
      const GemmItem it = items[ii];
      const ws::Geo q = ws::geo(it, blocks, grids, ptiles);
      if (!q.formed) {
        // packed B: the loader brings it; b_ready still completes one phase per chunk
        for (int win = q.w0; win < q.w1 && run; ++win, ++w) {
          const int nck = ws::chunks_in(q, win);
          for (int j = 0; j < nck; ++j, ++c) {
            const int sb = ws::bstage_of(c);
            const bool ok = ws::wait_b_free(sm, c, wait_ns);
            run = __all_sync(kFull, ok && !ws::aborted(sm));
            if (!run) { ws::fail(sm, status, 5); break; }
            if (lane == 0) ws::mbar_arrive(&sm.b_ready[sb]);
          }
        }
        continue;
      }
      const bool valid = col < q.nt;
      const int dx = valid ? q.pt->dx[col] : 0, dy = valid ? q.pt->dy[col] : 0;
      for (int win = q.w0; win < q.w1 && run; ++win, ++w, ++rw) {
        const int nck = ws::chunks_in(q, win);
        const int rb = rw & 1, set = w & 1;
        bool ok = ws::wait(&sm.raw_full[rb], (rw >> 1) & 1, &sm.abort, wait_ns);
        run = __all_sync(kFull, ok && !ws::aborted(sm));
        if (!run) { ws::fail(sm, status, 5); break; }
        const int64_t wleft = q.K - (int64_t)kWinPts * win;  // points of the window that exist
        float vh[kChunksPerWin][8], vl[kChunksPerWin][8];
        float mx = 0.0f;
#pragma unroll
        for (int cc = 0; cc < kChunksPerWin; ++cc) {
          const int p0 = kChunk * cc + 8 * g;
          const float* xh = sm.raw[rb][0][dx] + p0;
          const float* xl = sm.raw[rb][1][dx] + p0;
          const float* yh = sm.raw[rb][0][dy] + p0;
          const float* yl = sm.raw[rb][1][dy] + p0;
          const int64_t left = valid ? wleft - p0 : 0;
          if (left >= 8) {
            float a[8], al[8], bb[8], bl[8];
            *reinterpret_cast<float4*>(a) = *reinterpret_cast<const float4*>(xh);
            *reinterpret_cast<float4*>(a + 4) = *reinterpret_cast<const float4*>(xh + 4);
            *reinterpret_cast<float4*>(al) = *reinterpret_cast<const float4*>(xl);
            *reinterpret_cast<float4*>(al + 4) = *reinterpret_cast<const float4*>(xl + 4);
            *reinterpret_cast<float4*>(bb) = *reinterpret_cast<const float4*>(yh);
            *reinterpret_cast<float4*>(bb + 4) = *reinterpret_cast<const float4*>(yh + 4);
            *reinterpret_cast<float4*>(bl) = *reinterpret_cast<const float4*>(yl);
            *reinterpret_cast<float4*>(bl + 4) = *reinterpret_cast<const float4*>(yl + 4);
#pragma unroll
            for (int i = 0; i < 8; ++i) prod_unnorm(a[i], al[i], bb[i], bl[i], vh[cc][i], vl[cc][i]);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              vh[cc][i] = 0.0f;
              vl[cc][i] = 0.0f;
              if (i < left) prod_unnorm(xh[i], xl[i], yh[i], yl[i], vh[cc][i], vl[cc][i]);
            }
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) mx = fmaxf(mx, fabsf(vh[cc][i]));
        }
        // the staged rows are read: release the buffer for the window after next
        __syncwarp();
        if (lane == 0) ws::mbar_arrive(&sm.raw_free[rb]);
        // the column's window maximum over its four lanes
        mx = fmaxf(mx, __shfl_xor_sync(col_mask, mx, 1));
        mx = fmaxf(mx, __shfl_xor_sync(col_mask, mx, 2));
        const int e = row_exponent(mx);
        // the column exponents of this set were last read by the fold of window w - 2, which
        // releases them (eb_free) as soon as it has copied them: the fold stays off this path
        const bool okb = w < 2 || ws::wait(&sm.eb_free[set], ((w - 2) >> 1) & 1, &sm.abort, wait_ns);
        run = __all_sync(kFull, okb && !ws::aborted(sm));
        if (!run) { ws::fail(sm, status, 5); break; }
        if (g == 0) sm.eb[set][col] = e;
        float sc, scj;
        window_scales<1>(e, sc, scj);
#pragma unroll
        for (int cc = 0; cc < kChunksPerWin; ++cc) {
          if (cc < nck && run) {
            const int sb = ws::bstage_of(c);
            const bool okc = ws::wait_b_free(sm, c, wait_ns);
            run = __all_sync(kFull, okc && !ws::aborted(sm));
            if (!run) {
              ws::fail(sm, status, 5);
            } else {
              uint4 wv[kSlices];
              slice8_df<1>(vh[cc], vl[cc], sc, scj, wv);
#pragma unroll
              for (int k = 0; k < kSlices; ++k) *reinterpret_cast<uint4*>(sm.b[sb][k] + swz(col, g)) = wv[k];
              fence_async_smem();
              __syncwarp();
              if (lane == 0) ws::mbar_arrive(&sm.b_ready[sb]);
              ++c;
            }
          }
        }
        if (!run) break;
      }
    }
  } else if (warp == ws::kMmaWarp) {
    // ------------------------------------------------------------------ MMA issue
    if (lane == 0) {
      for (int ii = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1]; ii < ie && !ws::aborted(sm); ++ii) {
        const GemmItem it = items[ii];
        const ws::Geo q = ws::geo(it, blocks, grids, ptiles);
        bool ok = true;
        for (int win = q.w0; win < q.w1 && ok; ++win, ++w) {
          const int nck = ws::chunks_in(q, win);
          const int set = w & 1;
          if (w >= 2) ok = ws::wait(&sm.tmem_free[set], ((w - 2) >> 1) & 1, &sm.abort, wait_ns);
          const uint32_t tset = tmem + (uint32_t)set * 256u;
          for (int j = 0; j < nck && ok; ++j, ++c) {
            const int s = ws::stage_of(c), sb = ws::bstage_of(c);
            ok = ws::wait(&sm.a_full[s], ws::round_of(c) & 1, &sm.abort, wait_ns);
            if (ok) ok = ws::wait(&sm.b_ready[sb], ws::bround_of(c) & 1, &sm.abort, wait_ns);
            if (!ok) break;
            fence_after();
            // The B planes of a stage are contiguous (48 rows each), so plane i of A against
            // planes 0..4-i of B is one MMA of N = 48 (5 - i) whose columns land on the order
            // accumulators i..4 (order k at TMEM columns 48k..48k+47 of the set).
#pragma unroll
            for (int k = 0; k < kChunk / 16; ++k) {
              const uint32_t ko = 32u * k;
              const uint64_t db = make_desc(smem_u32(sm.b[sb][0]) + ko);
#pragma unroll
              for (int i = 0; i < kSlices; ++i) {
                const uint64_t da = make_desc(smem_u32(sm.a[s][i]) + ko);
                mma_bf16(tset + (uint32_t)(kTileN * i), da, db, make_idesc(kTileN * (kSlices - i)),
                         (j > 0 || k > 0 || i > 0) ? 1u : 0u);
              }
            }
            mma_commit(smem_u32(&sm.a_free[s]));
            mma_commit(smem_u32(&sm.b_free[sb]));
          }
          if (!ok) { ws::fail(sm, status, 6); break; }
          mma_commit(smem_u32(&sm.tmem_full[set]));
        }
        if (!ok) break;
      }
      // drain: every issued MMA must be complete before the TMEM is released (also when
      // another role gave up after this loop ended)
      mma_commit(smem_u32(&sm.drain));
      ws::wait(&sm.drain, 0, nullptr, kWaitNs);
    }
    __syncwarp();
  } else if (warp >= ws::kFoldWarp0) {
    // ------------------------------------------------------------------ fold
    const int ew = warp - ws::kFoldWarp0;  // 0..7
    const int quad = warp & 3;             // TMEM lane quadrant this warp may access
    const int half = ew >> 2;              // columns [24 half, 24 half + 24)
    const int row_in_tile = quad * 32 + lane;
    const int my_col = 24 * half + lane;   // lanes 0-23: the column whose scale this lane loads
    bool run = true;  // warp-uniform
    for (int ii = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1]; ii < ie && run; ++ii) {
      const GemmItem it = items[ii];
      const ws::Geo q = ws::geo(it, blocks, grids, ptiles);
      const MmaBlock& b = *q.blk;
      const Panel& pa = panels[b.a_panel];
      const Panel* pb = q.formed ? nullptr : panels + b.b_panel;
      const int rows_valid = min(kM, b.m - it.tm * kM);  // real rows of the A tile
      float H[24], L[24];
#pragma unroll
      for (int j = 0; j < 24; ++j) { H[j] = 0.0f; L[j] = 0.0f; }
      // the window's exponents (A rows from the packed panel; B columns from the packed panel,
      // one per lane for this warp's 24 columns, or from the producers), loaded one window ahead
      const int* ea_src = reinterpret_cast<const int*>(packed + pa.exp_off) + (int64_t)it.tm * pa.nwin * kM + row_in_tile;
      const int* eb_src = (pb && lane < 24)
                              ? reinterpret_cast<const int*>(packed + pb->exp_off) + (int64_t)it.tn * pb->nwin * kTileN + my_col
                              : nullptr;
      int ea_next = __ldg(ea_src + (int64_t)q.w0 * kM);
      int eb_next = eb_src ? __ldg(eb_src + (int64_t)q.w0 * kTileN) : 0;
      for (int win = q.w0; win < q.w1; ++win, ++w) {
        const int set = w & 1;
        const int ea = ea_next, eb_lane = eb_next;
        if (win + 1 < q.w1) {
          ea_next = __ldg(ea_src + (int64_t)(win + 1) * kM);
          if (eb_src) eb_next = __ldg(eb_src + (int64_t)(win + 1) * kTileN);
        }
        const bool ok = ws::wait(&sm.tmem_full[set], (w >> 1) & 1, &sm.abort, wait_ns);
        run = __all_sync(kFull, ok && !ws::aborted(sm));
        if (!run) { ws::fail(sm, status, 7); break; }
        fence_after();
        // column scales 2^(e_b - 7 - 8) for this warp, row scale 2^(e_a - 7 - 8) for this
        // thread (each stored digit carries 2^8)
        float* sbw = sm.sbw[ew];
        if (lane < 24) sbw[my_col] = pow2f((pb ? eb_lane : sm.eb[set][my_col]) - 7 - kDigitScaleExp);
        const float sa = pow2f(ea - 7 - kDigitScaleExp);
        __syncwarp();
        if (lane == 0) ws::mbar_arrive(&sm.eb_free[set]);  // the producers may refill eb[set]
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)set * 256u;
        // a warp whose 32 rows are all past the tile's last real row has nothing to fold
        if (quad * 32 < rows_valid) {
#pragma unroll
          for (int gi = 0; gi < 3; ++gi) {
            const int c0 = 24 * half + 8 * gi;  // first of 8 columns
            if (c0 < q.nt) {
              float o[kSlices][8];
#pragma unroll
              for (int k = 0; k < kSlices; ++k) tmem_ld8(lane_base + (uint32_t)(kTileN * k + c0), o[k]);
              tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int qq = 8 * gi + j;
                const float sc = sa * sbw[c0 + j];  // 2^(e_a + e_b - 30)
                // Order 1 splits exactly into q1, its nearest multiple of 2^24 (adding 1.5 x 2^47
                // rounds at that spacing), and r1 = o1 - q1; q1 / 256 joins order 0 exactly
                // (both multiples of 2^16 below 2^38).  That part, times the power of two sc,
                // enters the double-float sum through one TwoSum; r1 / 256 and orders 2-4 (at
                // most 2^-15 of order 0) join the lo word as one FP32 term, rounded at 2^-16 of
                // order 0's unit (2^-37 of the window's largest possible sum).
                const float q1 = __fsub_rn(__fadd_rn(o[1][j], 211106232532992.0f), 211106232532992.0f);
                const float r1 = __fsub_rn(o[1][j], q1);
                const df s0 = dfa::two_sum(H[qq], __fmaf_rn(q1, 0.00390625f, o[0][j]) * sc);
                const float tail =
                    fmaf(r1, 0.00390625f,
                         fmaf(o[2][j], 1.52587890625e-5f, fmaf(o[4][j], 2.3283064365386963e-10f, o[3][j] * 5.9604644775390625e-8f))) *
                    sc;
                const float lo = L[qq] + (s0.l + tail);
                const df r = dfa::fast_two_sum(s0.h, lo);
                H[qq] = r.h;
                L[qq] = r.l;
              }
            }
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) ws::mbar_arrive(&sm.tmem_free[set]);
      }
      if (!run) break;
      // (hi, lo) partial sums of this tile's window range
      const int grow = it.tm * kM + row_in_tile;
      if (grow < b.m) {
        float2* out = part + b.part_off + (int64_t)it.chunk * b.m * b.n + (int64_t)grow * b.n;
#pragma unroll
        for (int j = 0; j < 24; ++j) {
          const int cc = 24 * half + j;
          if (cc < q.nt) {
            const int ocol = q.formed ? q.pt->col[cc] : it.tn * kTileN + cc;
            out[ocol] = make_float2(H[j], L[j]);
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == ws::kMmaWarp) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// FP64 reduction of the (hi, lo) range partials of the tensor-core blocks, times the FP64
// constants of each element's row and column; one thread per element, ranges added in
// order (consecutive threads read consecutive partials).
__global__ void __launch_bounds__(256) reduce_mixed_kernel(const DevGrid* __restrict__ grids,
                                                           const MmaBlock* __restrict__ blocks, int n_blocks,
                                                           const int64_t* __restrict__ elem_begin, int64_t e0,
                                                           int64_t e1, const short2* __restrict__ rows,
                                                           const double* __restrict__ rowc,
                                                           const float2* __restrict__ part, double* __restrict__ res) {
  const int64_t idx = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= e1) return;
  int lo = 0, hi = n_blocks;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (elem_begin[mid] <= idx) lo = mid; else hi = mid;
  }
  const MmaBlock b = blocks[lo];
  const int64_t e = idx - elem_begin[lo];
  const int64_t mn = (int64_t)b.m * b.n;
  const float2* p = part + b.part_off + e;
  double s = 0.0;
  for (int c = 0; c < b.n_ranges; ++c) {
    const float2 v = __ldg(p + c * mn);
    s += (double)v.x + (double)v.y;
  }
  const int r = (int)(e / b.n), col = (int)(e % b.n);
  const double* rc = rowc + grids[b.grid].rc_off;
  const short2 qa = rows[b.a_off + r], qb = rows[b.b_off + col];
  const double ca = rc[qa.x] * (qa.y >= 0 ? rc[qa.y] : 1.0);
  const double cb = rc[qb.x] * (qb.y >= 0 ? rc[qb.y] : 1.0);
  res[b.res_off + e] = s * ca * cb;
}

// Diagnostics: operand rows (hi + lo) times their FP64 row constants, as FP64 rows of K values.
__global__ void combine_rows_kernel(const float* __restrict__ h, const float* __restrict__ l,
                                    const double* __restrict__ rc, int nrows, int64_t K, int64_t ld,
                                    double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nrows * K) return;
  const int r = (int)(i / K);
  const int64_t p = i - (int64_t)r * K;
  out[i] = ((double)h[r * ld + p] + (double)l[r * ld + p]) * rc[r];
}

// ------------------------------------------------------------------ launchers

cudaError_t launch_combine_rows(const float* h, const float* l, const double* rc, int nrows, int64_t K, int64_t ld,
                                double* out, cudaStream_t s) {
  const int64_t n = (int64_t)nrows * K;
  if (n == 0) return cudaSuccess;
  combine_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h, l, rc, nrows, K, ld, out);
  return cudaGetLastError();
}

cudaError_t launch_nodes(const DevGrid* grids, int n_grids, int max_entries, const double* edges, NodeEntry* tab,
                         cudaStream_t s) {
  if (n_grids == 0) return cudaSuccess;
  dim3 grid((max_entries + 127) / 128, n_grids);
  nodes_kernel<<<grid, 128, 0, s>>>(grids, edges, tab);
  return cudaGetLastError();
}

cudaError_t launch_eval_mixed(const LaunchTables& t, const NodeEntry* tab, const float2* xi, float* ops,
                              float* ops_lo, cudaStream_t s) {
  if (t.n_pblocks == 0) return cudaSuccess;
  eval_mixed_kernel<<<t.n_pblocks, 128, 0, s>>>(t, tab, xi, ops, ops_lo);
  return cudaGetLastError();
}

// the ring, staging buffers and barriers, plus 1 KB to align the ring's start
static_assert(sizeof(ws::Smem) + 1024 <= 232448, "contraction shared memory above the 227 KB a CTA may use");
size_t ws_smem_bytes() { return sizeof(ws::Smem) + 1024; }

cudaError_t prepare_kernels() {
  return cudaFuncSetAttribute(contract_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws_smem_bytes());
}

cudaError_t launch_pack(const DevGrid* grids, const Panel* panels, int n_panels, const int* hint, int64_t n_jobs,
                        const short2* rows, const float* ops, const float* ops_lo, uint8_t* packed, cudaStream_t s) {
  if (n_jobs == 0) return cudaSuccess;
  pack_kernel<<<(unsigned)n_jobs, 128, 0, s>>>(grids, panels, n_panels, hint, rows, ops, ops_lo, packed);
  return cudaGetLastError();
}

cudaError_t launch_contract_ws(const DevGrid* grids, const MmaBlock* blocks, const GemmItem* items,
                               const int* cta_begin, int n_ctas, const Panel* panels, const PairTile* ptiles,
                               const float* ops, const float* ops_lo, const uint8_t* packed, float2* part, int* status,
                               uint64_t wait_ns, const int* hold, cudaStream_t s) {
  if (n_ctas == 0) return cudaSuccess;
  contract_ws_kernel<<<n_ctas, ws::kThreads, ws_smem_bytes(), s>>>(grids, blocks, items, cta_begin, panels, ptiles, ops,
                                                                   ops_lo, packed, part, status, wait_ns, hold);
  return cudaGetLastError();
}

cudaError_t launch_ri_pack(const Panel* panels, int64_t n_jobs, const double* srcA, const double* srcB, int n,
                           uint8_t* packed, cudaStream_t s) {
  if (n_jobs == 0) return cudaSuccess;
  ri_pack_kernel<<<(unsigned)n_jobs, 128, 0, s>>>(panels, srcA, srcB, n, packed);
  return cudaGetLastError();
}

cudaError_t launch_reduce_mixed(const DevGrid* grids, const MmaBlock* blocks, int n_blocks, const int64_t* elem_begin,
                                int64_t e0, int64_t e1, const short2* rows, const double* rowc, const float2* part,
                                double* res, cudaStream_t s) {
  if (e1 <= e0) return cudaSuccess;
  reduce_mixed_kernel<<<(unsigned)((e1 - e0 + 255) / 256), 256, 0, s>>>(grids, blocks, n_blocks, elem_begin, e0, e1,
                                                                         rows, rowc, part, res);
  return cudaGetLastError();
}


}  // namespace psq
