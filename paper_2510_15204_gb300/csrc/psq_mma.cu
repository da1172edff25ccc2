// Mixed-precision path of the PS quadrature on sm_103a:
//  * node tables: the PS grid is a tensor product in (mu, nu, phi) per volume element, so the
//    per-node trigonometric factors (Section 2.1, eqs 2-6, 10-11) are computed once per grid
//    row in FP64 (nodes_kernel) and combined per point;
//  * eval_mixed_kernel: point weights, focal distances and offsets in FP32 from the FP64
//    tables (the cancellation-free forms need no FP64), the third-centre offset in FP64
//    (it cancels near that centre), STOs (eq 1), their kinetic operand and the aux
//    potentials (eq 16, incomplete gamma by its positive series below x = k) in FP32 as
//    functions of x = zeta r (x from an FP32 hi+lo scale, first-order corrected); every
//    constant factor of a row is left to FP64;
//  * pack_kernel: every operand row that a contraction tile reads whole is scaled by a power
//    of two per 128-point window (from the window's maximum) and cut into four integer
//    slices of at most 8 bits (exact in BF16), stored as the tcgen05 shared-memory image;
//  * contract_ws_kernel: the weighted contraction of eq 9 on tcgen05 tensor cores.  Packed
//    tiles arrive by bulk copies; the 3-index operand chi_i chi_j is formed and sliced in
//    shared memory from staged basis rows.  Per K step of 16 points four MMAs (A slice i
//    against B slices 0..3-i, contiguous in shared memory) accumulate the slice products of
//    orders 0..3 into four FP32 TMEM accumulators; all partial sums are integers below 2^23,
//    so the FP32 accumulation is exact.  After each window the accumulators are scaled back
//    and added into double-float (FP32 hi + lo) registers; each work item writes its point
//    range's (hi, lo) sums, and reduce_mixed_kernel adds the ranges in FP64 and applies the
//    FP64 constants of each row and column (normalisations, powers of zeta, a^3), which the
//    FP32 values omit.
#include "psq_internal.h"

#include <cuda_bf16.h>

#include <cstdint>

namespace psq {

// ------------------------------------------------------------------ node tables

__constant__ double c_glx2[kMaxQ + 1][kMaxQ];
__constant__ double c_glw2[kMaxQ + 1][kMaxQ];
__constant__ float c_klmf[(kMaxL + 1) * (kMaxL + 1)];
__constant__ float c_factf[2 * kMaxN + 4];
__constant__ float c_rcpf[128];  // 1/n

void upload_mixed_tables(const double* x, const double* w, const double* klm) {
  cudaMemcpyToSymbol(c_glx2, x, sizeof(double) * (kMaxQ + 1) * kMaxQ);
  cudaMemcpyToSymbol(c_glw2, w, sizeof(double) * (kMaxQ + 1) * kMaxQ);
  float k[(kMaxL + 1) * (kMaxL + 1)];
  for (int i = 0; i < (kMaxL + 1) * (kMaxL + 1); ++i) k[i] = (float)klm[i];
  cudaMemcpyToSymbol(c_klmf, k, sizeof(k));
  float f[2 * kMaxN + 4];
  double fd = 1.0;
  f[0] = 1.0f;
  for (int i = 1; i < 2 * kMaxN + 4; ++i) {
    fd *= i;
    f[i] = (float)fd;
  }
  cudaMemcpyToSymbol(c_factf, f, sizeof(f));
  float r[128];
  r[0] = 0.0f;
  for (int i = 1; i < 128; ++i) r[i] = (float)(1.0 / i);
  cudaMemcpyToSymbol(c_rcpf, r, sizeof(r));
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
  NodeEntry o;
  o.v = v;
  o.w = h * c_glw2[Q][q];
  if (dim == 0) {
    o.s = sinh(v);
    o.c = cosh(v);
    const double sh2 = sinh(0.5 * v);
    o.h2 = sh2 * sh2;
    o.g2 = 0.0;
  } else {
    sincos(v, &o.s, &o.c);
    double s2, c2;
    sincos(0.5 * v, &s2, &c2);
    o.h2 = s2 * s2;
    o.g2 = c2 * c2;
  }
  tab[g.nt_off + e] = o;
}

// ------------------------------------------------------------------ mixed evaluation

// Unnormalised real harmonics Yu_lm(u) = Q_l^|m|(u_z) {Re, Im}(u_x + i u_y)^|m| (the norms K_lm
// are applied in FP64 with the other row constants), index l*l + l + m.
__device__ __forceinline__ void real_ylm_u(int lmax, float ux, float uy, float uz, float* Y) {
  float C[kMaxL + 1], S[kMaxL + 1];
  C[0] = 1.0f; S[0] = 0.0f;
  for (int m = 1; m <= lmax; ++m) {
    C[m] = ux * C[m - 1] - uy * S[m - 1];
    S[m] = ux * S[m - 1] + uy * C[m - 1];
  }
  float dfact = 1.0f;
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) dfact *= (float)(2 * m - 1);
    float q2 = 0.0f, q1 = dfact;
    for (int l = m; l <= lmax; ++l) {
      float q;
      if (l == m) q = dfact;
      else if (l == m + 1) q = (float)(2 * m + 1) * uz * dfact;
      else q = ((float)(2 * l - 1) * uz * q1 - (float)(l + m - 1) * q2) * c_rcpf[l - m];
      if (l > m) { q2 = q1; q1 = q; }
      const int base = l * l + l;
      if (m == 0) {
        Y[base] = q;
      } else {
        Y[base + m] = q * C[m];
        Y[base - m] = q * S[m];
      }
    }
  }
}

__device__ __forceinline__ float ipowf(float x, int n) {
  float r = 1.0f;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

// Radial factors as functions of x = zeta r (row constants carry the powers of zeta):
//   chi: x^(n-1) e^-x;  lap chi: [(n(n-1) - l(l+1))/x^2 - 2n/x + 1] x^(n-1) e^-x;
//   V^P: gamma(n+l+2, x)/x^(l+1) + Gamma(n-l+1, x) x^l.
// x = xh + xl (FP32 pair); the result is corrected to first order in xl.
__device__ __forceinline__ float radial_x_e(int kind, int n, int l, float xh, float xl, float ex, float ix) {
  if (kind == 2) {
    const int k1 = n + l + 2, k2 = n - l + 1;
    float inner;
    if (xh < (float)k1) {
      float term = c_rcpf[k1], sum = term;
      for (int i = 1; i < 120 - k1; ++i) {
        term *= xh * c_rcpf[k1 + i];
        sum += term;
        if (term <= 3e-8f * sum) break;
      }
      inner = ipowf(xh, n + 1) * ex * sum;
    } else {
      float t = 1.0f, s = 1.0f;
      for (int j = 1; j < k1; ++j) { t *= xh * c_rcpf[j]; s += t; }
      const float f = c_factf[k1 - 1];
      inner = (f - f * ex * s) * ipowf(ix, l + 1);
    }
    float t = 1.0f, s = 1.0f;
    for (int j = 1; j < k2; ++j) { t *= xh * c_rcpf[j]; s += t; }
    const float outer = c_factf[k2 - 1] * ex * s * ipowf(xh, l);
    const float dh = ((float)l * outer - (float)(l + 1) * inner) * ix;  // dh/dx
    return fmaf(xl, dh, inner + outer);
  }
  const float g = ipowf(xh, n - 1) * ex;
  const float gc = g * fmaf(xl, (float)(n - 1) * ix - 1.0f, 1.0f);
  if (kind == 0) return gc;
  const float A = (float)(n * (n - 1) - l * (l + 1));
  const float f = fmaf(fmaf(A, ix, -2.0f * n), ix, 1.0f);
  const float df = (2.0f * n - 2.0f * A * ix) * ix * ix;
  return fmaf(xl, df, f) * gc;
}

__device__ __forceinline__ float radial_x(int kind, int n, int l, float xh, float xl) {
  return radial_x_e(kind, n, l, xh, xl, expf(-xh), 1.0f / xh);
}

// Rows of the shells [s0, s1) of one centre: kind 0 chi, 1 lap chi, 2 V^P.  xi[k] is the
// (hi, lo) FP32 pair of the scale that turns rho into x for shell s0 + k.
__device__ __forceinline__ void eval_shells_x(const DevShell* __restrict__ sh, const float2* __restrict__ xi,
                                              int s0, int s1, float rho, const float* Y, float* __restrict__ out,
                                              int64_t ld, int64_t p, int row0, int kind) {
  for (int s = s0; s < s1; ++s) {
    const DevShell q = sh[s];
    const float2 z = xi[s - s0];
    const float xh = z.x * rho;
    const float xl = fmaf(z.x, rho, -xh) + z.y * rho;
    const float radial = radial_x(kind, q.n, q.l, xh, xl);
    const int base = q.l * q.l + q.l;
    for (int m = -q.l; m <= q.l; ++m) out[(int64_t)(row0 + q.fn0 + q.l + m) * ld + p] = radial * Y[base + m];
  }
}

// The same for two row kinds of the same shells (chi and lap chi, or chi and V^P) at once:
// x, e^-x and 1/x are shared.
__device__ __forceinline__ void eval_shells_x2(const DevShell* __restrict__ sh, const float2* __restrict__ xi,
                                               int s0, int s1, float rho, const float* Y, float* __restrict__ out,
                                               int64_t ld, int64_t p, int row_a, int kind_a, int row_b,
                                               int kind_b) {
  for (int s = s0; s < s1; ++s) {
    const DevShell q = sh[s];
    const float2 z = xi[s - s0];
    const float xh = z.x * rho;
    const float xl = fmaf(z.x, rho, -xh) + z.y * rho;
    const float ex = expf(-xh), ix = 1.0f / xh;
    const float ra = radial_x_e(kind_a, q.n, q.l, xh, xl, ex, ix);
    const float rb = radial_x_e(kind_b, q.n, q.l, xh, xl, ex, ix);
    const int base = q.l * q.l + q.l;
    for (int m = -q.l; m <= q.l; ++m) {
      out[(int64_t)(row_a + q.fn0 + q.l + m) * ld + p] = ra * Y[base + m];
      out[(int64_t)(row_b + q.fn0 + q.l + m) * ld + p] = rb * Y[base + m];
    }
  }
}

__device__ __forceinline__ int shells_lmax_f(const DevShell* sh, int s0, int s1) {
  int l = 0;
  for (int s = s0; s < s1; ++s) l = max(l, sh[s].l);
  return l;
}

// v -> R v with R held as an FP32 pair (hi + lo); returns |Rv| and the unit vector.
__device__ __forceinline__ float rotate_unit(const DevGrid& g, float vx, float vy, float vz, float* u) {
  float d[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float hi = fmaf(g.Rh[c * 3], vx, fmaf(g.Rh[c * 3 + 1], vy, g.Rh[c * 3 + 2] * vz));
    const float lo = fmaf(g.Rl[c * 3], vx, fmaf(g.Rl[c * 3 + 1], vy, g.Rl[c * 3 + 2] * vz));
    d[c] = hi + lo;
  }
  const float n2 = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
  const float inv = rsqrtf(n2);
  u[0] = d[0] * inv; u[1] = d[1] * inv; u[2] = d[2] * inv;
  return n2 * inv;
}

// One thread per point.  The weight w = a^3 [G G G sinh mu sin nu (sinh^2 mu + sin^2 nu)]
// and r_A = 2a rho_A, r_B = 2a rho_B are written without their per-grid constants (a^3,
// a^2/2), which are applied in FP64 after the contraction; functions likewise.
__global__ void __launch_bounds__(128) eval_mixed_kernel(LaunchTables t, const NodeEntry* __restrict__ tab,
                                                         const float2* __restrict__ xi_tab,
                                                         float* __restrict__ ops) {
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
  const NodeEntry Mu = tab[g.nt_off + ri * g.q_mu + qi];
  const NodeEntry Nu = tab[g.nt_off + nmu + rj * g.q_nu + qj];
  const NodeEntry Ph = tab[g.nt_off + nmu + nnu + rk * g.q_phi + qk];
  const float sh = (float)Mu.s, s2m = (float)Mu.h2;
  const float sn = (float)Nu.s, cs = (float)Nu.c, s2n = (float)Nu.h2, c2n = (float)Nu.g2;
  const float sp = (float)Ph.s, cp = (float)Ph.c;
  const float w = dead ? 0.0f : (float)(Mu.w * Nu.w * Ph.w) * sh * sn * fmaf(sh, sh, sn * sn);
  const float rhoA = s2m + s2n, rhoB = s2m + c2n;
  // pair-frame offsets from A and B, in units of a: (sh sn cos phi, sh sn sin phi, 2(s2m cs -+ ...))
  const float xs = sh * sn * cp, ys = sh * sn * sp;
  float uA[3], uB[3], uC[3] = {0.f, 0.f, 1.f};
  rotate_unit(g, xs, ys, 2.0f * (s2m * cs - s2n), uA);
  rotate_unit(g, xs, ys, 2.0f * (s2m * cs + c2n), uB);
  float rC = 1.0f;
  if (g.C >= 0) {
    // offset from the third centre in the pair frame, FP64: it cancels near that centre
    const double X = g.a * Mu.s * Nu.s * Ph.c - g.xc;
    const double Yv = g.a * Mu.s * Nu.s * Ph.s;
    const double Z = g.a * Mu.c * Nu.c - g.zc;
    rC = rotate_unit(g, (float)X, (float)Yv, (float)Z, uC);
  }
  float* base = ops + g.op_off;
  const int64_t ld = g.ld;
  if (g.row_W >= 0) {
    base[(int64_t)(g.row_W + 0) * ld + p] = w;
    base[(int64_t)(g.row_W + 1) * ld + p] = w / rhoA;
    base[(int64_t)(g.row_W + 2) * ld + p] = w / rhoB;
    base[(int64_t)(g.row_W + 3) * ld + p] = g.C >= 0 ? w / rC : 0.0f;
  }
  const float2* xi = xi_tab + g.xi_off;  // basis A, basis B, aux c0, aux c1 shells
  const int nbA = g.shb_A1 - g.shb_A0, nbB = g.shb_B1 - g.shb_B0, na0 = g.sha_1 - g.sha_0;
  float Y[(kMaxL + 1) * (kMaxL + 1)];
  if (g.row_F >= 0 || g.row_L >= 0) {
    for (int c = 0; c < 2; ++c) {
      const int s0 = c == 0 ? g.shb_A0 : g.shb_B0, s1 = c == 0 ? g.shb_A1 : g.shb_B1;
      if (s1 <= s0) continue;
      const float rho = c == 0 ? rhoA : rhoB;
      const float* u = c == 0 ? uA : uB;
      real_ylm_u(shells_lmax_f(t.bshell, s0, s1), u[0], u[1], u[2], Y);
      const int roff = c == 0 ? 0 : g.nFA;
      const float2* z = xi + (c == 0 ? 0 : nbA);
      if (g.row_F >= 0 && g.row_L >= 0) {
        eval_shells_x2(t.bshell, z, s0, s1, rho, Y, base, ld, p, g.row_F + roff, 0, g.row_L + roff, 1);
      } else {
        if (g.row_F >= 0) eval_shells_x(t.bshell, z, s0, s1, rho, Y, base, ld, p, g.row_F + roff, 0);
        if (g.row_L >= 0) eval_shells_x(t.bshell, z, s0, s1, rho, Y, base, ld, p, g.row_L + roff, 1);
      }
    }
  }
  if (g.row_G >= 0 || g.row_U >= 0) {
    int roff = 0;
    for (int c = 0; c < 2; ++c) {
      const int s0 = c == 0 ? g.sha_0 : g.sha_2, s1 = c == 0 ? g.sha_1 : g.sha_3;
      const int atom = c == 0 ? g.aux_c0 : g.aux_c1;
      if (atom < 0 || s1 <= s0) continue;
      const float* u;
      float rho;
      if (atom == g.A) { u = uA; rho = rhoA; }
      else if (atom == g.B) { u = uB; rho = rhoB; }
      else { u = uC; rho = rC; }
      real_ylm_u(shells_lmax_f(t.ashell, s0, s1), u[0], u[1], u[2], Y);
      const float2* z = xi + nbA + nbB + (c == 0 ? 0 : na0);
      if (g.row_G >= 0 && g.row_U >= 0) {
        eval_shells_x2(t.ashell, z, s0, s1, rho, Y, base, ld, p, g.row_G + roff, 0, g.row_U + roff, 2);
      } else {
        if (g.row_G >= 0) eval_shells_x(t.ashell, z, s0, s1, rho, Y, base, ld, p, g.row_G + roff, 0);
        if (g.row_U >= 0) eval_shells_x(t.ashell, z, s0, s1, rho, Y, base, ld, p, g.row_U + roff, 2);
      }
      int nf = 0;
      for (int s = s0; s < s1; ++s) nf += 2 * t.ashell[s].l + 1;
      roff += nf;
    }
  }
}

// ------------------------------------------------------------------ tcgen05 contraction

namespace mma {

constexpr int kM = 128;         // tile rows (pairs, or the bigger side of a 2-index block)
constexpr int kTileN = 64;       // tile columns
constexpr int kChunk = 64;      // points per scale window and smem stage (128 bytes of BF16)
constexpr int kSlices = 4;      // 8-bit integer slices per operand value (orders 0..3 kept)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(16 >> 4) << 16;     // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;             // descriptor version for sm_100 family
  d |= (uint64_t)2 << 61;             // SWIZZLE_128B
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

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase of the given parity; gives up (false) after kWaitNs nanoseconds, or
// early once *abort (if given) is set by another role of the CTA.
constexpr uint64_t kWaitNs = 4000000000ull;
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, const int* abort = nullptr) {
  if (mbar_try(mbar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try(mbar, parity)) return true;
    if ((it & 255u) == 0) {
      if (abort && *(volatile const int*)abort) return false;
      if (global_ns() - t0 > kWaitNs) return false;
    }
  }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
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

namespace mma {

// Eight values, already scaled into (-128, 128), as four planes of 8-bit integers in BF16:
// plane k holds the nearest integer of what planes 0..k-1 left, times 256^k.  w[k] is the
// 16-byte group of plane k.
__device__ __forceinline__ void slice8(const float* v, float sc, uint4* w) {
  uint32_t o[kSlices][4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float r0 = v[2 * q] * sc, r1 = v[2 * q + 1] * sc;
#pragma unroll
    for (int k = 0; k < kSlices; ++k) {
      const float a0 = rintf(r0), a1 = rintf(r1);
      const __nv_bfloat162 p = __floats2bfloat162_rn(a0, a1);
      o[k][q] = *reinterpret_cast<const uint32_t*>(&p);
      r0 = (r0 - a0) * 256.0f;
      r1 = (r1 - a1) * 256.0f;
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

// Byte offset of 16-byte group j of row r in a 128-byte-row swizzled operand tile.
__device__ __forceinline__ uint32_t swz(int r, int j) { return (uint32_t)r * 128u + ((uint32_t)(j ^ (r & 7)) << 4); }

}  // namespace mma

// One packing job: 64 rows of one tile of one panel, one 128-point window; eight threads per
// row, thread (r, e) holding points [16 (e % 4), 16 (e % 4) + 16) of chunk e / 4.
struct PackJob {
  float v[16];
  int pn, t, w, r, c, qq;
};

// Decodes job and loads its values (source row times its weight row, zeros past K).
__device__ __forceinline__ void pack_load(int64_t job, const DevGrid* __restrict__ grids,
                                          const Panel* __restrict__ panels, int n_panels,
                                          const short2* __restrict__ rows, const float* __restrict__ ops,
                                          PackJob& J) {
  int lo = 0, hi = n_panels;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (panels[mid].job_begin <= job) lo = mid; else hi = mid;
  }
  const Panel& pn = panels[lo];
  const int gsh = pn.tr >> 7;  // 64-row groups per tile: 1 (tr 64) or 2 (tr 128)
  const int lj = (int)(job - pn.job_begin);  // jobs of one panel < 2^31 (one launch's grid)
  const int tw = lj >> gsh, grp = lj & gsh;
  J.pn = lo;
  J.t = tw / pn.nwin;
  J.w = tw - J.t * pn.nwin;
  J.r = 64 * grp + (threadIdx.x >> 3);
  const int e8 = threadIdx.x & 7;
  J.c = 2 * J.w + (e8 >> 2);
  J.qq = e8 & 3;
  const DevGrid& g = grids[pn.grid];
  const int row = J.t * pn.tr + J.r;
  const int64_t k0 = 64 * (int64_t)J.c + 16 * J.qq;
  const float* src = nullptr;
  const float* mul = nullptr;
  if (row < pn.nrows && J.c < pn.nch) {
    const short2 q = rows[pn.rows_off + row];
    src = ops + g.op_off + (int64_t)q.x * g.ld + k0;
    if (q.y >= 0) mul = ops + g.op_off + (int64_t)q.y * g.ld + k0;
  }
  const int64_t left = g.K - k0;
  if (src && left >= 16) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    const float4* m4 = reinterpret_cast<const float4*>(mul);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float4 a = __ldg(s4 + i);
      if (mul) {
        const float4 bb = __ldg(m4 + i);
        a.x *= bb.x; a.y *= bb.y; a.z *= bb.z; a.w *= bb.w;
      }
      J.v[4 * i] = a.x; J.v[4 * i + 1] = a.y; J.v[4 * i + 2] = a.z; J.v[4 * i + 3] = a.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) J.v[i] = (src && i < left) ? src[i] * (mul ? mul[i] : 1.0f) : 0.0f;
  }
}

// The row's window scale (the eight threads of the row share it), its exponent, and the
// four planes of this thread's 16 points.
__device__ __forceinline__ void pack_store(const PackJob& J, const Panel* __restrict__ panels,
                                           uint8_t* __restrict__ packed) {
  using namespace mma;
  const Panel& pn = panels[J.pn];
  float mx = 0.0f;
#pragma unroll
  for (int i = 0; i < 16; ++i) mx = fmaxf(mx, fabsf(J.v[i]));
  const unsigned m8 = 0xffu << ((threadIdx.x & 31) & ~7u);
  mx = fmaxf(mx, __shfl_xor_sync(m8, mx, 1));
  mx = fmaxf(mx, __shfl_xor_sync(m8, mx, 2));
  mx = fmaxf(mx, __shfl_xor_sync(m8, mx, 4));
  const int e = row_exponent(mx);
  if ((threadIdx.x & 7) == 0)
    *reinterpret_cast<int*>(packed + pn.exp_off + (((int64_t)J.t * pn.nwin + J.w) * pn.tr + J.r) * 4) = e;
  const int rt = min(pn.tr, pn.nrows - J.t * pn.tr);
  if (J.c >= pn.nch || J.r >= rt) return;
  const float sc = e == kZeroExp ? 0.0f : pow2f(7 - e);
  uint8_t* dst = packed + pn.pack_off + (int64_t)J.t * pn.nch * (4 * pn.tr * 128) + (int64_t)J.c * (4 * rt * 128);
  const int plane = rt * 128;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    uint4 wv[kSlices];
    slice8(J.v + 8 * j, sc, wv);
#pragma unroll
    for (int k = 0; k < kSlices; ++k) *reinterpret_cast<uint4*>(dst + k * plane + swz(J.r, 2 * J.qq + j)) = wv[k];
  }
}

// One CTA of 512 threads per packing job (panel, tile, 128-point window, 64-row group).
// (Two jobs per CTA with all loads issued first measured 1-6% slower: fewer CTAs fit.)
__global__ void __launch_bounds__(512, 3) pack_kernel(const DevGrid* __restrict__ grids, const Panel* __restrict__ panels,
                                                   int n_panels, const short2* __restrict__ rows,
                                                   const float* __restrict__ ops, uint8_t* __restrict__ packed) {
  PackJob J;
  pack_load(blockIdx.x, grids, panels, n_panels, rows, ops, J);
  pack_store(J, panels, packed);
}

// The same packed-panel image from FP64 operand rows (row-major, stride n): used for the
// RI 4-index product, whose operand rows are the (P|ij) columns after the forward solve.
// Panel k's rows start at src[k]; jobs as in pack_kernel, both panels' jobs in one launch.
// The digits are taken in FP64 (exact: the value times a power of two, rounded digit by
// digit), each exact in BF16.
__global__ void __launch_bounds__(512, 2) ri_pack_kernel(const Panel* __restrict__ panels, const double* __restrict__ srcA,
                                                      const double* __restrict__ srcB, int n, uint8_t* __restrict__ packed) {
  using namespace mma;
  const int64_t job = blockIdx.x;
  const int k = panels[1].job_begin <= job ? 1 : 0;
  const Panel& pn = panels[k];
  const double* src = k ? srcB : srcA;
  const int gsh = pn.tr >> 7;
  const int lj = (int)(job - pn.job_begin);
  const int tw = lj >> gsh, grp = lj & gsh;
  const int t = tw / pn.nwin, w = tw - t * pn.nwin;
  const int r = 64 * grp + (threadIdx.x >> 3), e8 = threadIdx.x & 7;
  const int c = 2 * w + (e8 >> 2), qq = e8 & 3;
  const int row = t * pn.tr + r;
  const int k0 = 64 * c + 16 * qq;
  double v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = 0.0;
  if (row < pn.nrows && c < pn.nch) {
    const double* rp = src + (int64_t)row * n + k0;
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (k0 + i < n) v[i] = rp[i];
  }
  double mx = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) mx = fmax(mx, fabs(v[i]));
  const unsigned m8 = 0xffu << ((threadIdx.x & 31) & ~7u);
  mx = fmax(mx, __shfl_xor_sync(m8, mx, 1));
  mx = fmax(mx, __shfl_xor_sync(m8, mx, 2));
  mx = fmax(mx, __shfl_xor_sync(m8, mx, 4));
  int e = 0;
  if (mx > 0.0) frexp(mx, &e);  // mx < 2^e <= 2 mx
  if (!(mx > 0.0) || e < -110) e = kZeroExp;
  if (e8 == 0) *reinterpret_cast<int*>(packed + pn.exp_off + (((int64_t)t * pn.nwin + w) * pn.tr + r) * 4) = e;
  const int rt = min(pn.tr, pn.nrows - t * pn.tr);
  if (c >= pn.nch || r >= rt) return;
  const double sc = e == kZeroExp ? 0.0 : ldexp(1.0, 7 - e);
  uint8_t* dst = packed + pn.pack_off + (int64_t)t * pn.nch * (4 * pn.tr * 128) + (int64_t)c * (4 * rt * 128);
  const int plane = rt * 128;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    uint32_t o[kSlices][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double x0 = v[8 * j + 2 * q] * sc, x1 = v[8 * j + 2 * q + 1] * sc;
#pragma unroll
      for (int d = 0; d < kSlices; ++d) {
        const double a0 = rint(x0), a1 = rint(x1);
        const __nv_bfloat162 pr = __floats2bfloat162_rn((float)a0, (float)a1);
        o[d][q] = *reinterpret_cast<const uint32_t*>(&pr);
        x0 = (x0 - a0) * 256.0;
        x1 = (x1 - a1) * 256.0;
      }
    }
#pragma unroll
    for (int d = 0; d < kSlices; ++d)
      *reinterpret_cast<uint4*>(dst + d * plane + swz(r, 2 * qq + j)) = make_uint4(o[d][0], o[d][1], o[d][2], o[d][3]);
  }
}

// ------------------------------------------------------------------ warp-specialised contraction
//
// One persistent CTA per SM, 512 threads, working through tiles (128 A rows x <= 64 B
// columns x a range of 128-point windows):
//   warp 4       loader: bulk copies of the packed A tile (and packed B tile) of every 64-point
//                chunk into a two-stage ring, and of the staged basis rows of formed B tiles
//                (one copy per row and window);
//   warps 0-3, 6, 7  producers: for a formed B, column c of the tile = product of two staged
//                rows; per window they find each column's scale, then slice chunk by chunk
//                into the B stages, so that the MMAs of one chunk overlap the slicing of the
//                next (for a packed B they only pass each chunk on);
//   warp 5       MMA issue: per chunk 4 K-steps x 10 slice products (orders 0..3) into the
//                window's TMEM accumulator set (4 orders x 64 columns; two sets);
//   warps 8-15   fold: per window, the four order sums of their TMEM lane quadrant and column
//                half, scaled by the window's row and column exponents, into double-float
//                registers; at the end of the tile, (hi, lo) partials to global memory.
// All integer sums stay below 2^23 (|slice| <= 128, <= 4 products per order, 128 points), so
// the FP32 accumulators hold them exactly.  Every wait is bounded; a timeout sets *status and
// the CTA's abort flag, and each role leaves its loops at its next wait.

namespace ws {

constexpr int kThreads = 512;
constexpr int kLoadWarp = 4, kMmaWarp = 5, kFoldWarp0 = 8;
constexpr int kRawStride = 132;  // floats per staged row: 128 points + 4 (bank spread)

struct Smem {
  alignas(1024) uint8_t a[2][mma::kSlices][mma::kM * 128];
  alignas(1024) uint8_t b[2][mma::kSlices][mma::kTileN * 128];
  alignas(16) float raw[2][kPairTileRows][kRawStride];
  int eb[2][mma::kTileN];
  float sbw[8][mma::kTileN];  // fold warp k: the column scales of the current window
  alignas(8) uint64_t a_full[2], b_ready[2], stage_free[2], tmem_full[2], tmem_free[2], raw_full[2], raw_free[2];
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

__device__ __forceinline__ bool wait(uint64_t* b, uint32_t parity, const int* abort = nullptr) {
  return mma::mbar_wait(mma::smem_u32(b), parity, abort);
}

// What every role needs to know about an item.
struct Geo {
  const MmaBlock* blk;
  int64_t K;
  int nch, nwin, w0, w1;
  int nt, ntp;      // B columns of the tile and their multiple of 16
  bool formed;
  const PairTile* pt;
};

__device__ __forceinline__ Geo geo(const GemmItem& it, const MmaBlock* blocks, const DevGrid* grids,
                                   const PairTile* ptiles) {
  Geo q;
  q.blk = blocks + it.block;
  const MmaBlock& b = *q.blk;
  q.K = grids[b.grid].K;
  q.nch = (int)((q.K + 63) / 64);
  q.nwin = (q.nch + 1) / 2;
  q.w0 = it.chunk * b.win_per;
  q.w1 = min(q.nwin, q.w0 + b.win_per);
  q.formed = b.b_panel < 0;
  q.pt = q.formed ? ptiles + b.ptile_off + it.tn : nullptr;
  q.nt = q.formed ? q.pt->ncols : min(mma::kTileN, b.n - it.tn * mma::kTileN);
  q.ntp = (q.nt + 15) & ~15;
  return q;
}

__device__ __forceinline__ void fail(Smem& sm, int* status, int code) {
  *(volatile int*)&sm.abort = 1;
  atomicCAS(status, 0, code);  // the first failure's code stays
}

__device__ __forceinline__ bool aborted(Smem& sm) { return *(volatile int*)&sm.abort != 0; }

}  // namespace ws

__global__ void __launch_bounds__(ws::kThreads, 1)
    contract_ws_kernel(const DevGrid* __restrict__ grids, const MmaBlock* __restrict__ blocks,
                       const GemmItem* __restrict__ items, const int* __restrict__ cta_begin,
                       const Panel* __restrict__ panels,
                       const PairTile* __restrict__ ptiles, const float* __restrict__ ops,
                       const uint8_t* __restrict__ packed, float2* __restrict__ part, int* __restrict__ status) {
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
    for (int s = 0; s < 2; ++s) {
      ws::mbar_init(&sm.a_full[s], 1);
      ws::mbar_init(&sm.b_ready[s], 6);
      ws::mbar_init(&sm.stage_free[s], 1);
      ws::mbar_init(&sm.tmem_full[s], 1);
      ws::mbar_init(&sm.tmem_free[s], 8);
      ws::mbar_init(&sm.raw_full[s], 1);
      ws::mbar_init(&sm.raw_free[s], 6);
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
    bool run = true;                 // warp-uniform
    int last_a = -1, last_raw = -1;  // last issued chunk / formed window (for the drain)
    for (int ii = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1]; ii < ie && run; ++ii) {
      const GemmItem it = items[ii];
      const ws::Geo q = ws::geo(it, blocks, grids, ptiles);
      const MmaBlock& b = *q.blk;
      const DevGrid& g = grids[b.grid];
      const Panel& pa = panels[b.a_panel];
      const Panel* pb = q.formed ? nullptr : panels + b.b_panel;
      for (int win = q.w0; win < q.w1 && run; ++win, ++w) {
        const int nck = min(2, q.nch - 2 * win);
        if (q.formed) {
          const int rb = rw & 1;
          const bool ok = rw < 2 || ws::wait(&sm.raw_free[rb], ((rw - 2) >> 1) & 1, &sm.abort);
          run = __all_sync(kFull, ok && !ws::aborted(sm));
          if (!run) { ws::fail(sm, status, 4); break; }
          const int nr = q.pt->nrows;
          if (lane == 0) ws::mbar_expect_tx(&sm.raw_full[rb], (uint32_t)nr * 512u);
          __syncwarp();
          if (lane < nr)
            ws::bulk_g2s(sm.raw[rb][lane], ops + g.op_off + (int64_t)q.pt->rows[lane] * g.ld + 128 * (int64_t)win,
                         512u, &sm.raw_full[rb]);
          last_raw = (int)rw;
          ++rw;
        }
        for (int j = 0; j < nck; ++j, ++c) {
          const int s = c & 1, ch = 2 * win + j;
          const bool ok = c < 2 || ws::wait(&sm.stage_free[s], ((c - 2) >> 1) & 1, &sm.abort);
          run = __all_sync(kFull, ok && !ws::aborted(sm));
          if (!run) { ws::fail(sm, status, 4); break; }
          // the stored rows of the tiles, one bulk copy per plane (lanes 0-3: A, 4-7: B)
          const int ra = min(kM, pa.nrows - it.tm * kM);
          const int rbw = pb ? min(kTileN, pb->nrows - it.tn * kTileN) : 0;
          if (lane == 0) ws::mbar_expect_tx(&sm.a_full[s], 4u * 128u * (uint32_t)(ra + rbw));
          __syncwarp();
          if (lane < 4) {
            const uint8_t* src = packed + pa.pack_off + (int64_t)it.tm * pa.nch * (4 * kM * 128) +
                                 (int64_t)ch * (4 * ra * 128) + (int64_t)lane * ra * 128;
            ws::bulk_g2s(sm.a[s][lane], src, 128u * (uint32_t)ra, &sm.a_full[s]);
          } else if (lane < 8 && pb) {
            const int k = lane - 4;
            const uint8_t* src = packed + pb->pack_off + (int64_t)it.tn * pb->nch * (4 * kTileN * 128) +
                                 (int64_t)ch * (4 * rbw * 128) + (int64_t)k * rbw * 128;
            ws::bulk_g2s(sm.b[s][k], src, 128u * (uint32_t)rbw, &sm.a_full[s]);
          }
          __syncwarp();
          last_a = (int)c;
        }
      }
    }
    // drain: nothing may still be copying into shared memory when the CTA exits
    if (!run) {
      for (int k = last_a; k >= 0 && k > last_a - 2; --k) ws::wait(&sm.a_full[k & 1], (k >> 1) & 1);
      for (int k = last_raw; k >= 0 && k > last_raw - 2; --k) ws::wait(&sm.raw_full[k & 1], (k >> 1) & 1);
    }
  } else if (warp < 4 || warp == 6 || warp == 7) {
    // ------------------------------------------------------------------ producers
    // Six warps.  A window's 64 columns are 16 rounds of 4 columns; producer warp pw takes
    // rounds pw, pw + 6, pw + 12.  In a round, eight lanes share a column, lane g owning
    // points 8g..8g+7 of both chunks: they read contiguous 32-byte pieces of the column's two
    // rows (one row per quarter warp), find the column's window maximum by shuffles, and
    // write the eight 16-byte groups of the column's 128-byte row in each plane.
    const int pw = warp < 4 ? warp : warp - 2;
    const int g = lane & 7;
    const unsigned col_mask = 0xffu << (lane & 24);
    bool run = true;  // warp-uniform
    for (int ii = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1]; ii < ie && run; ++ii) {
      const GemmItem it = items[ii];
      const ws::Geo q = ws::geo(it, blocks, grids, ptiles);
      if (!q.formed) {
        // packed B: the loader brings it; b_ready still completes one phase per chunk
        for (int win = q.w0; win < q.w1 && run; ++win, ++w) {
          const int nck = min(2, q.nch - 2 * win);
          for (int j = 0; j < nck; ++j, ++c) {
            const bool ok = c < 2 || ws::wait(&sm.stage_free[c & 1], ((c - 2) >> 1) & 1, &sm.abort);
            run = __all_sync(kFull, ok && !ws::aborted(sm));
            if (!run) { ws::fail(sm, status, 5); break; }
            if (lane == 0) ws::mbar_arrive(&sm.b_ready[c & 1]);
          }
        }
        continue;
      }
      // this lane's columns (one per round) and their two rows
      int colr[3], dxr[3], dyr[3];
      bool validr[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int R = pw + 6 * r;
        colr[r] = 4 * R + (lane >> 3);
        validr[r] = R < 16 && colr[r] < q.nt;
        dxr[r] = validr[r] ? q.pt->dx[colr[r]] : 0;
        dyr[r] = validr[r] ? q.pt->dy[colr[r]] : 0;
      }
      for (int win = q.w0; win < q.w1 && run; ++win, ++w, ++rw) {
        const int nck = min(2, q.nch - 2 * win);
        const int rb = rw & 1, set = w & 1;
        bool ok = ws::wait(&sm.raw_full[rb], (rw >> 1) & 1, &sm.abort);
        if (ok && w >= 2) ok = ws::wait(&sm.tmem_free[set], ((w - 2) >> 1) & 1, &sm.abort);
        run = __all_sync(kFull, ok && !ws::aborted(sm));
        if (!run) { ws::fail(sm, status, 5); break; }
        const int64_t wleft = q.K - 128 * (int64_t)win;  // points of the window that exist
        float v[3][2][8];
        float sc[3], mxr[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          float mx = 0.0f;
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int p0 = 64 * j + 8 * g;
            const float* rx = sm.raw[rb][dxr[r]] + p0;
            const float* ry = sm.raw[rb][dyr[r]] + p0;
            const int64_t left = validr[r] ? wleft - p0 : 0;
            if (left >= 8) {
              const float4 a0 = *reinterpret_cast<const float4*>(rx);
              const float4 a1 = *reinterpret_cast<const float4*>(rx + 4);
              const float4 b0 = *reinterpret_cast<const float4*>(ry);
              const float4 b1 = *reinterpret_cast<const float4*>(ry + 4);
              v[r][j][0] = a0.x * b0.x; v[r][j][1] = a0.y * b0.y; v[r][j][2] = a0.z * b0.z; v[r][j][3] = a0.w * b0.w;
              v[r][j][4] = a1.x * b1.x; v[r][j][5] = a1.y * b1.y; v[r][j][6] = a1.z * b1.z; v[r][j][7] = a1.w * b1.w;
            } else {
#pragma unroll
              for (int i = 0; i < 8; ++i) v[r][j][i] = i < left ? rx[i] * ry[i] : 0.0f;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) mx = fmaxf(mx, fabsf(v[r][j][i]));
          }
          mxr[r] = mx;
        }
        // the column maxima over the eight lanes of each column, the three rounds interleaved
#pragma unroll
        for (int d = 1; d < 8; d <<= 1)
#pragma unroll
          for (int r = 0; r < 3; ++r) mxr[r] = fmaxf(mxr[r], __shfl_xor_sync(col_mask, mxr[r], d));
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int e = row_exponent(mxr[r]);
          if (g == 0 && pw + 6 * r < 16) sm.eb[set][colr[r]] = e;
          sc[r] = e == kZeroExp ? 0.0f : pow2f(7 - e);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          if (j < nck && run) {
            const bool okc = c < 2 || ws::wait(&sm.stage_free[c & 1], ((c - 2) >> 1) & 1, &sm.abort);
            run = __all_sync(kFull, okc && !ws::aborted(sm));
            if (!run) {
              ws::fail(sm, status, 5);
            } else {
              uint8_t* dst = sm.b[c & 1][0];
#pragma unroll
              for (int r = 0; r < 3; ++r) {
                if (pw + 6 * r < 16) {
                  uint4 wv[kSlices];
                  slice8(v[r][j], sc[r], wv);
#pragma unroll
                  for (int k = 0; k < kSlices; ++k)
                    *reinterpret_cast<uint4*>(dst + k * (kTileN * 128) + swz(colr[r], g)) = wv[k];
                }
              }
              fence_async_smem();
              __syncwarp();
              if (lane == 0) ws::mbar_arrive(&sm.b_ready[c & 1]);
              ++c;
            }
          }
        }
        if (!run) break;
        __syncwarp();
        if (lane == 0) ws::mbar_arrive(&sm.raw_free[rb]);
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
          const int nck = min(2, q.nch - 2 * win);
          const int set = w & 1;
          if (w >= 2) ok = ws::wait(&sm.tmem_free[set], ((w - 2) >> 1) & 1, &sm.abort);
          const uint32_t tset = tmem + (uint32_t)set * 256u;
          for (int j = 0; j < nck && ok; ++j, ++c) {
            const int s = c & 1;
            ok = ws::wait(&sm.a_full[s], (c >> 1) & 1, &sm.abort);
            if (ok) ok = ws::wait(&sm.b_ready[s], (c >> 1) & 1, &sm.abort);
            if (!ok) break;
            fence_after();
            // The B planes of a stage are contiguous (64 rows each), so plane i of A against
            // planes 0..3-i of B is one MMA of N = 64 (4 - i) whose columns land on the order
            // accumulators i..3 (order k at TMEM columns 64k..64k+63 of the set).
#pragma unroll
            for (int k = 0; k < kChunk / 16; ++k) {
              const uint32_t ko = 32u * k;
              const uint64_t db = make_desc(smem_u32(sm.b[s][0]) + ko);
#pragma unroll
              for (int i = 0; i < kSlices; ++i) {
                const uint64_t da = make_desc(smem_u32(sm.a[s][i]) + ko);
                mma_bf16(tset + 64u * i, da, db, make_idesc(64 * (kSlices - i)), (j > 0 || k > 0 || i > 0) ? 1u : 0u);
              }
            }
            mma_commit(smem_u32(&sm.stage_free[s]));
          }
          if (!ok) { ws::fail(sm, status, 6); break; }
          mma_commit(smem_u32(&sm.tmem_full[set]));
        }
        if (!ok) break;
      }
      // drain: every issued MMA must be complete before the TMEM is released
      if (ws::aborted(sm)) {
        mma_commit(smem_u32(&sm.drain));
        ws::wait(&sm.drain, 0);
      }
    }
    __syncwarp();
  } else if (warp >= ws::kFoldWarp0) {
    // ------------------------------------------------------------------ fold
    const int ew = warp - ws::kFoldWarp0;  // 0..7
    const int quad = warp & 3;             // TMEM lane quadrant this warp may access
    const int half = ew >> 2;              // 16-column groups gq with gq % 2 == half
    const int row_in_tile = quad * 32 + lane;
    bool run = true;  // warp-uniform
    for (int ii = cta_begin[blockIdx.x], ie = cta_begin[blockIdx.x + 1]; ii < ie && run; ++ii) {
      const GemmItem it = items[ii];
      const ws::Geo q = ws::geo(it, blocks, grids, ptiles);
      const MmaBlock& b = *q.blk;
      const Panel& pa = panels[b.a_panel];
      const Panel* pb = q.formed ? nullptr : panels + b.b_panel;
      const int rows_valid = min(kM, b.m - it.tm * kM);  // real rows of the A tile
      float H[32], L[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) { H[j] = 0.0f; L[j] = 0.0f; }
      // the window's exponents (A rows from the packed panel, B columns from the packed panel,
      // one per lane for this warp's 32 columns, or from the producers), loaded one window ahead
      const int my_col = (2 * (lane >> 4) + half) * 16 + (lane & 15);
      const int* ea_src = reinterpret_cast<const int*>(packed + pa.exp_off) + (int64_t)it.tm * pa.nwin * kM + row_in_tile;
      const int* eb_src = pb ? reinterpret_cast<const int*>(packed + pb->exp_off) + (int64_t)it.tn * pb->nwin * kTileN + my_col
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
        const bool ok = ws::wait(&sm.tmem_full[set], (w >> 1) & 1, &sm.abort);
        run = __all_sync(kFull, ok && !ws::aborted(sm));
        if (!run) { ws::fail(sm, status, 7); break; }
        fence_after();
        // column scales 2^(e_b - 7) for this warp, row scale 2^(e_a - 7) for this thread
        float* sbw = sm.sbw[ew];
        sbw[my_col] = pow2f((pb ? eb_lane : sm.eb[set][my_col]) - 7);
        const float sa = pow2f(ea - 7);
        __syncwarp();
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)set * 256u;
#pragma unroll
        for (int gi = 0; gi < 2; ++gi) {
          const int gq = 2 * gi + half;  // 16-column group
          // a warp whose 32 rows are all past the tile's last real row has nothing to fold
          if (gq * 16 < q.ntp && quad * 32 < rows_valid) {
#pragma unroll
            for (int sub = 0; sub < 2; ++sub) {
              const int c0 = gq * 16 + 8 * sub;  // first of 8 columns
              float o0[8], o1[8], o2[8], o3[8];
              tmem_ld8(lane_base + 0 * kTileN + c0, o0);
              tmem_ld8(lane_base + 1 * kTileN + c0, o1);
              tmem_ld8(lane_base + 2 * kTileN + c0, o2);
              tmem_ld8(lane_base + 3 * kTileN + c0, o3);
              tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int qq = gi * 16 + 8 * sub + j;
                const float sc = sa * sbw[c0 + j];  // 2^(e_a + e_b - 14)
                // order 0 (exact integers) into the double-float sum, orders 1..3 (each 256
                // times smaller) as one FP32 correction
                const float x = o0[j] * sc;
                const float t = H[qq] + x;
                const float bb = t - H[qq];
                const float err = (H[qq] - (t - bb)) + (x - bb);
                H[qq] = t;
                const float lo = fmaf(o3[j], 5.9604644775390625e-8f, fmaf(o2[j], 1.52587890625e-5f, o1[j] * 0.00390625f));
                L[qq] += fmaf(lo, sc, err);
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
        for (int gi = 0; gi < 2; ++gi) {
          const int gq = 2 * gi + half;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int cc = gq * 16 + j;
            if (cc < q.nt) {
              const int col = q.formed ? q.pt->col[cc] : it.tn * kTileN + cc;
              out[col] = make_float2(H[gi * 16 + j], L[gi * 16 + j]);
            }
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
                                                           const int64_t* __restrict__ elem_begin, int64_t n_elems,
                                                           const short2* __restrict__ rows,
                                                           const double* __restrict__ rowc,
                                                           const float2* __restrict__ part, double* __restrict__ res) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_elems) return;
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

// ------------------------------------------------------------------ launchers

cudaError_t launch_nodes(const DevGrid* grids, int n_grids, int max_entries, const double* edges, NodeEntry* tab,
                         cudaStream_t s) {
  if (n_grids == 0) return cudaSuccess;
  dim3 grid((max_entries + 127) / 128, n_grids);
  nodes_kernel<<<grid, 128, 0, s>>>(grids, edges, tab);
  return cudaGetLastError();
}

cudaError_t launch_eval_mixed(const LaunchTables& t, const NodeEntry* tab, const float2* xi, float* ops,
                              cudaStream_t s) {
  if (t.n_pblocks == 0) return cudaSuccess;
  eval_mixed_kernel<<<t.n_pblocks, 128, 0, s>>>(t, tab, xi, ops);
  return cudaGetLastError();
}

size_t ws_smem_bytes() { return sizeof(ws::Smem) + 1024; }

cudaError_t prepare_kernels() {
  return cudaFuncSetAttribute(contract_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws_smem_bytes());
}

cudaError_t launch_pack(const DevGrid* grids, const Panel* panels, int n_panels, int64_t n_jobs, const short2* rows,
                        const float* ops, uint8_t* packed, cudaStream_t s) {
  if (n_jobs == 0) return cudaSuccess;
  pack_kernel<<<(unsigned)n_jobs, 512, 0, s>>>(grids, panels, n_panels, rows, ops, packed);
  return cudaGetLastError();
}

cudaError_t launch_contract_ws(const DevGrid* grids, const MmaBlock* blocks, const GemmItem* items,
                               const int* cta_begin, int n_ctas, const Panel* panels, const PairTile* ptiles,
                               const float* ops, const uint8_t* packed, float2* part, int* status, cudaStream_t s) {
  if (n_ctas == 0) return cudaSuccess;
  contract_ws_kernel<<<n_ctas, ws::kThreads, ws_smem_bytes(), s>>>(grids, blocks, items, cta_begin, panels, ptiles, ops,
                                                                   packed, part, status);
  return cudaGetLastError();
}

cudaError_t launch_ri_pack(const Panel* panels, int64_t n_jobs, const double* srcA, const double* srcB, int n,
                           uint8_t* packed, cudaStream_t s) {
  if (n_jobs == 0) return cudaSuccess;
  ri_pack_kernel<<<(unsigned)n_jobs, 512, 0, s>>>(panels, srcA, srcB, n, packed);
  return cudaGetLastError();
}

cudaError_t launch_reduce_mixed(const DevGrid* grids, const MmaBlock* blocks, int n_blocks, const int64_t* elem_begin,
                                int64_t n_elems, const short2* rows, const double* rowc, const float2* part,
                                double* res, cudaStream_t s) {
  if (n_elems == 0) return cudaSuccess;
  reduce_mixed_kernel<<<(unsigned)((n_elems + 255) / 256), 256, 0, s>>>(grids, blocks, n_blocks, elem_begin, n_elems,
                                                                         rows, rowc, part, res);
  return cudaGetLastError();
}


}  // namespace psq
