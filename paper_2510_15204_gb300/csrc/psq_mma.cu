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
//  * contract_ws_kernel: the weighted contraction of eq 9 on tcgen05 tensor cores.  Every
//    operand row of a 64-point chunk is scaled by a power of two from its maximum and cut
//    into four integer slices of at most 8 bits (exact in BF16).  Ten BF16 MMAs per K step
//    accumulate the slice products by order (0..3) into four FP32 TMEM accumulators; all
//    partial sums are integers below 2^24, so the FP32 accumulation is exact.  After each
//    chunk the accumulators are scaled back and added into double-float (FP32 hi + lo)
//    registers; each work item writes its point range's (hi, lo) sums, and reduce_mixed_kernel
//    adds the ranges in FP64 and applies the FP64 constants of each row and column
//    (normalisations, powers of zeta, a^3), which the FP32 values omit.
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
__device__ __forceinline__ float radial_x(int kind, int n, int l, float xh, float xl) {
  const float ex = expf(-xh);
  const float ix = 1.0f / xh;
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
  const int64_t p = pb.p0 + threadIdx.x;
  if (p >= g.K) return;
  const int q3 = g.q_mu * g.q_nu * g.q_phi;
  int ri, rj, rk;
  bool dead = false;
  int64_t pr;
  if (p < g.K_reg) {
    const int64_t cell = p / q3;
    pr = p - cell * q3;
    rk = (int)(cell % g.n_phi);
    rj = (int)((cell / g.n_phi) % g.n_nu);
    ri = (int)(cell / ((int64_t)g.n_phi * g.n_nu));
    if (g.n_touch > 0 && ri >= g.t_mu0 && ri <= g.t_mu1 && rj >= g.t_nu0 && rj <= g.t_nu1 &&
        (g.t_phi_all || rk == 0 || rk == g.n_phi - 1))
      dead = true;
  } else {
    const int64_t s = (p - g.K_reg) / q3;
    pr = (p - g.K_reg) - s * q3;
    const int ns = g.n_sp, ns3 = ns * ns * ns;
    const int tc = (int)(s / ns3), sub = (int)(s % ns3);
    const int ntp = g.nt_phi, nnu = g.nt_nu;
    const int ti = tc / (nnu * ntp), tj = (tc / ntp) % nnu, tk = tc % ntp;
    const int si = sub / (ns * ns), sj = (sub / ns) % ns, sk = sub % ns;
    ri = g.n_mu + ti * ns + si;
    rj = g.n_nu + tj * ns + sj;
    rk = g.n_phi + tk * ns + sk;
  }
  const int qi = (int)(pr / (g.q_nu * g.q_phi));
  const int qj = (int)((pr / g.q_phi) % g.q_nu);
  const int qk = (int)(pr % g.q_phi);
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
      if (g.row_F >= 0) eval_shells_x(t.bshell, z, s0, s1, rho, Y, base, ld, p, g.row_F + roff, 0);
      if (g.row_L >= 0) eval_shells_x(t.bshell, z, s0, s1, rho, Y, base, ld, p, g.row_L + roff, 1);
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
      if (g.row_G >= 0) eval_shells_x(t.ashell, z, s0, s1, rho, Y, base, ld, p, g.row_G + roff, 0);
      if (g.row_U >= 0) eval_shells_x(t.ashell, z, s0, s1, rho, Y, base, ld, p, g.row_U + roff, 2);
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
constexpr uint32_t kSpinLimit = 1u << 26;

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

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
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

// ------------------------------------------------------------------ warp-specialised version
//
// One persistent CTA per SM (512 threads).  Warps 0-7 produce: for each 64-point chunk they
// build the A tile (128 rows) and the B tile (<= 64 rows) as four integer slices in one of two
// shared-memory stages, two threads per row (32 points each); lane 0 of warp 0 then issues
// the chunk's 40 MMAs into one of two TMEM accumulator sets and commits them to full[stage].
// Warps 8-15 fold: they wait full[stage], read the four order accumulators of their lane
// quadrant and column half, add the chunk into double-float registers and arrive at
// free[stage], which lets the producers reuse the stage and the TMEM set.  A CTA's point
// range ends with a write of (hi, lo) pairs; the FP64 reduction applies the row constants.

namespace ws {

constexpr int kProducers = 256;
constexpr int kEpi = 256;
constexpr int kThreads = kProducers + kEpi;
constexpr int kStages = 2;

struct Smem {
  alignas(1024) uint8_t a[kStages][mma::kSlices][mma::kM * 128];
  alignas(1024) uint8_t b[kStages][mma::kSlices][mma::kTileN * 128];
  int ea[kStages][mma::kM];
  int eb[kStages][mma::kTileN];
  alignas(8) uint64_t full[kStages];
  alignas(8) uint64_t freed[kStages];
  uint32_t tmem_base;
  int abort;
};

// Barrier of the 256 producer threads that also ORs a predicate over them, so every producer
// takes the same decision from it.
__device__ __forceinline__ bool named_sync_producers_or(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "n"(kProducers)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void prefetch_l2(const float* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(mbar) : "memory");
}

// 32 values of half a row -> four slices (bytes [64h, 64h+64) of the row in each slice).
__device__ __forceinline__ void slice_half(const float* v, float sc, int row, int h, uint8_t* const* sl) {
  const uint32_t rowoff = (uint32_t)row * 128u;
  const uint32_t sw = (uint32_t)(row & 7);
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    const int c = 4 * h + cc;  // 16-byte chunk index within the 128-byte row
    uint32_t w[mma::kSlices][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float r0 = v[8 * cc + 2 * q] * sc, r1 = v[8 * cc + 2 * q + 1] * sc;
#pragma unroll
      for (int k = 0; k < mma::kSlices; ++k) {
        const float a0 = rintf(r0), a1 = rintf(r1);
        const __nv_bfloat162 p = __floats2bfloat162_rn(a0, a1);
        w[k][q] = *reinterpret_cast<const uint32_t*>(&p);
        r0 = (r0 - a0) * 256.0f;
        r1 = (r1 - a1) * 256.0f;
      }
    }
    const uint32_t off = rowoff + (((uint32_t)c ^ sw) << 4);
#pragma unroll
    for (int k = 0; k < mma::kSlices; ++k)
      *reinterpret_cast<uint4*>(sl[k] + off) = make_uint4(w[k][0], w[k][1], w[k][2], w[k][3]);
  }
}

__device__ __forceinline__ void load32(const float* __restrict__ src, const float* __restrict__ mul, int64_t k0,
                                       int64_t K, float* v) {
  if (k0 + 32 <= K) {
    const float4* s4 = reinterpret_cast<const float4*>(src + k0);
    const float4* m4 = reinterpret_cast<const float4*>(mul + k0);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float4 q = __ldg(s4 + i);
      if (mul) {
        const float4 m = __ldg(m4 + i);
        q.x *= m.x; q.y *= m.y; q.z *= m.z; q.w *= m.w;
      }
      v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = (k0 + i < K) ? src[k0 + i] * (mul ? mul[k0 + i] : 1.0f) : 0.0f;
  }
}

// One producer task: half h of operand row `row` of the tile (values from the grid's FP32
// rows), sliced into stage `st`.  Returns nothing; the row's exponent goes to *e_out (h == 0).
__device__ __forceinline__ void produce_half(const float* src, const float* mul, int64_t k0, int64_t K, bool valid,
                                             int row, int h, uint8_t* const* sl, int* e_out) {
  float v[32];
  if (valid) {
    load32(src, mul, k0 + 32 * h, K, v);
  } else {
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = 0.0f;
  }
  float mx = 0.0f;
#pragma unroll
  for (int i = 0; i < 32; ++i) mx = fmaxf(mx, fabsf(v[i]));
  mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  int e = 0;
  if (mx > 0.0f) frexpf(mx, &e);
  const bool zero = !(mx > 0.0f) || e < -110;
  slice_half(v, zero ? 0.0f : mma::pow2f(7 - e), row, h, sl);
  if (h == 0) *e_out = zero ? -100000 : e;
}

}  // namespace ws

__global__ void __launch_bounds__(ws::kThreads, 1) contract_ws_kernel(const DevGrid* __restrict__ grids,
                                                                      const MmaBlock* __restrict__ blocks,
                                                                      const GemmItem* __restrict__ items, int n_items,
                                                                      const short2* __restrict__ rows,
                                                                      const float* __restrict__ ops,
                                                                      float2* __restrict__ part,
                                                                      int* __restrict__ status) {
  using namespace mma;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  ws::Smem& sm = *reinterpret_cast<ws::Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < ws::kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_u32(&sm.freed[s])));
    }
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm.tmem_base;
  uint32_t c = 0;  // chunks of this CTA so far (stage = c & 1, TMEM set = c & 1)

  if (tid < ws::kProducers) {
    // ------------------------------------------------------------ producers (+ MMA issue)
    bool stop = false;
    for (int ii = blockIdx.x; ii < n_items; ii += gridDim.x) {
      const GemmItem it = items[ii];
      const MmaBlock b = blocks[it.block];
      const DevGrid& g = grids[b.grid];
      const float* base = ops + g.op_off;
      const int64_t ld = g.ld, K = g.K;
      const int nt = min(kTileN, b.n - it.tn * kTileN), ntp = (nt + 15) & ~15;
      const int r0 = it.tm * kM, c0 = it.tn * kTileN;
      const int64_t nchunk = (K + kChunk - 1) / kChunk;
      const int64_t per = (nchunk + b.n_ranges - 1) / b.n_ranges;
      const int64_t ch0 = (int64_t)it.chunk * per, ch1 = min(nchunk, ch0 + per);
      const uint32_t idesc = make_idesc(ntp);
      // this thread's A task: row tid/2, half tid%2; B task (tid < 2 ntp): column tid/2
      const int arow = tid >> 1, ah = tid & 1;
      const int grow = r0 + arow;
      const bool avalid = grow < b.m;
      const float *asrc = nullptr, *amul = nullptr;
      if (avalid) {
        const short2 q = rows[b.a_off + grow];
        asrc = base + (int64_t)q.x * ld;
        amul = q.y >= 0 ? base + (int64_t)q.y * ld : nullptr;
      }
      const int brow = tid >> 1;
      const bool btask = tid < 2 * ntp, bvalid = brow < nt;
      const float *bsrc = nullptr, *bmul = nullptr;
      if (bvalid) {
        const short2 q = rows[b.b_off + c0 + brow];
        bsrc = base + (int64_t)q.x * ld;
        bmul = q.y >= 0 ? base + (int64_t)q.y * ld : nullptr;
      }
      for (int64_t ch = ch0; ch < ch1; ++ch, ++c) {
        const int st = c & 1;
        // pull this thread's rows of the chunk after next into L2 while this one is built
        if (ch + 2 < ch1) {
          const int64_t kp = (ch + 2) * kChunk + 32 * ah;
          if (avalid) {
            ws::prefetch_l2(asrc + kp);
            if (amul) ws::prefetch_l2(amul + kp);
          }
          if (btask && bvalid) {
            const int64_t kb = (ch + 2) * kChunk + 32 * (tid & 1);
            ws::prefetch_l2(bsrc + kb);
            if (bmul) ws::prefetch_l2(bmul + kb);
          }
        }
        bool ok = true;
        if (c >= 2) ok = mbar_wait(smem_u32(&sm.freed[st]), ((c - 2) >> 1) & 1);
        if (!ok) atomicExch(status, 2);
        const int64_t k0 = ch * kChunk;
        uint8_t* asl[kSlices] = {sm.a[st][0], sm.a[st][1], sm.a[st][2], sm.a[st][3]};
        ws::produce_half(asrc, amul, k0, K, avalid, arow, ah, asl, &sm.ea[st][arow]);
        if (btask) {
          uint8_t* bsl[kSlices] = {sm.b[st][0], sm.b[st][1], sm.b[st][2], sm.b[st][3]};
          ws::produce_half(bsrc, bmul, k0, K, bvalid, brow, tid & 1, bsl, &sm.eb[st][brow]);
        }
        fence_async_smem();
        // one decision for all producers: stop if any of them timed out or the fold warps did
        if (ws::named_sync_producers_or(!ok || *(volatile int*)&sm.abort)) { stop = true; break; }
        if (tid == 0) {
          fence_after();
          const uint32_t tset = tmem + (uint32_t)st * 256u;
#pragma unroll
          for (int k = 0; k < kChunk / 16; ++k) {
            const uint32_t ko = 32u * k;
#pragma unroll
            for (int ord = 0; ord < kSlices; ++ord) {
#pragma unroll
              for (int i = 0; i <= ord; ++i) {
                const uint64_t da = make_desc(smem_u32(sm.a[st][i]) + ko);
                const uint64_t db = make_desc(smem_u32(sm.b[st][ord - i]) + ko);
                mma_bf16(tset + ord * ntp, da, db, idesc, (k > 0 || i > 0) ? 1u : 0u);
              }
            }
          }
          mma_commit(smem_u32(&sm.full[st]));
        }
      }
      if (stop) break;
    }
  } else {
    // ------------------------------------------------------------ fold (epilogue) warps
    const int lane = tid & 31;
    const int ew = warp - 8;             // 0..7
    const int quad = warp & 3;           // TMEM lane quadrant this warp may access
    const int half = ew >> 2;            // column groups g with g % 2 == half
    const int row_in_tile = quad * 32 + lane;
    for (int ii = blockIdx.x; ii < n_items; ii += gridDim.x) {
      const GemmItem it = items[ii];
      const MmaBlock b = blocks[it.block];
      const DevGrid& g = grids[b.grid];
      const int64_t K = g.K;
      const int nt = min(kTileN, b.n - it.tn * kTileN), ntp = (nt + 15) & ~15;
      const int r0 = it.tm * kM, c0 = it.tn * kTileN;
      const int64_t nchunk = (K + kChunk - 1) / kChunk;
      const int64_t per = (nchunk + b.n_ranges - 1) / b.n_ranges;
      const int64_t ch0 = (int64_t)it.chunk * per, ch1 = min(nchunk, ch0 + per);
      float H[32], L[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) { H[j] = 0.0f; L[j] = 0.0f; }
      bool ok = true;
      for (int64_t ch = ch0; ch < ch1; ++ch, ++c) {
        const int st = c & 1;
        ok = mbar_wait(smem_u32(&sm.full[st]), (c >> 1) & 1);
        if (!ok) { *(volatile int*)&sm.abort = 1; atomicExch(status, 3); break; }
        fence_after();
        const int ea = sm.ea[st][row_in_tile];
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)st * 256u;
#pragma unroll
        for (int gi = 0; gi < 2; ++gi) {
          const int gq = 2 * gi + half;  // 16-column group
          if (gq * 16 < ntp) {
            float hi[16], lo[16], d[16];
            tmem_ld16(lane_base + 0 * ntp + gq * 16, hi);
            tmem_ld16(lane_base + 1 * ntp + gq * 16, lo);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) lo[j] *= 0.00390625f;
#pragma unroll
            for (int ord = 2; ord < kSlices; ++ord) {
              tmem_ld16(lane_base + ord * ntp + gq * 16, d);
              tmem_wait_ld();
              const float sc = pow2f(-8 * ord);
#pragma unroll
              for (int j = 0; j < 16; ++j) lo[j] = fmaf(d[j], sc, lo[j]);
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float s = pow2f(ea + sm.eb[st][gq * 16 + j] - 14);
              const float x = hi[j] * s;
              const int q = gi * 16 + j;
              const float t = H[q] + x;
              const float bb = t - H[q];
              const float err = (H[q] - (t - bb)) + (x - bb);
              H[q] = t;
              L[q] += fmaf(lo[j], s, err);
            }
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) ws::mbar_arrive(smem_u32(&sm.freed[st]));
      }
      if (!ok) break;
      // (hi, lo) partial sums of this item's point range
      const int grow = r0 + row_in_tile;
      if (grow < b.m) {
        float2* out = part + b.part_off + (int64_t)it.chunk * b.m * b.n;
#pragma unroll
        for (int gi = 0; gi < 2; ++gi) {
          const int gq = 2 * gi + half;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = gq * 16 + j;
            if (col < nt) {
              out[(int64_t)grow * b.n + c0 + col] = make_float2(H[gi * 16 + j], L[gi * 16 + j]);
            }
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 8) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// FP64 reduction of the (hi, lo) range partials of the tensor-core blocks, times the FP64
// constants of each element's row and column; one warp per element, fixed order.
__global__ void __launch_bounds__(256) reduce_mixed_kernel(const DevGrid* __restrict__ grids,
                                                           const MmaBlock* __restrict__ blocks, int n_blocks,
                                                           const int64_t* __restrict__ elem_begin, int64_t n_elems,
                                                           const short2* __restrict__ rows,
                                                           const double* __restrict__ rowc,
                                                           const float2* __restrict__ part, double* __restrict__ res) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= n_elems) return;
  int lo = 0, hi = n_blocks;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (elem_begin[mid] <= wid) lo = mid; else hi = mid;
  }
  const MmaBlock b = blocks[lo];
  const int64_t e = wid - elem_begin[lo];
  const int64_t mn = (int64_t)b.m * b.n;
  double s = 0.0;
  for (int c = lane; c < b.n_ranges; c += 32) {
    const float2 v = part[b.part_off + c * mn + e];
    s += (double)v.x + (double)v.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) {
    const int r = (int)(e / b.n), col = (int)(e % b.n);
    const double* rc = rowc + grids[b.grid].rc_off;
    const short2 qa = rows[b.a_off + r], qb = rows[b.b_off + col];
    const double ca = rc[qa.x] * (qa.y >= 0 ? rc[qa.y] : 1.0);
    const double cb = rc[qb.x] * (qb.y >= 0 ? rc[qb.y] : 1.0);
    res[b.res_off + e] = s * ca * cb;
  }
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

cudaError_t launch_contract_ws(const DevGrid* grids, const MmaBlock* blocks, const GemmItem* items, int n_items,
                               int n_ctas, const short2* rows, const float* ops, float2* part, int* status,
                               cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  const size_t bytes = ws_smem_bytes();
  contract_ws_kernel<<<n_ctas, ws::kThreads, bytes, s>>>(grids, blocks, items, n_items, rows, ops, part, status);
  return cudaGetLastError();
}

cudaError_t launch_reduce_mixed(const DevGrid* grids, const MmaBlock* blocks, int n_blocks, const int64_t* elem_begin,
                                int64_t n_elems, const short2* rows, const double* rowc, const float2* part,
                                double* res, cudaStream_t s) {
  if (n_elems == 0) return cudaSuccess;
  const int64_t threads = n_elems * 32;
  reduce_mixed_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(grids, blocks, n_blocks, elem_begin, n_elems,
                                                                         rows, rowc, part, res);
  return cudaGetLastError();
}


}  // namespace psq
