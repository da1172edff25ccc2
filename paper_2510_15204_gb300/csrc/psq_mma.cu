// Mixed-precision path of the PS quadrature on sm_103a:
//  * node tables: the PS grid is a tensor product in (mu, nu, phi) per volume element, so the
//    per-node trigonometric factors (Section 2.1, eqs 2-6, 10-11) are computed once per grid
//    row in FP64 (nodes_kernel) and combined per point;
//  * eval_mixed_kernel: point weights, focal distances and offsets in FP32 from the FP64
//    tables (the cancellation-free forms need no FP64), the third-centre offset in FP64
//    (it cancels near that centre), STOs (eq 1), their kinetic operand and the aux
//    potentials (eq 16, incomplete gamma by its positive series below x = k) in FP32;
//  * contract_mma_kernel: the weighted contraction of eq 9 on tcgen05 tensor cores.  Every
//    operand row of a 64-point chunk is scaled by a power of two from its maximum and cut
//    into three integer slices of at most 8 bits (exact in BF16).  Six BF16 MMAs per K step
//    accumulate the slice products by order (0; 1; 2) into three FP32 TMEM accumulators;
//    all partial sums are integers below 2^24, so the FP32 accumulation is exact.  After each
//    chunk the accumulators are scaled back and added into double-float (FP32 hi + lo)
//    registers; each CTA writes its point range's sum in FP64.
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

__device__ __forceinline__ void real_ylm_f(int lmax, float ux, float uy, float uz, float* Y) {
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
        Y[base] = c_klmf[base] * q;
      } else {
        Y[base + m] = c_klmf[base + m] * q * C[m];
        Y[base - m] = c_klmf[base - m] * q * S[m];
      }
    }
  }
}

__device__ __forceinline__ float ipowf(float x, int n) {
  float r = 1.0f;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

__device__ float aux_pot_radial_f(int n, int l, float zeta, float norm, float r) {
  const float x = zeta * r;
  const int k1 = n + l + 2, k2 = n - l + 1;
  const float ex = expf(-x);
  float inner;
  if (x < (float)k1) {
    float term = c_rcpf[k1], sum = term;
    for (int i = 1; i < 120 - k1; ++i) {
      term *= x * c_rcpf[k1 + i];
      sum += term;
      if (term <= 3e-8f * sum) break;
    }
    inner = ipowf(r, n + 1) * ex * sum;
  } else {
    float t = 1.0f, s = 1.0f;
    for (int j = 1; j < k1; ++j) { t *= x * c_rcpf[j]; s += t; }
    const float f = c_factf[k1 - 1];
    inner = (f - f * ex * s) / (ipowf(zeta, k1) * ipowf(r, l + 1));
  }
  float t = 1.0f, s = 1.0f;
  for (int j = 1; j < k2; ++j) { t *= x * c_rcpf[j]; s += t; }
  const float outer = c_factf[k2 - 1] * ex * s * ipowf(r, l) / ipowf(zeta, k2);
  return (float)(4.0 * M_PI) * c_rcpf[2 * l + 1] * norm * (inner + outer);
}

__device__ __forceinline__ void eval_shells_f(const DevShell* __restrict__ sh, int s0, int s1, float r,
                                              const float* Y, float* __restrict__ out, int64_t ld,
                                              int64_t p, int row0, int kind) {
  for (int s = s0; s < s1; ++s) {
    const DevShell q = sh[s];
    const float zeta = (float)q.zeta, norm = (float)q.norm;
    float radial;
    if (kind == 2) {
      radial = aux_pot_radial_f(q.n, q.l, zeta, norm, r);
    } else {
      radial = norm * ipowf(r, q.n - 1) * expf(-zeta * r);
      if (kind == 1) {
        const float ir = 1.0f / r;
        radial *= ((float)(q.n * (q.n - 1) - q.l * (q.l + 1)) * ir - 2.0f * q.n * zeta) * ir + zeta * zeta;
      }
    }
    const int base = q.l * q.l + q.l;
    for (int m = -q.l; m <= q.l; ++m) out[(int64_t)(row0 + q.fn0 + q.l + m) * ld + p] = radial * Y[base + m];
  }
}

__device__ __forceinline__ int shells_lmax_f(const DevShell* sh, int s0, int s1) {
  int l = 0;
  for (int s = s0; s < s1; ++s) l = max(l, sh[s].l);
  return l;
}

__global__ void __launch_bounds__(128) eval_mixed_kernel(LaunchTables t, const NodeEntry* __restrict__ tab,
                                                         float* __restrict__ ops) {
  const PointBlock pb = t.pblocks[blockIdx.x];
  const DevGrid& g = t.grids[pb.grid];
  const int64_t p = pb.p0 + threadIdx.x;
  if (p >= g.K) return;
  const int q3 = g.q_mu * g.q_nu * g.q_phi;
  int ri, rj, rk, qi, qj, qk;
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
    const int ntp = g.nt_phi;
    const int nnu = g.nt_nu;
    const int ti = tc / (nnu * ntp), tj = (tc / ntp) % nnu, tk = tc % ntp;
    const int si = sub / (ns * ns), sj = (sub / ns) % ns, sk = sub % ns;
    ri = g.n_mu + ti * ns + si;
    rj = g.n_nu + tj * ns + sj;
    rk = g.n_phi + tk * ns + sk;
  }
  qi = (int)(pr / (g.q_nu * g.q_phi));
  qj = (int)((pr / g.q_phi) % g.q_nu);
  qk = (int)(pr % g.q_phi);
  const int nmu = (g.n_mu + g.nt_mu * g.n_sp) * g.q_mu;
  const int nnu = (g.n_nu + g.nt_nu * g.n_sp) * g.q_nu;
  const NodeEntry Mu = tab[g.nt_off + ri * g.q_mu + qi];
  const NodeEntry Nu = tab[g.nt_off + nmu + rj * g.q_nu + qj];
  const NodeEntry Ph = tab[g.nt_off + nmu + nnu + rk * g.q_phi + qk];
  const float a = (float)g.a;
  const float sh = (float)Mu.s, s2m = (float)Mu.h2;
  const float sn = (float)Nu.s, cs = (float)Nu.c, s2n = (float)Nu.h2, c2n = (float)Nu.g2;
  const float sp = (float)Ph.s, cp = (float)Ph.c;
  const float a3 = (float)(g.a * g.a * g.a);
  const float w = dead ? 0.0f
                       : (float)(Mu.w * Nu.w * Ph.w) * a3 * sh * sn * fmaf(sh, sh, sn * sn);
  const float rA = 2.0f * a * (s2m + s2n), rB = 2.0f * a * (s2m + c2n);
  const float x = a * sh * sn * cp, y = a * sh * sn * sp;
  const float zA = 2.0f * a * (s2m * cs - s2n), zB = 2.0f * a * (s2m * cs + c2n);
  float R[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = (float)g.R[i];
  float dA[3], dB[3], dC[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    dA[c] = R[c * 3] * x + R[c * 3 + 1] * y + R[c * 3 + 2] * zA;
    dB[c] = R[c * 3] * x + R[c * 3 + 1] * y + R[c * 3 + 2] * zB;
  }
  float rC = 1.0f;
  if (g.C >= 0) {
    // offset from the third centre in the pair frame, FP64: it cancels near that centre
    const double X = g.a * Mu.s * Nu.s * Ph.c - g.xc;
    const double Y = g.a * Mu.s * Nu.s * Ph.s;
    const double Z = g.a * Mu.c * Nu.c - g.zc;
    const float Xf = (float)X, Yf = (float)Y, Zf = (float)Z;
#pragma unroll
    for (int c = 0; c < 3; ++c) dC[c] = R[c * 3] * Xf + R[c * 3 + 1] * Yf + R[c * 3 + 2] * Zf;
    rC = sqrtf(Xf * Xf + Yf * Yf + Zf * Zf);
  }
  float* base = ops + g.op_off;
  const int64_t ld = g.ld;
  if (g.row_W >= 0) {
    base[(int64_t)(g.row_W + 0) * ld + p] = w;
    base[(int64_t)(g.row_W + 1) * ld + p] = w / rA;
    base[(int64_t)(g.row_W + 2) * ld + p] = w / rB;
    base[(int64_t)(g.row_W + 3) * ld + p] = g.C >= 0 ? w / rC : 0.0f;
  }
  float Y[(kMaxL + 1) * (kMaxL + 1)];
  if (g.row_F >= 0 || g.row_L >= 0) {
    for (int c = 0; c < 2; ++c) {
      const int s0 = c == 0 ? g.shb_A0 : g.shb_B0, s1 = c == 0 ? g.shb_A1 : g.shb_B1;
      if (s1 <= s0) continue;
      const float r = c == 0 ? rA : rB;
      const float* d = c == 0 ? dA : dB;
      const float ir = 1.0f / r;
      real_ylm_f(shells_lmax_f(t.bshell, s0, s1), d[0] * ir, d[1] * ir, d[2] * ir, Y);
      const int roff = c == 0 ? 0 : g.nFA;
      if (g.row_F >= 0) eval_shells_f(t.bshell, s0, s1, r, Y, base, ld, p, g.row_F + roff, 0);
      if (g.row_L >= 0) eval_shells_f(t.bshell, s0, s1, r, Y, base, ld, p, g.row_L + roff, 1);
    }
  }
  if (g.row_G >= 0 || g.row_U >= 0) {
    int roff = 0;
    for (int c = 0; c < 2; ++c) {
      const int s0 = c == 0 ? g.sha_0 : g.sha_2, s1 = c == 0 ? g.sha_1 : g.sha_3;
      const int atom = c == 0 ? g.aux_c0 : g.aux_c1;
      if (atom < 0 || s1 <= s0) continue;
      const float* d;
      float r;
      if (atom == g.A) { d = dA; r = rA; }
      else if (atom == g.B) { d = dB; r = rB; }
      else { d = dC; r = rC; }
      const float ir = 1.0f / r;
      real_ylm_f(shells_lmax_f(t.ashell, s0, s1), d[0] * ir, d[1] * ir, d[2] * ir, Y);
      if (g.row_G >= 0) eval_shells_f(t.ashell, s0, s1, r, Y, base, ld, p, g.row_G + roff, 0);
      if (g.row_U >= 0) eval_shells_f(t.ashell, s0, s1, r, Y, base, ld, p, g.row_U + roff, 2);
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
constexpr int kThreads = 128;
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

// Cuts 64 values of one operand row into three integer BF16 slices in the K-major 128-byte
// swizzled layout and returns the row's scale exponent e (|v| < 2^e).
__device__ __forceinline__ int slice_row(const float* v, int row, uint8_t* s0, uint8_t* s1, uint8_t* s2) {
  float mx = 0.0f;
#pragma unroll
  for (int i = 0; i < kChunk; ++i) mx = fmaxf(mx, fabsf(v[i]));
  int e = 0;
  if (mx > 0.0f) frexpf(mx, &e);
  const bool zero = !(mx > 0.0f) || e < -110;
  const float sc = zero ? 0.0f : pow2f(7 - e);
  const uint32_t rowoff = (uint32_t)row * 128u;
  const uint32_t sw = (uint32_t)(row & 7);
#pragma unroll
  for (int c = 0; c < 8; ++c) {  // 16-byte chunk c holds points 8c .. 8c+7
    uint32_t w0[4], w1[4], w2[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      uint16_t b0[2], b1[2], b2[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float al = v[8 * c + 2 * h + u] * sc;
        const float a0 = rintf(al);
        const float r1 = (al - a0) * 256.0f;
        const float a1 = rintf(r1);
        const float a2 = rintf((r1 - a1) * 256.0f);
        b0[u] = __bfloat16_as_ushort(__float2bfloat16_rn(a0));
        b1[u] = __bfloat16_as_ushort(__float2bfloat16_rn(a1));
        b2[u] = __bfloat16_as_ushort(__float2bfloat16_rn(a2));
      }
      w0[h] = (uint32_t)b0[0] | ((uint32_t)b0[1] << 16);
      w1[h] = (uint32_t)b1[0] | ((uint32_t)b1[1] << 16);
      w2[h] = (uint32_t)b2[0] | ((uint32_t)b2[1] << 16);
    }
    const uint32_t off = rowoff + (((uint32_t)c ^ sw) << 4);
    *reinterpret_cast<uint4*>(s0 + off) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    *reinterpret_cast<uint4*>(s1 + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *reinterpret_cast<uint4*>(s2 + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
  }
  return zero ? -100000 : e;
}

// v[i] = src[k0 + i] (* mul[k0 + i] when mul is given), zero past K.
__device__ __forceinline__ void load64(const float* __restrict__ src, const float* __restrict__ mul, int64_t k0,
                                       int64_t K, float* v) {
  if (k0 + kChunk <= K) {
    const float4* s4 = reinterpret_cast<const float4*>(src + k0);
    const float4* m4 = reinterpret_cast<const float4*>(mul + k0);
#pragma unroll
    for (int i = 0; i < kChunk / 4; ++i) {
      float4 q = __ldg(s4 + i);
      if (mul) {
        const float4 m = __ldg(m4 + i);
        q.x *= m.x; q.y *= m.y; q.z *= m.z; q.w *= m.w;
      }
      v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < kChunk; ++i) v[i] = (k0 + i < K) ? src[k0 + i] * (mul ? mul[k0 + i] : 1.0f) : 0.0f;
  }
}

struct Smem {
  alignas(1024) uint8_t a[3][kM * 128];       // A slices: 128 rows x 64 points BF16
  alignas(1024) uint8_t b[3][kTileN * 128];    // B slices: up to 64 rows
  int ea[kM];
  int eb[kTileN];
  alignas(8) uint64_t mbar;
  uint32_t tmem_base;
};

}  // namespace mma

__global__ void __launch_bounds__(mma::kThreads) contract_mma_kernel(const DevGrid* __restrict__ grids,
                                                                      const MmaBlock* __restrict__ blocks,
                                                                      const GemmItem* __restrict__ items,
                                                                      const short2* __restrict__ pairs,
                                                                      const float* __restrict__ ops,
                                                                      double* __restrict__ part,
                                                                      int* __restrict__ status) {
  using namespace mma;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const GemmItem it = items[blockIdx.x];
  const MmaBlock b = blocks[it.block];
  const DevGrid& g = grids[b.grid];
  const float* base = ops + g.op_off;
  const int64_t ld = g.ld, K = g.K;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nt = min(kTileN, b.n - it.tn * kTileN);           // columns in this tile
  const int ntp = (nt + 15) & ~15;                           // MMA N (multiple of 16)
  const int ncols = 3 * ntp <= 32 ? 32 : (3 * ntp <= 64 ? 64 : (3 * ntp <= 128 ? 128 : 256));
  const int r0 = it.tm * kM, c0 = it.tn * kTileN;
  // point range of this item, in whole chunks
  const int64_t nchunk = (K + kChunk - 1) / kChunk;
  const int64_t per = (nchunk + b.n_ranges - 1) / b.n_ranges;
  const int64_t ch0 = (int64_t)it.chunk * per, ch1 = min(nchunk, ch0 + per);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sm.tmem_base;
  const uint32_t idesc = make_idesc(ntp);

  float H[kTileN], L[kTileN];
#pragma unroll
  for (int c = 0; c < kTileN; ++c) { H[c] = 0.0f; L[c] = 0.0f; }
  bool ok = true;
  uint32_t phase = 0;

  const int row = r0 + tid;  // this thread's A row
  short2 pr = make_short2(0, 0);
  if (b.a_mode == 1 && row < b.m) pr = pairs[b.pair_off + row];

  for (int64_t ch = ch0; ch < ch1 && ok; ++ch) {
    const int64_t k0 = ch * kChunk;
    float v[kChunk];
    // ---- A row tid
    if (row < b.m) {
      if (b.a_mode == 1)
        load64(base + (int64_t)(b.a_row + pr.x) * ld, base + (int64_t)(b.a_row + pr.y) * ld, k0, K, v);
      else
        load64(base + (int64_t)(b.a_row + row) * ld, b.a_w >= 0 ? base + (int64_t)b.a_w * ld : nullptr, k0, K, v);
    } else {
#pragma unroll
      for (int i = 0; i < kChunk; ++i) v[i] = 0.0f;
    }
    sm.ea[tid] = slice_row(v, tid, sm.a[0], sm.a[1], sm.a[2]);
    // ---- B row tid (columns of the tile)
    if (tid < ntp) {
      if (tid < nt) {
        load64(base + (int64_t)(b.b_row + c0 + tid) * ld, b.b_w >= 0 ? base + (int64_t)b.b_w * ld : nullptr, k0, K,
               v);
      } else {
#pragma unroll
        for (int i = 0; i < kChunk; ++i) v[i] = 0.0f;
      }
      sm.eb[tid] = slice_row(v, tid, sm.b[0], sm.b[1], sm.b[2]);
    }
    fence_async_smem();
    __syncthreads();
    // ---- MMA issue (one thread): 4 K steps x 6 slice products into 3 accumulators
    if (tid == 0) {
      fence_after();
      const uint32_t a_addr[3] = {smem_u32(sm.a[0]), smem_u32(sm.a[1]), smem_u32(sm.a[2])};
      const uint32_t b_addr[3] = {smem_u32(sm.b[0]), smem_u32(sm.b[1]), smem_u32(sm.b[2])};
#pragma unroll
      for (int k = 0; k < kChunk / 16; ++k) {
        const uint32_t ko = 32u * k;
        // order 0
        mma_bf16(tmem + 0 * ntp, make_desc(a_addr[0] + ko), make_desc(b_addr[0] + ko), idesc, k > 0);
        // order 1
        mma_bf16(tmem + 1 * ntp, make_desc(a_addr[0] + ko), make_desc(b_addr[1] + ko), idesc, k > 0);
        mma_bf16(tmem + 1 * ntp, make_desc(a_addr[1] + ko), make_desc(b_addr[0] + ko), idesc, 1);
        // order 2
        mma_bf16(tmem + 2 * ntp, make_desc(a_addr[0] + ko), make_desc(b_addr[2] + ko), idesc, k > 0);
        mma_bf16(tmem + 2 * ntp, make_desc(a_addr[1] + ko), make_desc(b_addr[1] + ko), idesc, 1);
        mma_bf16(tmem + 2 * ntp, make_desc(a_addr[2] + ko), make_desc(b_addr[0] + ko), idesc, 1);
      }
      mma_commit(smem_u32(&sm.mbar));
    }
    __syncwarp();
    const bool done = mbar_wait(smem_u32(&sm.mbar), phase);
    if (__syncthreads_or(!done)) {  // the same decision in every thread of the CTA
      ok = false;
      if (tid == 0) atomicExch(status, 1);
      mbar_wait(smem_u32(&sm.mbar), phase);  // one more bounded wait for MMAs still in flight
    }
    phase ^= 1u;
    fence_after();
    // ---- fold the exact chunk sums into double-float accumulators
    if (ok) {
      const int ea = sm.ea[tid];
      const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
      for (int gq = 0; gq < kTileN / 16; ++gq) {
        if (gq * 16 < ntp) {
          float d0[16], d1[16], d2[16];
          tmem_ld16(lane_base + 0 * ntp + gq * 16, d0);
          tmem_ld16(lane_base + 1 * ntp + gq * 16, d1);
          tmem_ld16(lane_base + 2 * ntp + gq * 16, d2);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = gq * 16 + j;
            const float s = pow2f(ea + sm.eb[c] - 14);
            const float hi = d0[j] * s;
            const float lo = fmaf(d1[j], 0.00390625f, d2[j] * 1.52587890625e-05f) * s;
            const float t = H[c] + hi;
            const float bb = t - H[c];
            const float err = (H[c] - (t - bb)) + (hi - bb);
            H[c] = t;
            L[c] += err + lo;
          }
        }
      }
    }
    fence_before();
    __syncthreads();
  }
  // ---- write this item's partial sums (FP64)
  if (ok && row < b.m) {
    double* out = part + b.part_off + (int64_t)it.chunk * b.m * b.n;
#pragma unroll
    for (int c = 0; c < kTileN; ++c) {
      if (c < nt) {
        const double val = (double)H[c] + (double)L[c];
        if (b.transpose_out) out[(int64_t)(c0 + c) * b.m + row] = val;
        else out[(int64_t)row * b.n + c0 + c] = val;
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
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

cudaError_t launch_eval_mixed(const LaunchTables& t, const NodeEntry* tab, float* ops, cudaStream_t s) {
  if (t.n_pblocks == 0) return cudaSuccess;
  eval_mixed_kernel<<<t.n_pblocks, 128, 0, s>>>(t, tab, ops);
  return cudaGetLastError();
}

size_t mma_smem_bytes() { return sizeof(mma::Smem) + 1024; }

cudaError_t launch_contract_mma(const DevGrid* grids, const MmaBlock* blocks, const GemmItem* items, int n_items,
                                const short2* pairs, const float* ops, double* part, int* status, cudaStream_t s) {
  if (n_items == 0) return cudaSuccess;
  static bool attr_set = false;
  const size_t bytes = mma_smem_bytes();
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(contract_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  contract_mma_kernel<<<n_items, mma::kThreads, bytes, s>>>(grids, blocks, items, pairs, ops, part, status);
  return cudaGetLastError();
}

}  // namespace psq
