// FP64 kernels of the PS quadrature path: grid points and weights (Section 2.1, eqs 2-11;
// Algorithm 2), STO and aux-potential evaluation (eq 1, eqs 15-16), the weighted
// contraction of eq 9, the deterministic per-element reduction of its chunk partial sums,
// and the assembly of molecule matrices from per-grid blocks (Section 4).
#include "psq_internal.h"

#include <cstdio>

namespace psq {

__constant__ double c_glx[kMaxQ + 1][kMaxQ];  // Gauss-Legendre nodes on [-1,1], rule q
__constant__ double c_glw[kMaxQ + 1][kMaxQ];  // and weights
__constant__ double c_klm[(kMaxL + 1) * (kMaxL + 1)];  // harmonic norms, sqrt2 for m != 0
__constant__ double c_fact[2 * kMaxN + 4];             // k!
constexpr int kRcpD = 128;
__constant__ double c_rcpd[kRcpD];                     // 1/k (c_rcpd[0] unused)

void upload_gl_tables(const double* x, const double* w, const double* klm) {
  cudaMemcpyToSymbol(c_glx, x, sizeof(double) * (kMaxQ + 1) * kMaxQ);
  cudaMemcpyToSymbol(c_glw, w, sizeof(double) * (kMaxQ + 1) * kMaxQ);
  cudaMemcpyToSymbol(c_klm, klm, sizeof(double) * (kMaxL + 1) * (kMaxL + 1));
  double f[2 * kMaxN + 4];
  f[0] = 1.0;
  for (int k = 1; k < 2 * kMaxN + 4; ++k) f[k] = f[k - 1] * k;
  cudaMemcpyToSymbol(c_fact, f, sizeof(f));
  double r[kRcpD];
  r[0] = 0.0;
  for (int k = 1; k < kRcpD; ++k) r[k] = 1.0 / k;
  cudaMemcpyToSymbol(c_rcpd, r, sizeof(r));
}

// x / k for a positive integer k: a multiply by the rounded reciprocal from a table (one
// rounding more than a division, a relative 2^-52 per term; FP64 division is a long
// instruction sequence on this GPU's FP64 pipe), a division past the table.
__device__ __forceinline__ double div_int(double x, int k) { return k < kRcpD ? x * c_rcpd[k] : x / k; }

struct Pt {
  double P[3], dA[3], dB[3];
  double w, rA, rB, mu, nu;
};

// Point p of grid g.  The cell layout follows DevGrid's numbering; the node is the
// Gauss-Legendre node of each dimension mapped onto the cell, the weight is eq 10-11 with
// the Jacobian at the node, and r_A, r_B and the offsets from A and B use the forms
// 2a(sinh^2(mu/2) + sin^2(nu/2)) etc. that do not cancel near the foci.
__device__ __forceinline__ void ps_point(const DevGrid& g, const double* __restrict__ edges,
                                         int64_t p, Pt& o) {
  const int q3 = g.q_mu * g.q_nu * g.q_phi;
  const double* emu = edges + g.edge_off;
  const double* enu = emu + g.n_mu + 1;
  const double* eph = enu + g.n_nu + 1;
  int qi, qj, qk;
  double m0, m1, n0, n1, p0, p1;
  bool dead = false;
  if (p < g.K_reg) {
    const int64_t cell = p / q3;
    const int r = (int)(p - cell * q3);
    const int k = (int)(cell % g.n_phi);
    const int j = (int)((cell / g.n_phi) % g.n_nu);
    const int i = (int)(cell / ((int64_t)g.n_phi * g.n_nu));
    m0 = emu[i]; m1 = emu[i + 1];
    n0 = enu[j]; n1 = enu[j + 1];
    p0 = eph[k]; p1 = eph[k + 1];
    if (g.n_touch > 0 && i >= g.t_mu0 && i <= g.t_mu1 && j >= g.t_nu0 && j <= g.t_nu1 &&
        (g.t_phi_all || k == 0 || k == g.n_phi - 1))
      dead = true;
    qi = r / (g.q_nu * g.q_phi);
    qj = (r / g.q_phi) % g.q_nu;
    qk = r % g.q_phi;
  } else {
    const int64_t s = (p - g.K_reg) / q3;
    const int r = (int)((p - g.K_reg) - s * q3);
    const int ns = g.n_sp, ns3 = ns * ns * ns;
    const int tc = (int)(s / ns3), sub = (int)(s % ns3);
    const int ntp = g.t_phi_all ? g.n_phi : (g.n_phi == 1 ? 1 : 2);
    const int nnu = g.t_nu1 - g.t_nu0 + 1;
    const int ti = tc / (nnu * ntp), tj = (tc / ntp) % nnu, tk = tc % ntp;
    const int i = g.t_mu0 + ti, j = g.t_nu0 + tj;
    const int k = g.t_phi_all ? tk : (tk == 0 ? 0 : g.n_phi - 1);
    const int si = sub / (ns * ns), sj = (sub / ns) % ns, sk = sub % ns;
    const double M0 = emu[i], M1 = emu[i + 1], N0 = enu[j], N1 = enu[j + 1];
    const double P0 = eph[k], P1 = eph[k + 1];
    m0 = M0 + (M1 - M0) * si / ns; m1 = M0 + (M1 - M0) * (si + 1) / ns;
    n0 = N0 + (N1 - N0) * sj / ns; n1 = N0 + (N1 - N0) * (sj + 1) / ns;
    p0 = P0 + (P1 - P0) * sk / ns; p1 = P0 + (P1 - P0) * (sk + 1) / ns;
    qi = r / (g.q_nu * g.q_phi);
    qj = (r / g.q_phi) % g.q_nu;
    qk = r % g.q_phi;
  }
  const double hm = 0.5 * (m1 - m0), hn = 0.5 * (n1 - n0), hp = 0.5 * (p1 - p0);
  const double mu = 0.5 * (m0 + m1) + hm * c_glx[g.q_mu][qi];
  const double nu = 0.5 * (n0 + n1) + hn * c_glx[g.q_nu][qj];
  const double ph = 0.5 * (p0 + p1) + hp * c_glx[g.q_phi][qk];
  const double wq = (hm * c_glw[g.q_mu][qi]) * (hn * c_glw[g.q_nu][qj]) * (hp * c_glw[g.q_phi][qk]);
  const double a = g.a;
  const double sh = sinh(mu), ch = cosh(mu);
  double sn, cs, sp, cp;
  sincos(nu, &sn, &cs);
  sincos(ph, &sp, &cp);
  o.w = dead ? 0.0 : wq * (a * a * a) * sh * sn * (sh * sh + sn * sn);
  const double x = a * sh * sn * cp, y = a * sh * sn * sp, z = a * ch * cs;
  const double shm = sinh(0.5 * mu);
  double sn2, cs2;
  sincos(0.5 * nu, &sn2, &cs2);
  const double s2m = shm * shm, s2n = sn2 * sn2, c2n = cs2 * cs2;
  o.rA = 2.0 * a * (s2m + s2n);
  o.rB = 2.0 * a * (s2m + c2n);
  const double zA = 2.0 * a * (s2m * cs - s2n);
  const double zB = 2.0 * a * (s2m * cs + c2n);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double r0 = g.R[c * 3 + 0], r1 = g.R[c * 3 + 1], r2 = g.R[c * 3 + 2];
    o.P[c] = g.M[c] + (r0 * x + r1 * y + r2 * z);
    o.dA[c] = r0 * x + r1 * y + r2 * zA;
    o.dB[c] = r0 * x + r1 * y + r2 * zB;
  }
  o.mu = mu;
  o.nu = nu;
}

// Real orthonormal spherical harmonics Y_lm(u), |u| = 1, l <= lmax, index l*l + l + m:
// Y_lm = K_lm Q_l^|m|(u_z) {Re, Im}(u_x + i u_y)^|m|, with Q_m^m = (2m-1)!!,
// Q_{m+1}^m = (2m+1) u_z Q_m^m, (l-m) Q_l^m = (2l-1) u_z Q_{l-1}^m - (l+m-1) Q_{l-2}^m.
__device__ __forceinline__ void real_ylm(int lmax, double ux, double uy, double uz, double* Y) {
  double C[kMaxL + 1], S[kMaxL + 1];
  C[0] = 1.0; S[0] = 0.0;
  for (int m = 1; m <= lmax; ++m) {
    C[m] = ux * C[m - 1] - uy * S[m - 1];
    S[m] = ux * S[m - 1] + uy * C[m - 1];
  }
  double dfact = 1.0;  // (2m-1)!!
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) dfact *= (2 * m - 1);
    double q2 = 0.0, q1 = dfact;  // Q_{l-2}, Q_{l-1} as l climbs
    for (int l = m; l <= lmax; ++l) {
      double q;
      if (l == m) q = dfact;
      else if (l == m + 1) q = (2 * m + 1) * uz * dfact;
      else q = ((2 * l - 1) * uz * q1 - (l + m - 1) * q2) / (l - m);
      if (l > m) { q2 = q1; q1 = q; }
      const int base = l * l + l;
      if (m == 0) {
        Y[base] = c_klm[base] * q;
      } else {
        Y[base + m] = c_klm[base + m] * q * C[m];
        Y[base - m] = c_klm[base - m] * q * S[m];
      }
    }
  }
}

__device__ __forceinline__ double ipow(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

// Radial factor of V^P (eq 16 written out by the Laplace expansion of 1/r12):
// 4 pi/(2l+1) N [ gamma(n+l+2, zr)/(z^(n+l+2) r^(l+1)) + Gamma(n-l+1, zr) r^l / z^(n-l+1) ].
// gamma by its positive series below x = k (no cancellation), by (k-1)! - Gamma above.
__device__ double aux_pot_radial(int n, int l, double zeta, double norm, double r, double ex) {
  const double x = zeta * r;  // ex = e^-x
  const int k1 = n + l + 2, k2 = n - l + 1;
  double inner;
  if (x < (double)k1) {
    double term = c_rcpd[k1], sum = term;
#pragma unroll 1
    for (int i = 1; i < 1000; ++i) {
      term *= div_int(x, k1 + i);
      sum += term;
      if (term <= 1e-17 * sum) break;
    }
    inner = ipow(r, n + 1) * ex * sum;  // x^k1 / (z^k1 r^(l+1)) = r^(n+1)
  } else {
    double t = 1.0, s = 1.0;
#pragma unroll 1
    for (int j = 1; j < k1; ++j) { t *= div_int(x, j); s += t; }
    const double f = c_fact[k1 - 1];
    inner = (f - f * ex * s) / (ipow(zeta, k1) * ipow(r, l + 1));
  }
  double t = 1.0, s = 1.0;
#pragma unroll 1
  for (int j = 1; j < k2; ++j) { t *= div_int(x, j); s += t; }
  const double outer = c_fact[k2 - 1] * ex * s * ipow(r, l) / ipow(zeta, k2);
  return 4.0 * M_PI / (2 * l + 1) * norm * (inner + outer);
}

// Evaluates the shells [s0, s1) of one centre at distance r (ir = 1/r) for one or two row
// kinds (kind: 0 chi, 1 lap chi (kinetic operand), 2 V^P), writing from rows row_a and row_b
// (-1: not wanted) of the operand matrix; e^-zeta r is computed once per shell for both.
__device__ __forceinline__ void eval_shells(const DevShell* __restrict__ sh, int s0, int s1, double r, double ir,
                                            const double* Y, double* __restrict__ out, int64_t ld, int64_t p,
                                            int row_a, int kind_a, int row_b, int kind_b) {
  for (int s = s0; s < s1; ++s) {
    const DevShell q = sh[s];
    const double ex = exp(-q.zeta * r);
    const int base = q.l * q.l + q.l;
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int row0 = h == 0 ? row_a : row_b, kind = h == 0 ? kind_a : kind_b;
      if (row0 < 0) continue;
      double radial;
      if (kind == 2) {
        radial = aux_pot_radial(q.n, q.l, q.zeta, q.norm, r, ex);
      } else {
        radial = q.norm * ipow(r, q.n - 1) * ex;
        if (kind == 1) {
          const double f = (q.n * (q.n - 1) - q.l * (q.l + 1)) * (ir * ir) - 2.0 * q.n * q.zeta * ir +
                           q.zeta * q.zeta;
          radial *= f;
        }
      }
      for (int m = -q.l; m <= q.l; ++m)
        out[(int64_t)(row0 + q.fn0 + q.l + m) * ld + p] = radial * Y[base + m];
    }
  }
}

__device__ __forceinline__ int shells_lmax(const DevShell* sh, int s0, int s1) {
  int l = 0;
  for (int s = s0; s < s1; ++s) l = max(l, sh[s].l);
  return l;
}

// One thread per point: the point (ps_point), its weight rows and the requested function
// rows of the grid's centres.  Row layout: F/L rows are A's basis functions then B's
// (fn0 counted within each atom), G/U rows the aux functions of the grid's aux centres.
__global__ void __launch_bounds__(128) eval_fp64_kernel(LaunchTables t, double* __restrict__ ops) {
  const PointBlock pb = t.pblocks[blockIdx.x];
  const DevGrid& g = t.grids[pb.grid];
  const int64_t p = pb.p0 + threadIdx.x;
  if (p >= g.K) return;
  Pt pt;
  ps_point(g, t.edges, p, pt);
  double* base = ops + g.op_off;
  const int64_t ld = g.ld;
  double rC = 1.0, dC[3] = {0, 0, 0};
  if (g.C >= 0) {
    for (int c = 0; c < 3; ++c) dC[c] = pt.P[c] - g.RC[c];
    rC = sqrt(dC[0] * dC[0] + dC[1] * dC[1] + dC[2] * dC[2]);
  }
  if (g.row_W >= 0) {
    base[(int64_t)(g.row_W + 0) * ld + p] = pt.w;
    base[(int64_t)(g.row_W + 1) * ld + p] = pt.w / pt.rA;
    base[(int64_t)(g.row_W + 2) * ld + p] = pt.w / pt.rB;
    base[(int64_t)(g.row_W + 3) * ld + p] = g.C >= 0 ? pt.w / rC : 0.0;
  }
  double Y[(kMaxL + 1) * (kMaxL + 1)];
  // basis functions on A and B
  if (g.row_F >= 0 || g.row_L >= 0) {
    for (int c = 0; c < 2; ++c) {
      const int s0 = c == 0 ? g.shb_A0 : g.shb_B0, s1 = c == 0 ? g.shb_A1 : g.shb_B1;
      if (s1 <= s0) continue;
      const double r = c == 0 ? pt.rA : pt.rB, ir = 1.0 / r;
      const double* d = c == 0 ? pt.dA : pt.dB;
      real_ylm(shells_lmax(t.bshell, s0, s1), d[0] * ir, d[1] * ir, d[2] * ir, Y);
      const int roff = c == 0 ? 0 : g.nFA;
      eval_shells(t.bshell, s0, s1, r, ir, Y, base, ld, p, g.row_F >= 0 ? g.row_F + roff : -1, 0,
                  g.row_L >= 0 ? g.row_L + roff : -1, 1);
    }
  }
  // aux functions and their potentials
  if (g.row_G >= 0 || g.row_U >= 0) {
    int roff = 0;
    for (int c = 0; c < 2; ++c) {
      const int s0 = c == 0 ? g.sha_0 : g.sha_2, s1 = c == 0 ? g.sha_1 : g.sha_3;
      const int atom = c == 0 ? g.aux_c0 : g.aux_c1;
      if (atom < 0 || s1 <= s0) continue;
      const double* d;
      double r;
      if (atom == g.A) { d = pt.dA; r = pt.rA; }
      else if (atom == g.B) { d = pt.dB; r = pt.rB; }
      else { d = dC; r = rC; }
      const double ir = 1.0 / r;
      real_ylm(shells_lmax(t.ashell, s0, s1), d[0] * ir, d[1] * ir, d[2] * ir, Y);
      eval_shells(t.ashell, s0, s1, r, ir, Y, base, ld, p, g.row_G >= 0 ? g.row_G + roff : -1, 0,
                  g.row_U >= 0 ? g.row_U + roff : -1, 2);
      int nf = 0;
      for (int s = s0; s < s1; ++s) nf += 2 * t.ashell[s].l + 1;
      roff += nf;
    }
  }
}

cudaError_t launch_eval_fp64(const LaunchTables& t, double* ops, int /*kinds*/, cudaStream_t s) {
  if (t.n_pblocks == 0) return cudaSuccess;
  eval_fp64_kernel<<<t.n_pblocks, 128, 0, s>>>(t, ops);
  return cudaGetLastError();
}

// Weighted contraction, FP64 (eq 9): one CTA per (block, output tile, point chunk); the tile
// (tile_m x tile_n, chosen per block so that the block is covered with little padding) is
// mapped densely onto 256 threads, thread t owning outputs t, t + 256, ... of the tile's real
// rows x columns (row-major).  Per 16-point step the weighted A rows and the B columns (basis
// rows, or products of two basis rows) are formed once in shared memory; on GB300 the FP64
// pipe (a warp's DFMA every ~16 SM cycles) is the bound, so each output's sub-sum reads both
// operands from shared memory and no FP64 operation goes to padding.  Sub-sums of each step
// join the running sums (small outer-region terms are not absorbed one by one), and partial
// sums go to their own slot, so the result does not depend on scheduling.
constexpr int kFpPts = 16;
__global__ void __launch_bounds__(256) contract_fp64_kernel(LaunchTables t, const double* __restrict__ ops,
                                                             double* __restrict__ part) {
  const GemmItem it = t.items[blockIdx.x];
  const GemmBlock b = t.gblocks[it.block];
  const DevGrid& g = t.grids[b.grid];
  const double* base = ops + g.op_off;
  const int64_t ld = g.ld, K = g.K;
  const int64_t csz = (K + b.n_chunks - 1) / b.n_chunks;
  const int64_t k0 = (int64_t)it.chunk * csz;
  const int64_t k1 = min(K, k0 + csz);
  __shared__ double As[kFpPts][kFpTileRows];
  __shared__ double Bs[kFpPts][kFpTileCols];
  __shared__ short2 pr[kFpTileCols];
  const int r0 = it.tm * b.tile_m, c0 = it.tn * b.tile_n;
  const int rows = min(b.tile_m, b.m - r0), cols = min(b.tile_n, b.n - c0);
  for (int c = threadIdx.x; c < cols; c += blockDim.x)
    pr[c] = b.b_mode == 1 ? t.pairs[b.pair_off + c0 + c] : make_short2(0, 0);
  const double* drow = base + (int64_t)b.d_row * ld;
  const int nout = rows * cols;
  int orow[4], ocol[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int o = threadIdx.x + 256 * q;
    orow[q] = o < nout ? o / cols : 0;
    ocol[q] = o < nout ? o - (o / cols) * cols : 0;
  }
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  __syncthreads();
  for (int64_t k = k0; k < k1; k += kFpPts) {
    // operands of this step: A rows x points, B columns x points (zeros past the chunk)
    for (int e = threadIdx.x; e < rows * kFpPts; e += blockDim.x) {
      const int r = e / kFpPts, pp = e - r * kFpPts;
      const int64_t kk = k + pp;
      As[pp][r] = kk < k1 ? base[(int64_t)(b.a_row + r0 + r) * ld + kk] * drow[kk] : 0.0;
    }
    for (int e = threadIdx.x; e < cols * kFpPts; e += blockDim.x) {
      const int c = e / kFpPts, pp = e - c * kFpPts;
      const int64_t kk = k + pp;
      double bv = 0.0;
      if (kk < k1) {
        if (b.b_mode == 0) {
          bv = base[(int64_t)(b.b_row + c0 + c) * ld + kk];
        } else {
          const short2 q = pr[c];
          bv = base[(int64_t)(b.b_row + q.x) * ld + kk] * base[(int64_t)(b.b_row + q.y) * ld + kk];
        }
      }
      Bs[pp][c] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (threadIdx.x + 256 * q < nout) {
        double sq = 0.0;
#pragma unroll
        for (int pp = 0; pp < kFpPts; ++pp) sq = fma(As[pp][orow[q]], Bs[pp][ocol[q]], sq);
        acc[q] += sq;
      }
    }
    __syncthreads();
  }
  double* out = part + b.part_off + (int64_t)it.chunk * b.m * b.n;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (threadIdx.x + 256 * q < nout) out[(int64_t)(r0 + orow[q]) * b.n + c0 + ocol[q]] = acc[q];
}

cudaError_t launch_contract_fp64(const LaunchTables& t, const double* ops, double* part, cudaStream_t s) {
  if (t.n_items == 0) return cudaSuccess;
  contract_fp64_kernel<<<t.n_items, 256, 0, s>>>(t, ops, part);
  return cudaGetLastError();
}

// Per-element reduction of chunk partials: one warp per output element, lanes stride the
// chunks in a fixed order and combine by a shuffle tree (deterministic).
__global__ void __launch_bounds__(256) reduce_kernel(LaunchTables t, const double* __restrict__ part,
                                                      double* __restrict__ res) {
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= t.n_elems) return;
  int lo = 0, hi = t.n_gblocks;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (t.elem_begin[mid] <= wid) lo = mid; else hi = mid;
  }
  const GemmBlock b = t.gblocks[lo];
  const int64_t e = wid - t.elem_begin[lo];
  const int64_t mn = (int64_t)b.m * b.n;
  double s = 0.0;
  for (int c = lane; c < b.n_chunks; c += 32) s += part[b.part_off + c * mn + e];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) res[b.res_off + e] = s;
}

cudaError_t launch_reduce(const LaunchTables& t, const double* part, double* res, cudaStream_t s) {
  if (t.n_elems == 0) return cudaSuccess;
  const int64_t threads = t.n_elems * 32;
  reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(t, part, res);
  return cudaGetLastError();
}

// k! / z^(k+1) = int_0^inf r^k e^(-z r) dr (k >= 0), as a product of k + 1 factors.
__device__ double radial_moment(int k, double z) {
  double v = 1.0 / z;
  for (int i = 1; i <= k; ++i) v *= (double)i / z;
  return v;
}

// One-centre overlap (cls 1) or kinetic (cls 2) element of two basis functions of one atom,
// from the closed forms of eq 1's functions: with I(k) = k! / (zeta_a + zeta_b)^(k+1), for the
// same l and m S = N_a N_b I(n_a + n_b) and T = -1/2 N_a N_b [(n_b (n_b - 1) - l (l + 1))
// I(n_a + n_b - 2) - 2 n_b zeta_b I(n_a + n_b - 1) + zeta_b^2 I(n_a + n_b)] (the radial
// Laplacian written out), symmetrised; 0 for different l or m.
__device__ double one_centre_st(int cls, const DevShell& A, int ma, const DevShell& B, int mb) {
  if (A.l != B.l || ma != mb) return 0.0;
  const double z = A.zeta + B.zeta, nn = A.norm * B.norm;
  const int k = A.n + B.n;
  if (cls == 1) return nn * radial_moment(k, z);
  const double ll = (double)(A.l * (A.l + 1));
  const double i2 = radial_moment(k - 2, z), i1 = radial_moment(k - 1, z), i0 = radial_moment(k, z);
  const double tab = (B.n * (B.n - 1) - ll) * i2 - 2.0 * B.n * B.zeta * i1 + B.zeta * B.zeta * i0;
  const double tba = (A.n * (A.n - 1) - ll) * i2 - 2.0 * A.n * A.zeta * i1 + A.zeta * A.zeta * i0;
  return -0.25 * nn * (tab + tba);
}

// Molecule matrices from per-grid blocks.  cls: 1 S, 2 T, 4 V, 8 J2 (two-index), 16 J3.
// With `shells`, one-centre elements take their closed forms (S and T).
__global__ void assemble2_kernel(int cls, int nat, int nfn, const int* __restrict__ fn_atom,
                                 const int* __restrict__ fn_local, const SrcEntry* __restrict__ src,
                                 const int* __restrict__ src_ptr, const DevShell* __restrict__ shells,
                                 const int* __restrict__ fn_shell, const double* __restrict__ res,
                                 double* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)nfn * nfn) return;
  const int a = (int)(idx / nfn), b = (int)(idx % nfn);
  int X = fn_atom[a], Y = fn_atom[b], la = fn_local[a], lb = fn_local[b];
  if (shells && X == Y) {
    const DevShell& A = shells[fn_shell[a]];
    const DevShell& B = shells[fn_shell[b]];
    out[idx] = one_centre_st(cls, A, la - A.fn0, B, lb - B.fn0);
    return;
  }
  if (X > Y) { int t = X; X = Y; Y = t; t = la; la = lb; lb = t; }
  double v = 0.0;
  for (int e = src_ptr[X * nat + Y]; e < src_ptr[X * nat + Y + 1]; ++e) {
    const SrcEntry s = src[e];
    const double* M = res + s.off;
    if (s.mode == 0) {
      const double m1 = M[(int64_t)(s.rX + la) * s.ld + s.cY + lb];
      if (cls == 2 || cls == 8 || X == Y) {
        const double* M2 = s.ld2 > 0 ? res + s.off2 : M;
        const double m2 = M2[(int64_t)(s.rY + lb) * (s.ld2 > 0 ? s.ld2 : s.ld) + s.cX + la];
        v += (cls == 2 ? -0.25 : s.z * 0.5) * (m1 + m2);
      } else {
        v += s.z * m1;
      }
    } else {
      int64_t p;
      if (s.mode == 1) {
        const int i = min(s.rX + la, s.cY + lb), j = max(s.rX + la, s.cY + lb);
        p = (int64_t)i * s.nloc - (int64_t)i * (i - 1) / 2 + (j - i);
      } else {
        p = (int64_t)la * s.nloc + lb;
      }
      v += s.z * M[p * s.ld + (int64_t)s.cX * s.cs];
    }
  }
  out[idx] = v;
}

__global__ void assemble3_kernel(int nat, int nfn, int naux, const int* __restrict__ fn_atom,
                                 const int* __restrict__ fn_local, const int* __restrict__ aux_atom,
                                 const int* __restrict__ aux_local, const J3Src* __restrict__ j3,
                                 const double* __restrict__ res, double* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nn = (int64_t)nfn * nfn;
  if (idx >= nn * naux) return;
  const int P = (int)(idx / nn);
  const int a = (int)((idx / nfn) % nfn), b = (int)(idx % nfn);
  const int X = aux_atom[P], lp = aux_local[P];
  int Y = fn_atom[a], W = fn_atom[b], la = fn_local[a], lb = fn_local[b];
  if (Y > W) { int t = Y; Y = W; W = t; t = la; la = lb; lb = t; }
  const J3Src s = j3[((int64_t)X * nat + Y) * nat + W];
  int64_t pidx;
  const int i0 = s.offY + la, j0 = s.offW + lb;
  if (s.mode == 1) {
    const int i = min(i0, j0), j = max(i0, j0);
    pidx = (int64_t)i * s.nloc - (int64_t)i * (i - 1) / 2 + (j - i);
  } else {
    pidx = (int64_t)i0 * s.nloc + j0;
  }
  out[idx] = res[s.off + pidx * s.s_pair + (int64_t)lp * s.s_aux];
}

cudaError_t launch_assemble(int cls, int nat, int nfn, int naux, const int* fn_atom,
                            const int* fn_local, const int* aux_atom, const int* aux_local,
                            const SrcEntry* src, const int* src_ptr, const J3Src* j3,
                            const DevShell* shells, const int* fn_shell, const double* res, double* out,
                            cudaStream_t s) {
  if (cls == 16) {
    const int64_t n = (int64_t)naux * nfn * nfn;
    if (n == 0) return cudaSuccess;
    assemble3_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nat, nfn, naux, fn_atom, fn_local,
                                                                aux_atom, aux_local, j3, res, out);
  } else {
    const int64_t n = (int64_t)nfn * nfn;
    if (n == 0) return cudaSuccess;
    assemble2_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cls, nat, nfn, fn_atom, fn_local,
                                                                src, src_ptr, shells, fn_shell, res, out);
  }
  return cudaGetLastError();
}

// Diagnostics: the points of one grid (8 rows: x, y, z, w, r_A, r_B, mu, nu).
__global__ void grid_points_kernel(const DevGrid* grids, int gi, const double* edges, double* out) {
  const DevGrid& g = grids[gi];
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.K) return;
  Pt pt;
  ps_point(g, edges, p, pt);
  const int64_t K = g.K;
  out[0 * K + p] = pt.P[0];
  out[1 * K + p] = pt.P[1];
  out[2 * K + p] = pt.P[2];
  out[3 * K + p] = pt.w;
  out[4 * K + p] = pt.rA;
  out[5 * K + p] = pt.rB;
  out[6 * K + p] = pt.mu;
  out[7 * K + p] = pt.nu;
}

cudaError_t launch_grid_points(const LaunchTables& t, int g, double* out, cudaStream_t s) {
  // the point count is on the device; the host passes it through n_elems
  const int64_t K = t.n_elems;
  if (K == 0) return cudaSuccess;
  grid_points_kernel<<<(unsigned)((K + 255) / 256), 256, 0, s>>>(t.grids, g, t.edges, out);
  return cudaGetLastError();
}

}  // namespace psq
