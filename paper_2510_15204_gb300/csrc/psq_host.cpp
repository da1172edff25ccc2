// Host side of the PS quadrature library: C ABI, input validation, the planner that turns a
// job (atoms, shells, grid specs) into device tables, and the launch sequence.
//
// Planner steps (independent of any other implementation in this repository):
//  * pair frames (Section 2.1: foci at (0,0,+-a), grid rotated and translated onto a pair);
//  * cell edges: mu = C1 atanh(i/(N_mu+1)), C1 = 2.3 a^(1/4); nu = j pi/N_nu; phi = 2 pi k/N_phi
//    (eqs 7, 12, 17; Section 2.3);
//  * third centre (Section 2.2, Fig. 2): frame turned so the centre sits at phi = 0, the
//    nearest interior mu and nu lines moved onto it, the cells that touch it split N_SP ways;
//  * assembly over grids of at most three atoms (Section 4): every matrix element is taken
//    from one grid chosen by the distinct centres of its integrand;
//  * Gauss-Legendre nodes (Newton on the Legendre recurrence) and harmonic norms.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/psq.h"
#include "psq_internal.h"

using namespace psq;

namespace {

thread_local std::string g_err;

psq_status fail(psq_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CUDA_TRY(expr)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(PSQ_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                            \
  } while (0)

constexpr double kOnAxisTol = 1e-10;  // a third centre this close (x a) to the axis is on it
constexpr int kPointsPerBlock = 128;
constexpr int64_t kMaxChunkPoints = 32768;  // FP64 path: points per sequential partial sum
constexpr int kSmCount = 152;
constexpr size_t kDefaultWaveBytes = (size_t)6 << 30;  // mixed path: operand + packed bytes per wave

// Gauss-Legendre rule by Newton's method on P_q (Bonnet recurrence); nodes ascending.
void gauss_legendre(int q, double* x, double* w) {
  for (int i = 0; i < q; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= q; ++k) {
        const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (q == 1) p0 = 1.0;
      dp = q * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= q; ++k) {
      const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    if (q == 1) p0 = 1.0;
    dp = q * (z * p1 - p0) / (z * z - 1.0);
    x[q - 1 - i] = z;  // z runs from the largest node down
    w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

struct Vec3 {
  double x, y, z;
};
Vec3 sub(Vec3 a, Vec3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
Vec3 add(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
Vec3 scale(Vec3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
double dot(Vec3 a, Vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
double norm(Vec3 a) { return std::sqrt(dot(a, a)); }
Vec3 cross(Vec3 a, Vec3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }

}  // namespace

struct psq_context {
  int device;
  int sm_count = 152;
};

namespace {

// Everything psq_compute needs for one class mask.
struct Plan {
  unsigned mask = 0;
  std::vector<DevGrid> grids;
  std::vector<double> edges;
  std::vector<PointBlock> pblocks;
  std::vector<GemmBlock> gblocks;
  std::vector<GemmItem> items;
  std::vector<short2> pairs;
  std::vector<int64_t> elem_begin;
  // assembly sources
  std::vector<SrcEntry> src[4];
  std::vector<int> src_ptr[4];
  std::vector<J3Src> j3;
  // workspace layout (bytes)
  size_t table_bytes = 0, ops_off = 0, part_off = 0, res_off = 0, ws_bytes = 0;
  size_t o_grids, o_edges, o_bsh, o_ash, o_xyz, o_pb, o_gb, o_it, o_pairs, o_eb;
  size_t o_fa, o_fl, o_fs, o_aa, o_al, o_src[4], o_ptr[4], o_j3, o_status;
  // mixed path
  bool mixed = false;
  std::vector<MmaBlock> mblocks;
  std::vector<GemmItem> mitems;
  std::vector<Panel> panels;
  std::vector<PairTile> ptiles;
  int64_t n_pack_jobs = 0, pack_bytes = 0;
  std::vector<int> cta_begin;  // contraction: CTA b of wave k takes items [cta_begin[cb_off + b], .. + 1])
  int n_ctas = 0;
  // Waves (mixed path): consecutive grids whose operand rows and packed panels fit the wave
  // budget together; each wave runs evaluation, packing, contraction and range reduction in
  // the shared operand / packed / partial regions (offsets of its grids, panels and blocks
  // are relative to them), the blocks' results stay in the one result region.
  struct Wave {
    int g0, g1, pb0, pb1, pn0, pn1, mb0, mb1, cb_off, n_ctas;
    int64_t jobs;
    int64_t ph_off;  // its panel hint table in pack_hint
  };
  std::vector<int> pack_hint;  // per wave, per kPackHintJobs packing jobs: the panel of the first
  size_t o_ph = 0;
  std::vector<Wave> waves;
  size_t o_cb = 0;
  size_t o_mb = 0, o_mi = 0, o_pn = 0, o_pt = 0, nodes_off = 0, o_xi = 0, o_rc = 0, pack_off = 0;
  std::vector<float2> xi;    // per grid: (hi, lo) scale turning rho into x = zeta r, per shell
  std::vector<double> rowc;  // per grid: FP64 constant of every operand row
  int64_t n_nodes = 0;
  int max_node_entries = 0;
  int64_t n_ops = 0;  // operand elements (mixed path: the lo plane follows the hi plane)
  double* staging = nullptr;  // copy of the tables, page-locked when pinned
  bool pinned = false;
  int64_t n_points = 0;
  double contractions = 0;
  double issued_flops = 0;
  int launches = 0;
  int work_split = 16;  // work items (mixed) or 8-CTA waves (FP64) per SM; psq_job_autotune picks it
  ~Plan() {
    if (staging && pinned) cudaFreeHost(staging);
    if (staging && !pinned) std::free(staging);
  }
};

}  // namespace

struct psq_job {
  psq_context* ctx;
  int nat;
  std::vector<psq_atom> atoms;
  std::vector<psq_shell> basis, aux;
  std::vector<psq_grid_spec> specs;
  psq_precision prec;
  std::vector<int> nb, na, sb0, sb1, sa0, sa1, fn_atom, fn_local, aux_atom, aux_local, nn;
  std::vector<int> fn_shell;  // basis function -> its shell (index into dbs)
  std::vector<DevShell> dbs, das;
  int nbf = 0, naux = 0;
  std::map<unsigned, std::shared_ptr<Plan>> plans;  // shared: a running compute keeps its plan alive
  std::map<unsigned, int> work_split;  // per mask, chosen by psq_job_autotune
  uint64_t wait_ns = 4000000000ull;    // limit of every bounded device wait (psq_job_set_wait_limit)
  size_t wave_bytes = 0;               // mixed path: operand + packed bytes per wave (0: default)
  bool test_stall = false;             // failure-detection test hook (psq_job_test_stall)
  std::mutex mu;
  // launch timing: events recorded on the compute stream, read back on request
  struct ProfRec { int kind; cudaEvent_t ev; };
  bool prof_on = false;
  bool capturing = false;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_free;
  // instantiated CUDA graphs of the launch sequence, per (mask, workspace, outputs)
  struct GraphKey {
    unsigned mask;
    void* ws;
    double* out[5];
    bool operator<(const GraphKey& o) const {
      if (mask != o.mask) return mask < o.mask;
      if (ws != o.ws) return ws < o.ws;
      for (int c = 0; c < 5; ++c)
        if (out[c] != o.out[c]) return out[c] < o.out[c];
      return false;
    }
  };
  std::map<GraphKey, cudaGraphExec_t> graphs;
  ~psq_job() {
    for (auto& r : prof) cudaEventDestroy(r.ev);
    for (auto e : ev_free) cudaEventDestroy(e);
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
  }
};

namespace {

Vec3 pos(const psq_job* j, int X) { return {j->atoms[X].xyz[0], j->atoms[X].xyz[1], j->atoms[X].xyz[2]}; }

const psq_grid_spec& spec_for(const psq_job* j, int A, int B) {
  if (j->specs.size() == 1) return j->specs[0];
  if (A > B) std::swap(A, B);
  const int n = j->nat;
  return j->specs[A * n - A * (A + 1) / 2 + (B - A - 1)];
}

// Grid of the term with basis atoms A, B and operator / aux atom C, by its distinct centres.
struct GridKey {
  int A, B, C;  // C = -1: unrefined pair grid
  bool operator<(const GridKey& o) const {
    if (A != o.A) return A < o.A;
    if (B != o.B) return B < o.B;
    return C < o.C;
  }
};

GridKey grid_for(const psq_job* j, int A, int B, int C) {
  int s[3] = {A, B, C};
  std::sort(s, s + 3);
  const int nd = 1 + (s[1] != s[0]) + (s[2] != s[1]);
  if (nd == 1) {
    const int X = s[0], Y = j->nn[X];
    return {std::min(X, Y), std::max(X, Y), -1};
  }
  if (nd == 2) return {s[0], s[2], -1};
  return {std::min(A, B), std::max(A, B), C};
}

// Pair frame and third-centre placement of one grid.
psq_status build_grid(const psq_job* j, GridKey key, DevGrid& g, std::vector<double>& edges) {
  std::memset(&g, 0, sizeof(g));
  const psq_grid_spec& sp = spec_for(j, key.A, key.B);
  const Vec3 RA = pos(j, key.A), RB = pos(j, key.B);
  const Vec3 d = sub(RA, RB);
  const double R = norm(d);
  const double a = 0.5 * R;
  const Vec3 M = scale(add(RA, RB), 0.5);
  const Vec3 ez = scale(d, 1.0 / R);
  Vec3 ex{0, 0, 0};
  bool have_ex = false;
  Vec3 RC{0, 0, 0};
  if (key.C >= 0) {
    RC = pos(j, key.C);
    const Vec3 v = sub(RC, M);
    const Vec3 perp = sub(v, scale(ez, dot(v, ez)));
    const double pn = norm(perp);
    if (pn > kOnAxisTol * a) {
      ex = scale(perp, 1.0 / pn);
      have_ex = true;
    }
  }
  if (!have_ex) {
    Vec3 e{1, 0, 0};
    ex = sub(e, scale(ez, dot(e, ez)));
    if (norm(ex) < 0.5) {
      e = {0, 1, 0};
      ex = sub(e, scale(ez, dot(e, ez)));
    }
    ex = scale(ex, 1.0 / norm(ex));
  }
  const Vec3 ey = cross(ez, ex);
  const Vec3 axes[3] = {ex, ey, ez};
  for (int c = 0; c < 3; ++c) {
    g.R[c * 3 + 0] = c == 0 ? axes[0].x : (c == 1 ? axes[0].y : axes[0].z);
    g.R[c * 3 + 1] = c == 0 ? axes[1].x : (c == 1 ? axes[1].y : axes[1].z);
    g.R[c * 3 + 2] = c == 0 ? axes[2].x : (c == 1 ? axes[2].y : axes[2].z);
  }
  g.M[0] = M.x; g.M[1] = M.y; g.M[2] = M.z;
  g.a = a;
  g.A = key.A; g.B = key.B; g.C = key.C;
  g.n_mu = sp.n_mu; g.n_nu = sp.n_nu; g.n_phi = sp.n_phi;
  g.q_mu = sp.q_mu; g.q_nu = sp.q_nu; g.q_phi = sp.q_phi; g.n_sp = sp.n_sp;
  // cell edges (eqs 7, 12, 17)
  std::vector<double> mu(sp.n_mu + 1), nu(sp.n_nu + 1), ph(sp.n_phi + 1);
  const double C1 = 2.3 * std::pow(a, 0.25);
  for (int i = 0; i <= sp.n_mu; ++i) mu[i] = C1 * std::atanh(i / (sp.n_mu + 1.0));
  for (int i = 0; i <= sp.n_nu; ++i) nu[i] = M_PI * i / sp.n_nu;
  for (int i = 0; i <= sp.n_phi; ++i) ph[i] = 2.0 * M_PI * i / sp.n_phi;
  g.n_touch = 0;
  if (key.C >= 0) {
    if (sp.n_mu < 2 || sp.n_nu < 2)
      return fail(PSQ_ERR_ARG, "a refined grid needs n_mu >= 2 and n_nu >= 2");
    g.RC[0] = RC.x; g.RC[1] = RC.y; g.RC[2] = RC.z;
    const Vec3 v = sub(RC, M);
    const double xc = dot(v, ex), yc = dot(v, ey), zc = dot(v, ez);
    const double rho = std::hypot(xc, yc);
    const double rA = std::hypot(rho, zc - a), rB = std::hypot(rho, zc + a);
    const double mu_c = std::acosh(std::max(1.0, (rA + rB) / (2 * a)));
    const double nu_c = std::acos(std::min(1.0, std::max(-1.0, (rB - rA) / (2 * a))));
    if (mu_c < mu[sp.n_mu]) {
      const bool on_axis = rho <= kOnAxisTol * a;
      if (on_axis && std::fabs(zc) < a) {
        g.t_mu0 = g.t_mu1 = 0;
      } else {
        int best = 1;
        for (int i = 2; i <= sp.n_mu - 1; ++i)
          if (std::fabs(mu[i] - mu_c) < std::fabs(mu[best] - mu_c)) best = i;
        mu[best] = mu_c;
        g.t_mu0 = best - 1;
        g.t_mu1 = best;
      }
      if (on_axis && std::fabs(zc) >= a) {
        g.t_nu0 = g.t_nu1 = zc > 0 ? 0 : sp.n_nu - 1;
      } else {
        int best = 1;
        for (int i = 2; i <= sp.n_nu - 1; ++i)
          if (std::fabs(nu[i] - nu_c) < std::fabs(nu[best] - nu_c)) best = i;
        nu[best] = nu_c;
        g.t_nu0 = best - 1;
        g.t_nu1 = best;
      }
      g.t_phi_all = on_axis ? 1 : 0;
      const int nph = on_axis ? sp.n_phi : (sp.n_phi == 1 ? 1 : 2);
      g.n_touch = (g.t_mu1 - g.t_mu0 + 1) * (g.t_nu1 - g.t_nu0 + 1) * nph;
      g.nt_mu = g.t_mu1 - g.t_mu0 + 1;
      g.nt_nu = g.t_nu1 - g.t_nu0 + 1;
      g.nt_phi = nph;
    }
    g.xc = xc;
    g.zc = zc;
  }
  g.edge_off = (int)edges.size();
  edges.insert(edges.end(), mu.begin(), mu.end());
  edges.insert(edges.end(), nu.begin(), nu.end());
  edges.insert(edges.end(), ph.begin(), ph.end());
  const int64_t q3 = (int64_t)sp.q_mu * sp.q_nu * sp.q_phi;
  g.K_reg = (int64_t)sp.n_mu * sp.n_nu * sp.n_phi * q3;
  g.K = g.K_reg + (int64_t)g.n_touch * sp.n_sp * sp.n_sp * sp.n_sp * q3;
  if (g.K > ((int64_t)1 << 31) - 256)  // point indices are 32-bit in the kernels
    return fail(PSQ_ERR_UNSUPPORTED, "a grid with its split cells has more than 2^31 - 256 points");
  return PSQ_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

double klm_norm(int l, int m) {
  const int am = std::abs(m);
  const double k = std::sqrt((2 * l + 1) / (4 * M_PI) * factorial(l - am) / factorial(l + am));
  return m != 0 ? k * std::sqrt(2.0) : k;
}

// FP64 constants of the mixed path's operand rows of one kind on grid g (kind 0 basis chi,
// 1 lap chi, 2 aux chi, 3 aux V^P; rows in function order of the grid's centres): the FP32/df
// row values are functions of x = zeta r and of the direction only, times
//   chi: N K_lm zeta^-(n-1);  lap chi: N K_lm zeta^-(n-1) zeta^2;
//   V^P: 4 pi/(2l+1) N K_lm zeta^-(n+1)  (eq 16 through the Laplace expansion).
void row_constants(const psq_job* j, const DevGrid& g, int kind, std::vector<double>& out) {
  if (kind <= 1) {
    for (int c = 0; c < 2; ++c) {
      const int s0 = c == 0 ? g.shb_A0 : g.shb_B0, s1 = c == 0 ? g.shb_A1 : g.shb_B1;
      for (int q = s0; q < s1; ++q) {
        const DevShell& d = j->dbs[q];
        for (int m = -d.l; m <= d.l; ++m)
          out.push_back(d.norm * klm_norm(d.l, m) * std::pow(d.zeta, -(d.n - 1) + (kind == 1 ? 2.0 : 0.0)));
      }
    }
    return;
  }
  for (int c = 0; c < 2; ++c) {
    const int s0 = c == 0 ? g.sha_0 : g.sha_2, s1 = c == 0 ? g.sha_1 : g.sha_3;
    if ((c == 0 ? g.aux_c0 : g.aux_c1) < 0) continue;
    for (int q = s0; q < s1; ++q) {
      const DevShell& d = j->das[q];
      for (int m = -d.l; m <= d.l; ++m)
        out.push_back(kind == 3 ? 4.0 * M_PI / (2 * d.l + 1) * d.norm * klm_norm(d.l, m) * std::pow(d.zeta, -(d.n + 1))
                                : d.norm * klm_norm(d.l, m) * std::pow(d.zeta, -(d.n - 1)));
    }
  }
}

psq_status make_plan(psq_job* j, unsigned mask, Plan& P) {
  P.mask = mask;
  const int nat = j->nat;
  // grids: every pair, then every (pair, third centre) when a 3-centre class is asked
  std::vector<GridKey> keys;
  for (int A = 0; A < nat; ++A)
    for (int B = A + 1; B < nat; ++B) keys.push_back({A, B, -1});
  if ((mask & (PSQ_V | PSQ_J3)) && nat >= 3)
    for (int A = 0; A < nat; ++A)
      for (int B = A + 1; B < nat; ++B)
        for (int C = 0; C < nat; ++C)
          if (C != A && C != B) keys.push_back({A, B, C});
  if (mask == 0) keys.clear();
  std::map<GridKey, int> gidx;
  for (size_t i = 0; i < keys.size(); ++i) gidx[keys[i]] = (int)i;
  P.grids.resize(keys.size());
  for (size_t i = 0; i < keys.size(); ++i) {
    psq_status st = build_grid(j, keys[i], P.grids[i], P.edges);
    if (st != PSQ_OK) return st;
  }
  // operand rows and shells per grid
  P.mixed = j->prec == PSQ_MIXED;
  const size_t esize = P.mixed ? sizeof(float) : sizeof(double);
  int64_t ops = 0;  // elements
  for (auto& g : P.grids) {
    const bool refined = g.C >= 0;
    g.nFA = j->nb[g.A];
    g.nFB = j->nb[g.B];
    g.shb_A0 = j->sb0[g.A]; g.shb_A1 = j->sb1[g.A];
    g.shb_B0 = j->sb0[g.B]; g.shb_B1 = j->sb1[g.B];
    if (refined) {
      g.aux_c0 = g.C; g.aux_c1 = -1;
      g.sha_0 = j->sa0[g.C]; g.sha_1 = j->sa1[g.C]; g.sha_2 = g.sha_3 = 0;
      g.nG = j->na[g.C];
    } else {
      g.aux_c0 = g.A; g.aux_c1 = g.B;
      g.sha_0 = j->sa0[g.A]; g.sha_1 = j->sa1[g.A];
      g.sha_2 = j->sa0[g.B]; g.sha_3 = j->sa1[g.B];
      g.nG = j->na[g.A] + j->na[g.B];
    }
    const int nl = g.nFA + g.nFB;
    int rows = 0;
    g.row_F = g.row_L = g.row_G = g.row_U = -1;
    if (!refined) {
      if (mask & (PSQ_S | PSQ_T | PSQ_V | PSQ_J3)) { g.row_F = rows; rows += nl; }
      if (mask & PSQ_T) { g.row_L = rows; rows += nl; }
      if (mask & PSQ_J2) { g.row_G = rows; rows += g.nG; }
      if (mask & (PSQ_J2 | PSQ_J3)) { g.row_U = rows; rows += g.nG; }
    } else {
      g.row_F = rows; rows += nl;
      if (mask & PSQ_J3) { g.row_U = rows; rows += g.nG; }
    }
    g.row_W = rows;
    rows += 4;
    g.ld = (int64_t)align_up((size_t)g.K, 128);
    g.op_off = ops;
    ops += (int64_t)rows * g.ld;
    P.n_points += g.K;
  }
  // contraction blocks and assembly sources
  int64_t res = 0, part = 0;
  auto local_off = [&](const DevGrid& g, int X) { return X == g.A ? 0 : g.nFA; };
  auto aux_off = [&](const DevGrid& g, int X) { return X == g.A ? 0 : j->na[g.A]; };
  for (int c = 0; c < 4; ++c) P.src_ptr[c].assign(nat * nat + 1, 0);
  P.j3.assign((size_t)nat * nat * nat, J3Src{0, 0, 0, 0, 0, 0, 0});
  auto J3at = [&](int X, int Y, int W) -> J3Src& { return P.j3[((size_t)X * nat + Y) * nat + W]; };
  if (!P.mixed) {
    // FP64 path: one block per (grid, class) and per (grid, aux atom, basis atom pair)
    // On a pair grid (A < B) only the blocks that some element reads: S the A x B block (the
    // one-centre S and T come from their closed forms); T the A x B block and its mirror
    // (B rows against A's kinetic columns), averaged; (P|Q) the A x B block and its mirror, and
    // the A x A (B x B) block where the grid is A's (B's) one-centre grid; V_ne of nucleus A the
    // A x B block, the B x B block (B's functions in A's field) and the A x A block where the
    // grid is A's one-centre grid (and likewise for nucleus B).
    struct Fp2 { int64_t ab = -1, ba = -1, aa = -1, bb = -1; };
    std::vector<int64_t> s_loc(P.grids.size(), -1), vc_loc(P.grids.size(), -1);
    std::vector<Fp2> t_loc(P.grids.size()), j2_loc(P.grids.size()), va_loc(P.grids.size()), vb_loc(P.grids.size());
    auto own_grid = [&](const DevGrid& g, int X) {
      const GridKey k = grid_for(j, X, X, X);
      return k.A == g.A && k.B == g.B && k.C == -1;
    };
    auto add_block = [&](int g, int a_row, int m, int b_row, int n, int b_mode, int pair_off, int d_row) {
      GemmBlock b{};
      b.grid = g; b.a_row = a_row; b.m = m; b.b_row = b_row; b.n = n; b.b_mode = b_mode;
      b.pair_off = pair_off; b.d_row = d_row; b.res_off = res;
      res += (int64_t)m * n;
      P.gblocks.push_back(b);
      return b.res_off;
    };
    for (size_t gi = 0; gi < P.grids.size(); ++gi) {
      DevGrid& g = P.grids[gi];
      const int nl = g.nFA + g.nFB;
      const int w = g.row_W;
      const int gint = (int)gi;
      if (g.C < 0) {
        if (g.nFA > 0 && g.nFB > 0) {
          if (mask & PSQ_S) s_loc[gi] = add_block(gint, g.row_F, g.nFA, g.row_F + g.nFA, g.nFB, 0, 0, w);
          if (mask & PSQ_T) {
            t_loc[gi].ab = add_block(gint, g.row_F, g.nFA, g.row_L + g.nFA, g.nFB, 0, 0, w);
            t_loc[gi].ba = add_block(gint, g.row_F + g.nFA, g.nFB, g.row_L, g.nFA, 0, 0, w);
          }
        }
        if (mask & PSQ_V) {
          const bool oA = own_grid(g, g.A), oB = own_grid(g, g.B);
          for (int c = 0; c < 2; ++c) {  // nucleus A (weight row w + 1), nucleus B (w + 2)
            Fp2& v = c == 0 ? va_loc[gi] : vb_loc[gi];
            if (g.nFA > 0 && g.nFB > 0) v.ab = add_block(gint, g.row_F, g.nFA, g.row_F + g.nFA, g.nFB, 0, 0, w + 1 + c);
            if (g.nFA > 0 && (c == 1 || oA)) v.aa = add_block(gint, g.row_F, g.nFA, g.row_F, g.nFA, 0, 0, w + 1 + c);
            if (g.nFB > 0 && (c == 0 || oB))
              v.bb = add_block(gint, g.row_F + g.nFA, g.nFB, g.row_F + g.nFA, g.nFB, 0, 0, w + 1 + c);
          }
        }
        if (mask & PSQ_J2) {
          const int naA = j->na[g.A], naB = j->na[g.B];
          if (naA > 0 && naB > 0) {
            j2_loc[gi].ab = add_block(gint, g.row_U, naA, g.row_G + naA, naB, 0, 0, w);
            j2_loc[gi].ba = add_block(gint, g.row_U + naA, naB, g.row_G, naA, 0, 0, w);
          }
          if (naA > 0 && own_grid(g, g.A)) j2_loc[gi].aa = add_block(gint, g.row_U, naA, g.row_G, naA, 0, 0, w);
          if (naB > 0 && own_grid(g, g.B))
            j2_loc[gi].bb = add_block(gint, g.row_U + naA, naB, g.row_G + naA, naB, 0, 0, w);
        }
        if (mask & PSQ_J3) {
          const int atoms2[2] = {g.A, g.B};
          for (int xi = 0; xi < 2; ++xi) {
            const int X = atoms2[xi];
            if (j->na[X] == 0) continue;
            const int aoff = xi == 0 ? 0 : j->na[g.A];
            const int yw[3][2] = {{g.A, g.A}, {g.A, g.B}, {g.B, g.B}};
            for (auto& pq : yw) {
              const int Y = pq[0], W = pq[1];
              if (j->nb[Y] == 0 || j->nb[W] == 0) continue;
              const GridKey k = grid_for(j, Y, W, X);
              if (k.A != g.A || k.B != g.B || k.C != -1) continue;
              const int yoff = Y == g.A ? 0 : g.nFA, woff = W == g.A ? 0 : g.nFA;
              const int pair_off = (int)P.pairs.size();
              if (Y != W) {
                for (int i = 0; i < j->nb[Y]; ++i)
                  for (int jj = 0; jj < j->nb[W]; ++jj) P.pairs.push_back(make_short2(yoff + i, woff + jj));
              } else {
                for (int i = 0; i < j->nb[Y]; ++i)
                  for (int jj = i; jj < j->nb[Y]; ++jj) P.pairs.push_back(make_short2(yoff + i, yoff + jj));
              }
              const int np = (int)P.pairs.size() - pair_off;
              const int64_t off = add_block(gint, g.row_U + aoff, j->na[X], g.row_F, np, 1, pair_off, w);
              J3at(X, Y, W) = J3Src{off, 1, np, Y == W ? 1 : 0, Y == W ? j->nb[Y] : j->nb[W], 0, 0};
            }
          }
        }
      } else {
        if ((mask & PSQ_V) && g.nFA > 0 && g.nFB > 0)
          vc_loc[gi] = add_block(gint, g.row_F, g.nFA, g.row_F + g.nFA, g.nFB, 0, 0, w + 3);
        if ((mask & PSQ_J3) && j->na[g.C] > 0 && g.nFA > 0 && g.nFB > 0) {
          const int pair_off = (int)P.pairs.size();
          for (int i = 0; i < g.nFA; ++i)
            for (int jj = 0; jj < g.nFB; ++jj) P.pairs.push_back(make_short2(i, g.nFA + jj));
          const int np = g.nFA * g.nFB;
          const int64_t off = add_block(gint, g.row_U, j->na[g.C], g.row_F, np, 1, pair_off, w);
          J3at(g.C, g.A, g.B) = J3Src{off, 1, np, 0, g.nFB, 0, 0};
        }
      }
    }
    // chunking: enough CTAs for several waves, chunks of at least 2048 points
    int64_t tiles = 0;
    // output tile per block: balanced row tiles of <= 64 rows, then balanced column tiles of
    // <= min(256, 1024 / rows) columns (little padding; no FP64 operation on padding)
    for (auto& b : P.gblocks) {
      const int ntm = (b.m + kFpTileRows - 1) / kFpTileRows;
      b.tile_m = std::max(1, (b.m + ntm - 1) / ntm);
      const int tn_max = std::max(1, std::min(kFpTileCols, kFpTileOut / b.tile_m));
      const int ntn = (b.n + tn_max - 1) / tn_max;
      b.tile_n = std::max(1, (b.n + ntn - 1) / ntn);
      tiles += (int64_t)ntm * ntn;
    }
    const int64_t want = 2LL * kSmCount * P.work_split;
    const int cglob = (int)std::max<int64_t>(1, tiles > 0 ? (want + tiles - 1) / tiles : 1);
    for (size_t bi = 0; bi < P.gblocks.size(); ++bi) {
      GemmBlock& b = P.gblocks[bi];
      const int64_t K = P.grids[b.grid].K;
      // at most kMaxChunkPoints per sequential partial sum (bounded rounding growth), and
      // more chunks where the grid has too few tiles to fill the GPU
      b.n_chunks = (int)std::max<int64_t>((K + kMaxChunkPoints - 1) / kMaxChunkPoints,
                                          std::min<int64_t>(cglob, (K + 2047) / 2048));
      b.n_chunks = std::max(1, b.n_chunks);
      b.part_off = part;
      part += (int64_t)b.n_chunks * b.m * b.n;
      const int tm = (b.m + b.tile_m - 1) / b.tile_m, tn = (b.n + b.tile_n - 1) / b.tile_n;
      for (int c = 0; c < b.n_chunks; ++c)
        for (int x = 0; x < tm; ++x)
          for (int y = 0; y < tn; ++y) P.items.push_back(GemmItem{(int)bi, x, y, c});
    }
    // Largest items first (outputs x points, a formed pair column costing one more product per
    // point): the CTA scheduler hands out blocks in index order, so the last wave holds the
    // small items and the tail of the launch is short.
    auto fp_cost = [&](const GemmItem& it) {
      const GemmBlock& b = P.gblocks[it.block];
      const int64_t K = P.grids[b.grid].K;
      const int64_t csz = (K + b.n_chunks - 1) / b.n_chunks;
      const int64_t pts = std::max<int64_t>(0, std::min<int64_t>(K, (int64_t)it.chunk * csz + csz) - (int64_t)it.chunk * csz);
      const int rows = std::min(b.tile_m, b.m - it.tm * b.tile_m), cols = std::min(b.tile_n, b.n - it.tn * b.tile_n);
      return (double)pts * ((double)rows * cols + rows + (b.b_mode == 1 ? 2.0 : 1.0) * cols);
    };
    std::stable_sort(P.items.begin(), P.items.end(),
                     [&](const GemmItem& x, const GemmItem& y) { return fp_cost(x) > fp_cost(y); });
    P.elem_begin.resize(P.gblocks.size() + 1);
    P.elem_begin[0] = 0;
    for (size_t bi = 0; bi < P.gblocks.size(); ++bi)
      P.elem_begin[bi + 1] = P.elem_begin[bi] + (int64_t)P.gblocks[bi].m * P.gblocks[bi].n;
    for (const GemmBlock& b : P.gblocks) P.issued_flops += 2.0 * b.m * b.n * (double)P.grids[b.grid].K;
    for (int X = 0; X < nat; ++X) {
      for (int Y = 0; Y < nat; ++Y) {
        for (int c = 0; c < 4; ++c) P.src_ptr[c][X * nat + Y] = (int)P.src[c].size();
        if (X > Y || mask == 0) continue;
        const int gb = gidx[grid_for(j, X, Y, X)];
        const DevGrid& G = P.grids[gb];
        // X < Y: the grid of (X, Y) is the pair grid with A = X, B = Y; X == Y: closed forms
        // for S and T (no source), (P|Q) from the one-centre grid's own block
        if (X < Y && (mask & PSQ_S) && s_loc[gb] >= 0)
          P.src[0].push_back(SrcEntry{s_loc[gb], G.nFB, 0, 0, 0, 0, 0, 0, 0, 1.0, 0, 0});
        if (X < Y && (mask & PSQ_T) && t_loc[gb].ab >= 0)
          P.src[1].push_back(SrcEntry{t_loc[gb].ab, G.nFB, 0, 0, 0, 0, 0, 0, 0, 1.0, t_loc[gb].ba, G.nFA});
        if (mask & PSQ_V) {
          for (int C = 0; C < nat; ++C) {
            const GridKey k = grid_for(j, X, Y, C);
            const int gv = gidx[k];
            const DevGrid& H = P.grids[gv];
            const double z = -(double)j->atoms[C].Z;
            if (k.C >= 0) {
              P.src[2].push_back(SrcEntry{vc_loc[gv], H.nFB, 0, 0, 0, 0, 0, 0, 0, z});
            } else {
              // C is A or B of the pair grid; X < Y: (X, Y) = (A, B), the A x B block; X == Y:
              // the X x X block
              const Fp2& v = C == H.A ? va_loc[gv] : vb_loc[gv];
              const int64_t off = X < Y ? v.ab : (X == H.A ? v.aa : v.bb);
              P.src[2].push_back(SrcEntry{off, j->nb[Y], 0, 0, 0, 0, 0, 0, 0, z, 0, 0});
            }
          }
        }
        if (mask & PSQ_J2) {
          const Fp2& b = j2_loc[gb];
          if (X < Y && b.ab >= 0)
            P.src[3].push_back(SrcEntry{b.ab, j->na[Y], 0, 0, 0, 0, 0, 0, 0, 1.0, b.ba, j->na[X]});
          const int64_t own = X == G.A ? b.aa : b.bb;
          if (X == Y && own >= 0) P.src[3].push_back(SrcEntry{own, j->na[X], 0, 0, 0, 0, 0, 0, 0, 1.0, 0, 0});
        }
      }
    }
  } else {
    // Tensor-core path.  Per pair grid: the weighted aux potentials U w form the A panel of
    // the 3-index block (against the pair products chi_i chi_j, formed in the kernel: J3) and
    // of the (P|Q) block (against the aux functions: J2); the weighted operand rows
    // [w lap chi | w chi | w/r_A chi | w/r_B chi] form the A panel of the 2-index block
    // against the basis functions (T, S, V).  Per refined grid: [U_C w | w/r_C] against the
    // A x B pair products (J3 and V).
    struct GridBlocks { int pair = -1, kin = -1, j2 = -1, rowT = -1, rowS = -1, rowVA = -1, rowVB = -1, rowVC = -1; };
    std::vector<GridBlocks> gbk(P.grids.size());
    auto add_panel = [&](int g, int rows_off, int nrows, int tr) {
      const DevGrid& G = P.grids[g];
      Panel pn{};
      pn.grid = g; pn.rows_off = rows_off; pn.nrows = nrows; pn.tr = tr;
      pn.n_tiles = (nrows + tr - 1) / tr;
      pn.nch = (int)((G.K + kChunkPts - 1) / kChunkPts);
      pn.nwin = (int)((G.K + kWinPts - 1) / kWinPts);
      pn.pack_off = P.pack_bytes;
      P.pack_bytes += (int64_t)align_up((size_t)nrows * pn.nch * kSlices * 2 * kChunkPts, 256);
      pn.exp_off = P.pack_bytes;
      P.pack_bytes += (int64_t)align_up((size_t)pn.n_tiles * pn.nwin * tr * 4, 256);
      pn.job_begin = P.n_pack_jobs;
      P.n_pack_jobs += (int64_t)pn.n_tiles * pn.nwin * (tr / kPackRows);  // 16-row groups
      P.panels.push_back(pn);
      return (int)P.panels.size() - 1;
    };
    auto add_mblock = [&](int g, int m, int n, int a_off, int b_off, int a_panel, int b_panel, int ptile_off,
                          int n_btiles) {
      MmaBlock b{};
      b.grid = g; b.m = m; b.n = n; b.a_off = a_off; b.b_off = b_off;
      b.a_panel = a_panel; b.b_panel = b_panel; b.ptile_off = ptile_off; b.n_btiles = n_btiles;
      b.res_off = res;
      res += (int64_t)m * n;
      P.mblocks.push_back(b);
      return (int)P.mblocks.size() - 1;
    };
    // Pair tiles of a 3-index block: the pairs (result column, row x, row y) visited in 8 x 8
    // blocks of (i, j), cut into tiles of <= 64 columns and <= kPairTileRows distinct rows.
    struct PairRef { int col, x, y; };
    auto add_pair_tiles = [&](const std::vector<PairRef>& pl) {
      const int first = (int)P.ptiles.size();
      PairTile t{};
      auto flush = [&]() {
        if (t.ncols > 0) P.ptiles.push_back(t);
        t = PairTile{};
      };
      auto slot = [&](int row) {
        for (int k = 0; k < t.nrows; ++k)
          if (t.rows[k] == row) return k;
        return -1;
      };
      for (const PairRef& pr : pl) {
        const int need = (slot(pr.x) < 0) + (pr.y != pr.x && slot(pr.y) < 0);
        if (t.ncols == kMmaN || t.nrows + need > kPairTileRows) flush();
        int sx = slot(pr.x);
        if (sx < 0) { sx = t.nrows; t.rows[t.nrows++] = (short)pr.x; }
        int sy = slot(pr.y);
        if (sy < 0) { sy = t.nrows; t.rows[t.nrows++] = (short)pr.y; }
        t.dx[t.ncols] = (unsigned char)sx;
        t.dy[t.ncols] = (unsigned char)sy;
        t.col[t.ncols] = pr.col;
        ++t.ncols;
      }
      flush();
      return std::make_pair(first, (int)P.ptiles.size() - first);
    };
    for (size_t gi = 0; gi < P.grids.size(); ++gi) {
      const DevGrid& g = P.grids[gi];
      const int nl = g.nFA + g.nFB, W = g.row_W;
      GridBlocks& gb = gbk[gi];
      if (g.C < 0) {
        const bool j3 = (mask & PSQ_J3) && g.nG > 0 && nl > 0;
        const bool j2 = (mask & PSQ_J2) && g.nG > 0;
        // the weighted potentials of the aux functions: one panel per atom (A tiles of one
        // atom's rows, so that whole tiles of unused elements can be left out) when that takes
        // no more 128-row tiles than one panel of both atoms' rows, else one panel
        const int naA = j->na[g.A], naB = j->na[g.B];
        auto ntiles = [](int r) { return (r + kMmaM - 1) / kMmaM; };
        const bool split = naA > 0 && naB > 0 && ntiles(naA) + ntiles(naB) == ntiles(g.nG);
        int pu[2] = {-1, -1}, u_off = -1;
        if (j3 || j2) {
          u_off = (int)P.pairs.size();
          for (int q = 0; q < g.nG; ++q) P.pairs.push_back(make_short2(g.row_U + q, W));
          if (split) {
            pu[0] = add_panel((int)gi, u_off, naA, kMmaM);
            pu[1] = add_panel((int)gi, u_off + naA, naB, kMmaM);
          } else {
            pu[0] = add_panel((int)gi, u_off, g.nG, kMmaM);
          }
        }
        if (j3) {
          // all local pairs i <= j, result columns in packed row-major order
          const int b_off = (int)P.pairs.size();
          for (int i = 0; i < nl; ++i)
            for (int jj = i; jj < nl; ++jj) P.pairs.push_back(make_short2(g.row_F + i, g.row_F + jj));
          // pair tiles per class (A,A), (A,B), (B,B), in that order, each in 6 x 8 blocks of
          // (i, j): 48 columns from at most 14 distinct rows
          const int nA = g.nFA;
          auto col_of = [&](int i, int jj) { return i * nl - i * (i - 1) / 2 + (jj - i); };
          std::vector<PairRef> pl;
          auto tiles = [&](int i0, int i1, int j0, int j1, bool upper) {
            pl.clear();
            for (int ib = i0; ib < i1; ib += 6)
              for (int jb = upper ? j0 + (ib - i0) / 8 * 8 : j0; jb < j1; jb += 8)
                for (int i = ib; i < std::min(i1, ib + 6); ++i)
                  for (int jj = upper ? std::max(i, jb) : jb; jj < std::min(j1, jb + 8); ++jj)
                    pl.push_back(PairRef{col_of(i, jj), g.row_F + i, g.row_F + jj});
            return add_pair_tiles(pl);
          };
          // (without the split: one class of all pairs, fewer partial tiles)
          const auto tAA = split ? tiles(0, nA, 0, nA, true) : tiles(0, nl, 0, nl, true);
          const auto tAB = split ? tiles(0, nA, nA, nl, false) : std::make_pair(tAA.first + tAA.second, 0);
          const auto tBB = split ? tiles(nA, nl, nA, nl, true) : std::make_pair(tAB.first, 0);
          // an atom's rows need the one-centre pairs (its own functions) only where this grid
          // is its one-centre grid; the other classes are two-centre terms of this pair
          auto here = [&](int Y, int Wt, int X) {
            const GridKey k = grid_for(j, Y, Wt, X);
            return k.A == g.A && k.B == g.B && k.C < 0;
          };
          const int end_all = tBB.first + tBB.second;
          if (split) {
            // rows of A: (A,A) if here, then (A,B), (B,B); rows of B: (A,A), (A,B), then (B,B)
            // if here; the two blocks' results are consecutive (rows of A, then rows of B)
            const int t0 = here(g.A, g.A, g.A) ? tAA.first : tAB.first;
            gb.pair = add_mblock((int)gi, naA, nl * (nl + 1) / 2, u_off, b_off, pu[0], -1, t0, end_all - t0);
            const int t1 = here(g.B, g.B, g.B) ? end_all : tAB.first + tAB.second;
            add_mblock((int)gi, naB, nl * (nl + 1) / 2, u_off + naA, b_off, pu[1], -1, tAA.first, t1 - tAA.first);
          } else {
            gb.pair = add_mblock((int)gi, g.nG, nl * (nl + 1) / 2, u_off, b_off, pu[0], -1, tAA.first,
                                 end_all - tAA.first);
          }
        }
        if ((mask & (PSQ_S | PSQ_T | PSQ_V)) && nl > 0) {
          // 2-index block: [w lap chi | w chi | w/r_A chi | w/r_B chi] against chi
          const int a_off = (int)P.pairs.size();
          if (mask & PSQ_T) {
            gb.rowT = 0;
            for (int i = 0; i < nl; ++i) P.pairs.push_back(make_short2(g.row_L + i, W));
          }
          if (mask & PSQ_S) {
            gb.rowS = (int)P.pairs.size() - a_off;
            for (int i = 0; i < nl; ++i) P.pairs.push_back(make_short2(g.row_F + i, W));
          }
          if (mask & PSQ_V) {
            gb.rowVA = (int)P.pairs.size() - a_off;
            for (int i = 0; i < nl; ++i) P.pairs.push_back(make_short2(g.row_F + i, W + 1));
            gb.rowVB = (int)P.pairs.size() - a_off;
            for (int i = 0; i < nl; ++i) P.pairs.push_back(make_short2(g.row_F + i, W + 2));
          }
          const int na_rows = (int)P.pairs.size() - a_off;
          const int pk = add_panel((int)gi, a_off, na_rows, kMmaM);
          const int b_off = (int)P.pairs.size();
          for (int i = 0; i < nl; ++i) P.pairs.push_back(make_short2(g.row_F + i, -1));
          const int pf = add_panel((int)gi, b_off, nl, kMmaN);
          gb.kin = add_mblock((int)gi, na_rows, nl, a_off, b_off, pk, pf, -1, 0);
        }
        if (j2) {
          const int b_off = (int)P.pairs.size();
          for (int q = 0; q < g.nG; ++q) P.pairs.push_back(make_short2(g.row_G + q, -1));
          const int pg = add_panel((int)gi, b_off, g.nG, kMmaN);
          if (split) {  // rows of A, then rows of B (consecutive results, as one nG x nG block)
            gb.j2 = add_mblock((int)gi, naA, g.nG, u_off, b_off, pu[0], pg, -1, 0);
            add_mblock((int)gi, naB, g.nG, u_off + naA, b_off, pu[1], pg, -1, 0);
          } else {
            gb.j2 = add_mblock((int)gi, g.nG, g.nG, u_off, b_off, pu[0], pg, -1, 0);
          }
        }
      } else if (g.nFA > 0 && g.nFB > 0) {
        const bool j3 = (mask & PSQ_J3) && g.nG > 0;
        if (j3 || (mask & PSQ_V)) {
          const int a_off = (int)P.pairs.size();
          if (j3)
            for (int q = 0; q < g.nG; ++q) P.pairs.push_back(make_short2(g.row_U + q, W));
          if (mask & PSQ_V) { gb.rowVC = (int)P.pairs.size() - a_off; P.pairs.push_back(make_short2(W + 3, -1)); }
          const int na_rows = (int)P.pairs.size() - a_off;
          const int pc = add_panel((int)gi, a_off, na_rows, kMmaM);
          const int b_off = (int)P.pairs.size();
          for (int i = 0; i < g.nFA; ++i)
            for (int jj = 0; jj < g.nFB; ++jj) P.pairs.push_back(make_short2(g.row_F + i, g.row_F + g.nFA + jj));
          std::vector<PairRef> pl;
          for (int ib = 0; ib < g.nFA; ib += 6)
            for (int jb = 0; jb < g.nFB; jb += 8)
              for (int i = ib; i < std::min(g.nFA, ib + 6); ++i)
                for (int jj = jb; jj < std::min(g.nFB, jb + 8); ++jj)
                  pl.push_back(PairRef{i * g.nFB + jj, g.row_F + i, g.row_F + g.nFA + jj});
          const auto tl = add_pair_tiles(pl);
          gb.pair = add_mblock((int)gi, na_rows, g.nFA * g.nFB, a_off, b_off, pc, -1, tl.first, tl.second);
        }
      }
    }
    // assembly sources
    auto blk = [&](int b) -> const MmaBlock& { return P.mblocks[b]; };
    for (int X = 0; X < nat; ++X) {
      for (int Y = 0; Y < nat; ++Y) {
        for (int c = 0; c < 4; ++c) P.src_ptr[c][X * nat + Y] = (int)P.src[c].size();
        if (X > Y || mask == 0) continue;
        const int gi = gidx[grid_for(j, X, Y, X)];
        const DevGrid& G = P.grids[gi];
        const GridBlocks& gb = gbk[gi];
        const int oX = local_off(G, X), oY = local_off(G, Y);
        if ((mask & PSQ_S) && gb.kin >= 0) {
          const MmaBlock& k = blk(gb.kin);
          P.src[0].push_back(SrcEntry{k.res_off, k.n, gb.rowS + oX, oY, gb.rowS + oY, oX, 0, 0, 0, 1.0});
        }
        if ((mask & PSQ_T) && gb.kin >= 0) {
          const MmaBlock& k = blk(gb.kin);
          P.src[1].push_back(SrcEntry{k.res_off, k.n, gb.rowT + oX, oY, gb.rowT + oY, oX, 0, 0, 0, 1.0});
        }
        if (mask & PSQ_V) {
          for (int C = 0; C < nat; ++C) {
            const GridKey k = grid_for(j, X, Y, C);
            const int hv = gidx[k];
            const DevGrid& H = P.grids[hv];
            const GridBlocks& hb = gbk[hv];
            const double z = -(double)j->atoms[C].Z;
            if (k.C >= 0) {
              if (hb.pair < 0) continue;
              const MmaBlock& pb = blk(hb.pair);
              P.src[2].push_back(SrcEntry{pb.res_off, 1, 0, 0, 0, hb.rowVC, 2, H.nFB, pb.n, z});
            } else {
              if (hb.kin < 0) continue;
              const MmaBlock& kb = blk(hb.kin);
              const int row = C == H.A ? hb.rowVA : hb.rowVB;
              const int hX = local_off(H, X), hY = local_off(H, Y);
              P.src[2].push_back(SrcEntry{kb.res_off, kb.n, row + hX, hY, row + hY, hX, 0, 0, 0, z});
            }
          }
        }
        if ((mask & PSQ_J2) && gb.j2 >= 0) {
          const int aX = aux_off(G, X), aY = aux_off(G, Y);
          P.src[3].push_back(SrcEntry{blk(gb.j2).res_off, G.nG, aX, aY, aY, aX, 0, 0, 0, 1.0});
        }
      }
    }
    if (mask & PSQ_J3) {
      for (int X = 0; X < nat; ++X)
        for (int Y = 0; Y < nat; ++Y)
          for (int W = Y; W < nat; ++W) {
            if (j->na[X] == 0 || j->nb[Y] == 0 || j->nb[W] == 0) continue;
            const GridKey k = grid_for(j, Y, W, X);
            const int gi = gidx[k];
            const DevGrid& G = P.grids[gi];
            const GridBlocks& gb = gbk[gi];
            if (gb.pair < 0) continue;
            const MmaBlock& b = blk(gb.pair);
            if (k.C >= 0)
              J3at(X, Y, W) = J3Src{b.res_off, 1, b.n, 0, G.nFB, 0, 0};
            else
              J3at(X, Y, W) = J3Src{b.res_off + (int64_t)aux_off(G, X) * b.n, 1, b.n, 1, G.nFA + G.nFB,
                                    local_off(G, Y), local_off(G, W)};
          }
    }
    // Waves: consecutive grids while their operand rows (hi and lo planes) and packed panels
    // fit the budget (a wave holds at least one grid).  Offsets of grids, panels and blocks
    // are then made relative to the wave; the regions are sized by the largest wave.
    const int nG = (int)P.grids.size();
    std::vector<int64_t> g_ops(nG, 0), g_bytes(nG, 0);
    for (int gi = 0; gi < nG; ++gi) {
      const int64_t end = gi + 1 < nG ? P.grids[gi + 1].op_off : ops;
      g_ops[gi] = end - P.grids[gi].op_off;
      g_bytes[gi] = 2 * (int64_t)sizeof(float) * g_ops[gi];
    }
    auto panel_bytes = [&](const Panel& pn, int64_t* pack, int64_t* expb) {
      *pack = (int64_t)align_up((size_t)pn.nrows * pn.nch * kSlices * 2 * kChunkPts, 256);
      *expb = (int64_t)align_up((size_t)pn.n_tiles * pn.nwin * pn.tr * 4, 256);
    };
    for (const Panel& pn : P.panels) {
      int64_t pk, ex;
      panel_bytes(pn, &pk, &ex);
      g_bytes[pn.grid] += pk + ex;
    }
    const int64_t budget = (int64_t)(j->wave_bytes ? j->wave_bytes : kDefaultWaveBytes);
    for (int g0 = 0; g0 < nG;) {
      int g1 = g0;
      int64_t acc = 0;
      while (g1 < nG && (g1 == g0 || acc + g_bytes[g1] <= budget)) acc += g_bytes[g1++];
      Plan::Wave wv{};
      wv.g0 = g0;
      wv.g1 = g1;
      P.waves.push_back(wv);
      g0 = g1;
    }
    int64_t ops_max = 0, pack_max = 0, part_max = 0;
    size_t pn_i = 0, mb_i = 0;
    const double kSliceProducts = kSlices * (kSlices + 1) / 2;
    constexpr int64_t kCpw = kWinPts / kChunkPts;  // chunks per window
    auto item_chunks = [&](const GemmItem& it) {
      const MmaBlock& mb = P.mblocks[it.block];
      const int64_t nch = (P.grids[mb.grid].K + kChunkPts - 1) / kChunkPts;
      const int64_t c0 = kCpw * it.chunk * mb.win_per;
      return std::max<int64_t>(0, std::min<int64_t>(nch, c0 + kCpw * mb.win_per) - c0);
    };
    // Items by estimated cost (chunks; a formed pair tile's window counts twice: its
    // producers' slicing), largest first, each given to the persistent CTA with the least
    // cost so far (LPT); a CTA takes its items largest first.
    auto item_cost = [&](const GemmItem& it) {
      return (double)item_chunks(it) * (P.mblocks[it.block].b_panel < 0 ? 2.0 : 1.0);
    };
    P.cta_begin.clear();
    P.pack_hint.clear();
    for (Plan::Wave& wv : P.waves) {
      // operand rows of the wave's grids from 0
      int64_t o = 0;
      for (int gi = wv.g0; gi < wv.g1; ++gi) {
        P.grids[gi].op_off = o;
        o += g_ops[gi];
      }
      ops_max = std::max(ops_max, o);
      // its panels (consecutive, in grid order) packed from 0, packing jobs counted from 0
      wv.pn0 = (int)pn_i;
      int64_t pb = 0, jobs = 0;
      while (pn_i < P.panels.size() && P.panels[pn_i].grid < wv.g1) {
        Panel& pn = P.panels[pn_i++];
        int64_t pk, ex;
        panel_bytes(pn, &pk, &ex);
        pn.pack_off = pb;
        pn.exp_off = pb + pk;
        pb += pk + ex;
        pn.job_begin = jobs;
        jobs += (int64_t)pn.n_tiles * pn.nwin * (pn.tr / kPackRows);  // 16-row groups
      }
      wv.pn1 = (int)pn_i;
      wv.jobs = jobs;
      wv.ph_off = (int64_t)P.pack_hint.size();
      for (int64_t jb = 0, k = wv.pn0; jb < jobs; jb += kPackHintJobs) {
        while (k + 1 < wv.pn1 && P.panels[k + 1].job_begin <= jb) ++k;
        P.pack_hint.push_back((int)(k - wv.pn0));
      }
      pack_max = std::max(pack_max, pb);
      // its blocks: tiles (128 rows x 48 columns) x window ranges, work_split items per SM
      // (a static LPT deal then ends within a few percent of the mean), ranges of >= 4 windows
      wv.mb0 = (int)mb_i;
      while (mb_i < P.mblocks.size() && P.mblocks[mb_i].grid < wv.g1) ++mb_i;
      wv.mb1 = (int)mb_i;
      int64_t mtiles = 0;
      for (int bi = wv.mb0; bi < wv.mb1; ++bi) {
        const MmaBlock& mb = P.mblocks[bi];
        mtiles += (int64_t)((mb.m + kMmaM - 1) / kMmaM) * (mb.b_panel >= 0 ? (mb.n + kMmaN - 1) / kMmaN : mb.n_btiles);
      }
      const int64_t want = (int64_t)P.work_split * kSmCount;
      const int cr = (int)std::max<int64_t>(1, mtiles > 0 ? (want + mtiles - 1) / mtiles : 1);
      std::vector<GemmItem> items;
      int64_t pt = 0;
      for (int bi = wv.mb0; bi < wv.mb1; ++bi) {
        MmaBlock& mb = P.mblocks[bi];
        const int64_t nwin = (P.grids[mb.grid].K + kWinPts - 1) / kWinPts;
        const int64_t r0 = std::max<int64_t>(1, std::min<int64_t>(cr, (nwin + 3) / 4));
        mb.win_per = (int)((nwin + r0 - 1) / r0);
        mb.n_ranges = (int)((nwin + mb.win_per - 1) / mb.win_per);
        mb.part_off = pt;
        pt += (int64_t)mb.n_ranges * mb.m * mb.n;
        const int tm = (mb.m + kMmaM - 1) / kMmaM, tn = mb.b_panel >= 0 ? (mb.n + kMmaN - 1) / kMmaN : mb.n_btiles;
        for (int c = 0; c < mb.n_ranges; ++c)
          for (int x = 0; x < tm; ++x)
            for (int y = 0; y < tn; ++y) items.push_back(GemmItem{bi, x, y, c});
      }
      part_max = std::max(part_max, pt);
      // Gangs: the items of one (block, A tile, window range) read the same packed A chunks,
      // one item per B tile.  A gang's items go to different CTAs at the same depth of their
      // queues, so that they run at about the same time and the A chunks come from L2 after
      // the first read (a refined grid's A panel exceeds the L2).  Gangs by cost, largest
      // first; each item of a gang to the CTA with the least cost so far (LPT over gangs).
      std::stable_sort(items.begin(), items.end(), [&](const GemmItem& x, const GemmItem& y) {
        if (x.block != y.block) return x.block < y.block;
        if (x.tm != y.tm) return x.tm < y.tm;
        if (x.chunk != y.chunk) return x.chunk < y.chunk;
        return x.tn < y.tn;
      });
      std::vector<std::pair<size_t, size_t>> gangs;  // [begin, end) in items
      for (size_t i = 0; i < items.size();) {
        size_t k = i + 1;
        while (k < items.size() && items[k].block == items[i].block && items[k].tm == items[i].tm &&
               items[k].chunk == items[i].chunk)
          ++k;
        gangs.push_back({i, k});
        i = k;
      }
      auto gang_cost = [&](const std::pair<size_t, size_t>& g) {
        double c = 0;
        for (size_t i = g.first; i < g.second; ++i) c += item_cost(items[i]);
        return c;
      };
      std::stable_sort(gangs.begin(), gangs.end(), [&](const std::pair<size_t, size_t>& x,
                                                        const std::pair<size_t, size_t>& y) {
        return gang_cost(x) > gang_cost(y);
      });
      wv.n_ctas = (int)std::min<int64_t>((int64_t)items.size(), j->ctx->sm_count);
      std::vector<std::vector<GemmItem>> per(wv.n_ctas);
      std::vector<std::pair<double, int>> heap;  // (cost so far, CTA), min-heap
      for (int b = 0; b < wv.n_ctas; ++b) heap.push_back({0.0, b});
      auto cmp = [](const std::pair<double, int>& x, const std::pair<double, int>& y) { return x > y; };
      std::make_heap(heap.begin(), heap.end(), cmp);
      std::vector<std::pair<double, int>> taken;
      for (const auto& g : gangs) {
        // the gang's items to the least loaded CTAs, one each (a gang larger than the CTA
        // count wraps around)
        for (size_t i = g.first; i < g.second;) {
          taken.clear();
          for (; i < g.second && !heap.empty(); ++i) {
            std::pop_heap(heap.begin(), heap.end(), cmp);
            auto slot = heap.back();
            heap.pop_back();
            per[slot.second].push_back(items[i]);
            slot.first += item_cost(items[i]);
            taken.push_back(slot);
          }
          for (const auto& t : taken) {
            heap.push_back(t);
            std::push_heap(heap.begin(), heap.end(), cmp);
          }
        }
      }
      wv.cb_off = (int)P.cta_begin.size();
      P.cta_begin.push_back((int)P.mitems.size());
      for (auto& v : per) {
        P.mitems.insert(P.mitems.end(), v.begin(), v.end());
        P.cta_begin.push_back((int)P.mitems.size());
      }
      // issued tensor work: per 32-point chunk of an item, the slice products of orders 0..4
      // (15 of 128 x 48 x 32, issued per 16-point K step as five MMAs of N = 240 .. 48)
      for (const GemmItem& it : items)
        P.issued_flops += (double)item_chunks(it) * kSliceProducts * 2.0 * kMmaM * kMmaN * kChunkPts;
    }
    P.n_ctas = 0;
    for (const Plan::Wave& wv : P.waves) P.n_ctas = std::max(P.n_ctas, wv.n_ctas);
    ops = ops_max;
    P.pack_bytes = pack_max;
    part = part_max;
    P.elem_begin.resize(P.mblocks.size() + 1);
    P.elem_begin[0] = 0;
    for (size_t bi = 0; bi < P.mblocks.size(); ++bi)
      P.elem_begin[bi + 1] = P.elem_begin[bi] + (int64_t)P.mblocks[bi].m * P.mblocks[bi].n;
  }
  for (int c = 0; c < 4; ++c) P.src_ptr[c][nat * nat] = (int)P.src[c].size();
  if (P.mixed) {
    // FP32-pair rotation, x-scales of the shells and FP64 row constants
    auto split = [](double v) {
      const float hi = (float)v;
      return make_float2(hi, (float)(v - (double)hi));
    };
    for (auto& g : P.grids) {
      for (int i = 0; i < 9; ++i) {
        g.Rh[i] = (float)g.R[i];
        g.Rl[i] = (float)(g.R[i] - (double)g.Rh[i]);
      }
      g.xi_off = (int)P.xi.size();
      auto add_xi = [&](const std::vector<DevShell>& sh, int s0, int s1, bool focus) {
        for (int q = s0; q < s1; ++q) P.xi.push_back(split(focus ? 2.0 * g.a * sh[q].zeta : sh[q].zeta));
      };
      add_xi(j->dbs, g.shb_A0, g.shb_A1, true);
      add_xi(j->dbs, g.shb_B0, g.shb_B1, true);
      if (g.aux_c0 >= 0) add_xi(j->das, g.sha_0, g.sha_1, g.aux_c0 == g.A || g.aux_c0 == g.B);
      if (g.aux_c1 >= 0) add_xi(j->das, g.sha_2, g.sha_3, g.aux_c1 == g.A || g.aux_c1 == g.B);
      g.rc_off = (int)P.rowc.size();
      int nrows = g.row_W + 4;
      P.rowc.resize(P.rowc.size() + nrows, 1.0);
      double* rc = P.rowc.data() + g.rc_off;
      auto put_rows = [&](int row0, int kind) {
        std::vector<double> v;
        row_constants(j, g, kind, v);
        for (size_t r = 0; r < v.size(); ++r) rc[row0 + r] = v[r];
      };
      if (g.row_F >= 0) put_rows(g.row_F, 0);
      if (g.row_L >= 0) put_rows(g.row_L, 1);
      if (g.row_G >= 0) put_rows(g.row_G, 2);
      if (g.row_U >= 0) put_rows(g.row_U, 3);
      rc[g.row_W + 0] = g.a * g.a * g.a;
      rc[g.row_W + 1] = 0.5 * g.a * g.a;
      rc[g.row_W + 2] = 0.5 * g.a * g.a;
      rc[g.row_W + 3] = g.a * g.a * g.a;
    }
    // node tables
    for (auto& g : P.grids) {
      g.nt_off = (int)P.n_nodes;
      const int n = (g.n_mu + g.nt_mu * g.n_sp) * g.q_mu + (g.n_nu + g.nt_nu * g.n_sp) * g.q_nu +
                    (g.n_phi + g.nt_phi * g.n_sp) * g.q_phi;
      P.n_nodes += n;
      P.max_node_entries = std::max(P.max_node_entries, n);
    }
  }
  for (size_t gi = 0; gi < P.grids.size(); ++gi)
    for (int64_t p0 = 0; p0 < P.grids[gi].K; p0 += kPointsPerBlock) P.pblocks.push_back(PointBlock{(int)gi, 0, p0});
  for (Plan::Wave& wv : P.waves) {
    wv.pb0 = wv.pb1 = (int)P.pblocks.size();
    for (int k = 0; k < (int)P.pblocks.size(); ++k) {
      if (P.pblocks[k].grid >= wv.g0 && wv.pb0 == (int)P.pblocks.size()) wv.pb0 = k;
      if (P.pblocks[k].grid >= wv.g1) { wv.pb1 = k; break; }
    }
  }
  // useful contractions: for every molecule-matrix block, rows x cols x the live points of
  // the one grid that integrates it (same-atom blocks count i <= j once)
  P.contractions = 0;
  auto live = [&](GridKey k) {
    const DevGrid& g = P.grids[gidx[k]];
    return (double)(g.K - (int64_t)g.n_touch * g.q_mu * g.q_nu * g.q_phi);
  };
  if (mask) {
    for (int A = 0; A < nat; ++A)
      for (int B = A; B < nat; ++B) {
        const double nab = A != B ? (double)j->nb[A] * j->nb[B] : 0.5 * j->nb[A] * (j->nb[A] + 1.0);
        if (mask & PSQ_S) P.contractions += nab * live(grid_for(j, A, B, A));
        if (mask & PSQ_T) P.contractions += nab * live(grid_for(j, A, B, A));
        for (int C = 0; C < nat; ++C) {
          if (mask & PSQ_V) P.contractions += nab * live(grid_for(j, A, B, C));
          if (mask & PSQ_J3) P.contractions += j->na[C] * nab * live(grid_for(j, A, B, C));
        }
        if (mask & PSQ_J2) {
          const double ncd = A != B ? (double)j->na[A] * j->na[B] : 0.5 * j->na[A] * (j->na[A] + 1.0);
          P.contractions += ncd * live(grid_for(j, A, B, A));
        }
      }
  }
  int nclasses = 0;
  for (int c = 0; c < 5; ++c) nclasses += (mask >> c) & 1;
  P.launches = P.grids.empty() ? 0 : (P.mixed ? 1 + 4 * (int)P.waves.size() : 3) + nclasses;
  // table layout
  size_t off = 0;
  auto sec = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  P.o_grids = sec(sizeof(DevGrid) * P.grids.size());
  P.o_edges = sec(sizeof(double) * P.edges.size());
  P.o_bsh = sec(sizeof(DevShell) * j->dbs.size());
  P.o_ash = sec(sizeof(DevShell) * j->das.size());
  P.o_xyz = sec(sizeof(double) * 3 * nat);
  P.o_pb = sec(sizeof(PointBlock) * P.pblocks.size());
  P.o_gb = sec(sizeof(GemmBlock) * P.gblocks.size());
  P.o_it = sec(sizeof(GemmItem) * P.items.size());
  P.o_pairs = sec(sizeof(short2) * P.pairs.size());
  P.o_eb = sec(sizeof(int64_t) * P.elem_begin.size());
  P.o_fa = sec(sizeof(int) * j->fn_atom.size());
  P.o_fl = sec(sizeof(int) * j->fn_local.size());
  P.o_fs = sec(sizeof(int) * j->fn_shell.size());
  P.o_aa = sec(sizeof(int) * j->aux_atom.size());
  P.o_al = sec(sizeof(int) * j->aux_local.size());
  for (int c = 0; c < 4; ++c) {
    P.o_src[c] = sec(sizeof(SrcEntry) * P.src[c].size());
    P.o_ptr[c] = sec(sizeof(int) * P.src_ptr[c].size());
  }
  P.o_j3 = sec(sizeof(J3Src) * P.j3.size());
  P.o_mb = sec(sizeof(MmaBlock) * P.mblocks.size());
  P.o_mi = sec(sizeof(GemmItem) * P.mitems.size());
  P.o_cb = sec(sizeof(int) * P.cta_begin.size());
  P.o_pn = sec(sizeof(Panel) * P.panels.size());
  P.o_ph = sec(sizeof(int) * P.pack_hint.size());
  P.o_pt = sec(sizeof(PairTile) * P.ptiles.size());
  P.o_status = sec(sizeof(int) * 4);
  P.o_xi = sec(sizeof(float2) * P.xi.size());
  P.o_rc = sec(sizeof(double) * P.rowc.size());
  P.table_bytes = off;
  P.nodes_off = off;
  off = align_up(off + sizeof(NodeEntry) * (size_t)P.n_nodes, 256);
  P.ops_off = off;
  P.n_ops = ops;
  off = align_up(off + esize * (size_t)ops * (P.mixed ? 2 : 1), 256);
  P.pack_off = off;
  off = align_up(off + (size_t)P.pack_bytes, 256);
  P.part_off = off;
  off = align_up(off + sizeof(double) * (size_t)part, 256);
  P.res_off = off;
  off = align_up(off + sizeof(double) * (size_t)res, 256);
  P.ws_bytes = off;
  // staging copy of the tables (page-locked when the context has a device)
  P.pinned = j->ctx->device >= 0;
  if (P.pinned) {
    if (cudaMallocHost((void**)&P.staging, std::max<size_t>(P.table_bytes, 256)) != cudaSuccess) {
      P.staging = nullptr;
      return fail(PSQ_ERR_OOM, "cudaMallocHost of %zu bytes failed", P.table_bytes);
    }
  } else {
    P.staging = (double*)std::malloc(std::max<size_t>(P.table_bytes, 256));
    if (!P.staging) return fail(PSQ_ERR_OOM, "malloc of %zu bytes failed", P.table_bytes);
  }
  char* s = (char*)P.staging;
  std::memset(s, 0, P.table_bytes);
  auto put = [&](size_t o, const void* src, size_t bytes) {
    if (bytes) std::memcpy(s + o, src, bytes);
  };
  put(P.o_grids, P.grids.data(), sizeof(DevGrid) * P.grids.size());
  put(P.o_edges, P.edges.data(), sizeof(double) * P.edges.size());
  put(P.o_bsh, j->dbs.data(), sizeof(DevShell) * j->dbs.size());
  put(P.o_ash, j->das.data(), sizeof(DevShell) * j->das.size());
  std::vector<double> xyz(3 * nat);
  for (int X = 0; X < nat; ++X)
    for (int c = 0; c < 3; ++c) xyz[3 * X + c] = j->atoms[X].xyz[c];
  put(P.o_xyz, xyz.data(), sizeof(double) * xyz.size());
  put(P.o_pb, P.pblocks.data(), sizeof(PointBlock) * P.pblocks.size());
  put(P.o_gb, P.gblocks.data(), sizeof(GemmBlock) * P.gblocks.size());
  put(P.o_it, P.items.data(), sizeof(GemmItem) * P.items.size());
  put(P.o_pairs, P.pairs.data(), sizeof(short2) * P.pairs.size());
  put(P.o_eb, P.elem_begin.data(), sizeof(int64_t) * P.elem_begin.size());
  put(P.o_fa, j->fn_atom.data(), sizeof(int) * j->fn_atom.size());
  put(P.o_fl, j->fn_local.data(), sizeof(int) * j->fn_local.size());
  put(P.o_fs, j->fn_shell.data(), sizeof(int) * j->fn_shell.size());
  put(P.o_aa, j->aux_atom.data(), sizeof(int) * j->aux_atom.size());
  put(P.o_al, j->aux_local.data(), sizeof(int) * j->aux_local.size());
  for (int c = 0; c < 4; ++c) {
    put(P.o_src[c], P.src[c].data(), sizeof(SrcEntry) * P.src[c].size());
    put(P.o_ptr[c], P.src_ptr[c].data(), sizeof(int) * P.src_ptr[c].size());
  }
  put(P.o_j3, P.j3.data(), sizeof(J3Src) * P.j3.size());
  put(P.o_mb, P.mblocks.data(), sizeof(MmaBlock) * P.mblocks.size());
  put(P.o_mi, P.mitems.data(), sizeof(GemmItem) * P.mitems.size());
  put(P.o_cb, P.cta_begin.data(), sizeof(int) * P.cta_begin.size());
  put(P.o_pn, P.panels.data(), sizeof(Panel) * P.panels.size());
  put(P.o_ph, P.pack_hint.data(), sizeof(int) * P.pack_hint.size());
  put(P.o_pt, P.ptiles.data(), sizeof(PairTile) * P.ptiles.size());
  put(P.o_xi, P.xi.data(), sizeof(float2) * P.xi.size());
  put(P.o_rc, P.rowc.data(), sizeof(double) * P.rowc.size());
  return PSQ_OK;
}

// The job's plan for mask (made on first use), shared with the caller so that a concurrent
// psq_job_autotune replacing it cannot free it under a running compute.
psq_status get_plan_shared(psq_job* j, unsigned mask, std::shared_ptr<Plan>* out) {
  std::lock_guard<std::mutex> lk(j->mu);
  auto it = j->plans.find(mask);
  if (it != j->plans.end()) {
    *out = it->second;
    return PSQ_OK;
  }
  std::shared_ptr<Plan> p(new (std::nothrow) Plan());
  if (!p) return fail(PSQ_ERR_OOM, "plan allocation failed");
  auto ws = j->work_split.find(mask);
  if (ws != j->work_split.end()) p->work_split = ws->second;
  else p->work_split = j->prec == PSQ_MIXED ? 16 : 8;
  psq_status st = make_plan(j, mask, *p);
  if (st != PSQ_OK) return st;
  *out = p;
  j->plans[mask] = std::move(p);
  return PSQ_OK;
}

// The same for queries that only read the plan's sizes while the caller holds the job.
psq_status get_plan(psq_job* j, unsigned mask, Plan** out) {
  std::shared_ptr<Plan> sp;
  psq_status st = get_plan_shared(j, mask, &sp);
  if (st == PSQ_OK) *out = sp.get();
  return st;
}

// Records a timing event before a launch of `kind` (kind -1 closes a psq_compute call).
cudaError_t mark(psq_job* j, int kind, cudaStream_t s) {
  if (!j->prof_on || j->capturing || j->prof.size() >= (1u << 20)) return cudaSuccess;
  cudaEvent_t e;
  if (!j->ev_free.empty()) {
    e = j->ev_free.back();
    j->ev_free.pop_back();
  } else {
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
  }
  j->prof.push_back({kind, e});
  return cudaEventRecord(e, s);
}

LaunchTables tables_at(const Plan& P, char* ws) {
  LaunchTables t{};
  t.grids = (const DevGrid*)(ws + P.o_grids);
  t.edges = (const double*)(ws + P.o_edges);
  t.bshell = (const DevShell*)(ws + P.o_bsh);
  t.ashell = (const DevShell*)(ws + P.o_ash);
  t.atom_xyz = (const double*)(ws + P.o_xyz);
  t.pblocks = (const PointBlock*)(ws + P.o_pb);
  t.n_pblocks = (int)P.pblocks.size();
  t.gblocks = (const GemmBlock*)(ws + P.o_gb);
  t.n_gblocks = (int)P.gblocks.size();
  t.items = (const GemmItem*)(ws + P.o_it);
  t.n_items = (int)P.items.size();
  t.pairs = (const short2*)(ws + P.o_pairs);
  t.elem_begin = (const int64_t*)(ws + P.o_eb);
  t.n_elems = P.elem_begin.empty() ? 0 : P.elem_begin.back();
  return t;
}

}  // namespace

// ------------------------------------------------------------------------------ C ABI

extern "C" {

const char* psq_last_error(void) { return g_err.c_str(); }

psq_status psq_context_create(int device, psq_context** out) {
  if (!out) return fail(PSQ_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (device == -1) {  // planning only: jobs can be created and queried, not computed
    psq_context* c = new (std::nothrow) psq_context{-1};
    if (!c) return fail(PSQ_ERR_OOM, "context allocation failed");
    *out = c;
    return PSQ_OK;
  }
  int n = 0;
  CUDA_TRY(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(PSQ_ERR_ARG, "device %d of %d", device, n);
  CUDA_TRY(cudaSetDevice(device));
  double x[(kMaxQ + 1) * kMaxQ] = {0}, w[(kMaxQ + 1) * kMaxQ] = {0};
  for (int q = 1; q <= kMaxQ; ++q) gauss_legendre(q, x + q * kMaxQ, w + q * kMaxQ);
  double klm[(kMaxL + 1) * (kMaxL + 1)];
  for (int l = 0; l <= kMaxL; ++l)
    for (int m = -l; m <= l; ++m) {
      const int am = std::abs(m);
      double k = std::sqrt((2 * l + 1) / (4 * M_PI) * factorial(l - am) / factorial(l + am));
      if (m != 0) k *= std::sqrt(2.0);
      klm[l * l + l + m] = k;
    }
  upload_gl_tables(x, w, klm);
  upload_mixed_tables(x, w, klm);
  CUDA_TRY(prepare_kernels());
  CUDA_TRY(cudaGetLastError());
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  psq_context* c = new (std::nothrow) psq_context{device, sms > 0 ? sms : 152};
  if (!c) return fail(PSQ_ERR_OOM, "context allocation failed");
  *out = c;
  return PSQ_OK;
}

psq_status psq_context_destroy(psq_context* ctx) {
  delete ctx;
  return PSQ_OK;
}

psq_status psq_job_create(psq_context* ctx, const psq_atom* atoms, int n_atoms, const psq_shell* basis,
                          int n_basis_shells, const psq_shell* aux, int n_aux_shells,
                          const psq_grid_spec* pair_specs, int n_specs, psq_precision precision,
                          psq_job** out) {
  if (!out) return fail(PSQ_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!ctx || !atoms || (!basis && n_basis_shells) || (!aux && n_aux_shells) || !pair_specs)
    return fail(PSQ_ERR_ARG, "NULL argument");
  if (n_atoms < 2) return fail(PSQ_ERR_UNSUPPORTED, "a job needs at least two atoms (got %d)", n_atoms);
  if (n_basis_shells < 0 || n_aux_shells < 0) return fail(PSQ_ERR_ARG, "negative shell count");
  const int npairs = n_atoms * (n_atoms - 1) / 2;
  if (n_specs != 1 && n_specs != npairs)
    return fail(PSQ_ERR_ARG, "n_specs must be 1 or n_atoms*(n_atoms-1)/2 = %d (got %d)", npairs, n_specs);
  if (precision != PSQ_FP64 && precision != PSQ_MIXED) return fail(PSQ_ERR_ARG, "unknown precision");
  for (int i = 0; i < n_atoms; ++i) {
    if (atoms[i].Z < 0 || atoms[i].Z > 200) return fail(PSQ_ERR_ARG, "atom %d: Z = %d", i, atoms[i].Z);
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(atoms[i].xyz[c])) return fail(PSQ_ERR_ARG, "atom %d: position not finite", i);
  }
  for (int i = 0; i < n_atoms; ++i)
    for (int k = i + 1; k < n_atoms; ++k) {
      const double dx = atoms[i].xyz[0] - atoms[k].xyz[0], dy = atoms[i].xyz[1] - atoms[k].xyz[1],
                   dz = atoms[i].xyz[2] - atoms[k].xyz[2];
      if (std::sqrt(dx * dx + dy * dy + dz * dz) < 1e-6)
        return fail(PSQ_ERR_GEOMETRY, "atoms %d and %d coincide", i, k);
    }
  auto check_shells = [&](const psq_shell* s, int n, const char* what) -> psq_status {
    for (int i = 0; i < n; ++i) {
      if (s[i].atom < 0 || s[i].atom >= n_atoms) return fail(PSQ_ERR_ARG, "%s shell %d: atom %d", what, i, s[i].atom);
      if (i > 0 && s[i].atom < s[i - 1].atom)
        return fail(PSQ_ERR_ARG, "%s shells must be grouped by atom in ascending order", what);
      if (s[i].n < 1 || s[i].l < 0 || s[i].l >= s[i].n)
        return fail(PSQ_ERR_ARG, "%s shell %d: n = %d, l = %d (need n > l >= 0)", what, i, s[i].n, s[i].l);
      if (s[i].l > kMaxL || s[i].n > kMaxN)
        return fail(PSQ_ERR_UNSUPPORTED, "%s shell %d: l = %d, n = %d (max l %d, n %d)", what, i, s[i].l, s[i].n,
                    kMaxL, kMaxN);
      if (!(s[i].zeta > 0) || !std::isfinite(s[i].zeta))
        return fail(PSQ_ERR_ARG, "%s shell %d: zeta = %g", what, i, s[i].zeta);
    }
    return PSQ_OK;
  };
  psq_status st = check_shells(basis, n_basis_shells, "basis");
  if (st != PSQ_OK) return st;
  st = check_shells(aux, n_aux_shells, "aux");
  if (st != PSQ_OK) return st;
  for (int i = 0; i < n_specs; ++i) {
    const psq_grid_spec& s = pair_specs[i];
    if (s.n_mu < 1 || s.n_nu < 1 || s.n_phi < 1 || s.n_sp < 1)
      return fail(PSQ_ERR_ARG, "grid spec %d: cell counts and n_sp must be >= 1", i);
    if (s.q_mu < 1 || s.q_nu < 1 || s.q_phi < 1 || s.q_mu > kMaxQ || s.q_nu > kMaxQ || s.q_phi > kMaxQ)
      return fail(PSQ_ERR_UNSUPPORTED, "grid spec %d: Q must be within 1..%d", i, kMaxQ);
    if ((int64_t)s.n_mu * s.n_nu * s.n_phi * s.q_mu * s.q_nu * s.q_phi > (int64_t)1 << 31)
      return fail(PSQ_ERR_UNSUPPORTED, "grid spec %d: more than 2^31 points", i);
  }
  psq_job* j = new (std::nothrow) psq_job();
  if (!j) return fail(PSQ_ERR_OOM, "job allocation failed");
  j->ctx = ctx;
  j->nat = n_atoms;
  j->atoms.assign(atoms, atoms + n_atoms);
  j->basis.assign(basis, basis + n_basis_shells);
  j->aux.assign(aux, aux + n_aux_shells);
  j->specs.assign(pair_specs, pair_specs + n_specs);
  j->prec = precision;
  auto layout = [&](const std::vector<psq_shell>& sh, std::vector<int>& cnt, std::vector<int>& s0,
                    std::vector<int>& s1, std::vector<int>& fatom, std::vector<int>& flocal,
                    std::vector<DevShell>& dsh) {
    cnt.assign(n_atoms, 0);
    s0.assign(n_atoms, (int)sh.size());
    s1.assign(n_atoms, (int)sh.size());
    for (size_t i = 0; i < sh.size(); ++i) {
      const int X = sh[i].atom;
      if (s0[X] == (int)sh.size()) s0[X] = (int)i;
      s1[X] = (int)i + 1;
      DevShell d{};
      d.n = sh[i].n;
      d.l = sh[i].l;
      d.atom = X;
      d.fn0 = cnt[X];
      d.zeta = sh[i].zeta;
      d.norm = std::pow(2.0 * sh[i].zeta, sh[i].n + 0.5) / std::sqrt(factorial(2 * sh[i].n));
      dsh.push_back(d);
      for (int m = 0; m < 2 * sh[i].l + 1; ++m) {
        fatom.push_back(X);
        flocal.push_back(cnt[X] + m);
      }
      cnt[X] += 2 * sh[i].l + 1;
    }
    for (int X = 0; X < n_atoms; ++X)
      if (s1[X] < s0[X] || s0[X] == (int)sh.size()) s0[X] = s1[X] = 0;
  };
  layout(j->basis, j->nb, j->sb0, j->sb1, j->fn_atom, j->fn_local, j->dbs);
  for (size_t q = 0; q < j->dbs.size(); ++q)
    for (int m = 0; m < 2 * j->dbs[q].l + 1; ++m) j->fn_shell.push_back((int)q);
  layout(j->aux, j->na, j->sa0, j->sa1, j->aux_atom, j->aux_local, j->das);
  j->nbf = (int)j->fn_atom.size();
  j->naux = (int)j->aux_atom.size();
  j->nn.assign(n_atoms, 0);
  for (int X = 0; X < n_atoms; ++X) {
    int best = -1;
    double bd = 0;
    for (int Y = 0; Y < n_atoms; ++Y) {
      if (Y == X) continue;
      const double d = norm(sub(pos(j, X), pos(j, Y)));
      if (best < 0 || d < bd) { best = Y; bd = d; }
    }
    j->nn[X] = best;
  }
  *out = j;
  return PSQ_OK;
}

psq_status psq_job_destroy(psq_job* job) {
  delete job;
  return PSQ_OK;
}

psq_status psq_job_sizes(const psq_job* job, int* n_bf, int* n_aux) {
  if (!job) return fail(PSQ_ERR_ARG, "job is NULL");
  if (n_bf) *n_bf = job->nbf;
  if (n_aux) *n_aux = job->naux;
  return PSQ_OK;
}

psq_status psq_job_workspace(const psq_job* job, unsigned mask, size_t* bytes) {
  if (!job || !bytes) return fail(PSQ_ERR_ARG, "NULL argument");
  if (mask & ~31u) return fail(PSQ_ERR_ARG, "mask 0x%x has unknown bits", mask);
  Plan* P = nullptr;
  psq_status st = get_plan(const_cast<psq_job*>(job), mask, &P);
  if (st != PSQ_OK) return st;
  *bytes = P->ws_bytes;
  return PSQ_OK;
}

psq_status psq_job_stats(const psq_job* job, unsigned mask, int* n_grids, int64_t* n_points,
                         double* contractions, int* launches) {
  if (!job) return fail(PSQ_ERR_ARG, "job is NULL");
  if (mask & ~31u) return fail(PSQ_ERR_ARG, "mask 0x%x has unknown bits", mask);
  Plan* P = nullptr;
  psq_status st = get_plan(const_cast<psq_job*>(job), mask, &P);
  if (st != PSQ_OK) return st;
  if (n_grids) *n_grids = (int)P->grids.size();
  if (n_points) *n_points = P->n_points;
  if (contractions) *contractions = P->contractions;
  if (launches) *launches = P->launches;
  return PSQ_OK;
}

psq_status psq_job_issued_flops(const psq_job* job, unsigned mask, double* flops) {
  if (!job || !flops) return fail(PSQ_ERR_ARG, "job or flops is NULL");
  if (mask & ~31u) return fail(PSQ_ERR_ARG, "mask 0x%x has unknown bits", mask);
  Plan* P = nullptr;
  psq_status st = get_plan(const_cast<psq_job*>(job), mask, &P);
  if (st != PSQ_OK) return st;
  *flops = P->issued_flops;
  return PSQ_OK;
}

psq_status psq_compute(psq_job* job, unsigned mask, void* d_workspace, size_t ws_bytes, double* d_out[5],
                       void* stream) {
  return psq::compute_on(job, mask, d_workspace, ws_bytes, d_out, stream, false);
}

}  // extern "C"

psq_status psq::set_error(psq_status s, const char* msg) { return fail(s, "%s", msg); }

int psq::context_device(const psq_context* ctx) { return ctx ? ctx->device : -1; }

int psq::job_device(const psq_job* job) { return job && job->ctx ? job->ctx->device : -1; }

size_t psq::status_offset(psq_job* job, unsigned mask) {
  std::lock_guard<std::mutex> lk(job->mu);
  auto it = job->plans.find(mask);
  return it == job->plans.end() ? 0 : it->second->o_status;
}

namespace {
psq_status run_plan(psq_job* job, Plan* P, unsigned mask, char* ws, double* d_out[5], cudaStream_t s,
                    bool timing = true);
}

psq_status psq::compute_on(psq_job* job, unsigned mask, void* d_workspace, size_t ws_bytes, double* d_out[5],
                           void* stream, bool plan_must_exist) {
  if (!job) return fail(PSQ_ERR_ARG, "job is NULL");
  if (job->ctx->device < 0) return fail(PSQ_ERR_ARG, "the job's context has no device (planning only)");
  if (mask & ~31u) return fail(PSQ_ERR_ARG, "mask 0x%x has unknown bits", mask);
  if (mask == 0) return PSQ_OK;
  if (!d_out) return fail(PSQ_ERR_ARG, "d_out is NULL");
  for (int c = 0; c < 5; ++c)
    if ((mask >> c) & 1 && !d_out[c]) return fail(PSQ_ERR_ARG, "output %d is NULL", c);
  std::shared_ptr<Plan> SP;
  if (plan_must_exist) {
    std::lock_guard<std::mutex> lk(job->mu);
    auto it = job->plans.find(mask);
    if (it == job->plans.end())
      return fail(PSQ_ERR_ARG, "no plan for mask 0x%x yet: call psq_job_workspace(job, mask) first", mask);
    SP = it->second;
  } else {
    psq_status st = get_plan_shared(job, mask, &SP);
    if (st != PSQ_OK) return st;
  }
  Plan* P = SP.get();
  if (!d_workspace || ws_bytes < P->ws_bytes)
    return fail(PSQ_ERR_OOM, "workspace of %zu bytes given, %zu needed", ws_bytes, P->ws_bytes);
  if ((uintptr_t)d_workspace % 256) return fail(PSQ_ERR_ARG, "workspace must be 256-byte aligned");
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != job->ctx->device)
    return fail(PSQ_ERR_ARG, "device %d is current, the job's context is on device %d", dev, job->ctx->device);
  // the allocation-free path (plan_must_exist outside a capture) records no timing events:
  // creating them would allocate
  return run_plan(job, P, mask, (char*)d_workspace, d_out, (cudaStream_t)stream, !plan_must_exist);
}

namespace {

// The launch sequence of one psq_compute on plan P (arguments checked by the caller).
psq_status run_plan(psq_job* job, Plan* P, unsigned mask, char* ws, double* d_out[5], cudaStream_t s,
                    bool timing) {
  auto mark = [&](psq_job* j, int kind, cudaStream_t st) { return timing ? ::mark(j, kind, st) : cudaSuccess; };
  CUDA_TRY(mark(job, 0, s));
  CUDA_TRY(cudaMemcpyAsync(ws, P->staging, P->table_bytes, cudaMemcpyHostToDevice, s));
  if (job->test_stall) CUDA_TRY(cudaMemsetAsync(ws + P->o_status + sizeof(int), 1, sizeof(int), s));
  const LaunchTables t = tables_at(*P, ws);
  double* part = (double*)(ws + P->part_off);
  double* res = (double*)(ws + P->res_off);
  if (P->mixed) {
    float* ops = (float*)(ws + P->ops_off);
    float* ops_lo = ops + P->n_ops;
    NodeEntry* nodes = (NodeEntry*)(ws + P->nodes_off);
    uint8_t* packed = (uint8_t*)(ws + P->pack_off);
    const Panel* panels = (const Panel*)(ws + P->o_pn);
    CUDA_TRY(mark(job, 1, s));
    CUDA_TRY(launch_nodes(t.grids, (int)P->grids.size(), P->max_node_entries, t.edges, nodes, s));
    for (const Plan::Wave& wv : P->waves) {
      LaunchTables tw = t;
      tw.pblocks = t.pblocks + wv.pb0;
      tw.n_pblocks = wv.pb1 - wv.pb0;
      CUDA_TRY(mark(job, 1, s));
      CUDA_TRY(launch_eval_mixed(tw, nodes, (const float2*)(ws + P->o_xi), ops, ops_lo, s));
      CUDA_TRY(mark(job, 5, s));
      CUDA_TRY(launch_pack(t.grids, panels + wv.pn0, wv.pn1 - wv.pn0, (const int*)(ws + P->o_ph) + wv.ph_off, wv.jobs,
                           t.pairs, ops, ops_lo, packed, s));
      CUDA_TRY(mark(job, 2, s));
      CUDA_TRY(launch_contract_ws(t.grids, (const MmaBlock*)(ws + P->o_mb), (const GemmItem*)(ws + P->o_mi),
                                  (const int*)(ws + P->o_cb) + wv.cb_off, wv.n_ctas, panels,
                                  (const PairTile*)(ws + P->o_pt), ops, ops_lo, packed, (float2*)part,
                                  (int*)(ws + P->o_status), job->wait_ns, (const int*)(ws + P->o_status) + 1, s));
      CUDA_TRY(mark(job, 3, s));
      CUDA_TRY(launch_reduce_mixed(t.grids, (const MmaBlock*)(ws + P->o_mb), (int)P->mblocks.size(), t.elem_begin,
                                   P->elem_begin[wv.mb0], P->elem_begin[wv.mb1], t.pairs,
                                   (const double*)(ws + P->o_rc), (const float2*)part, res, s));
    }
  } else {
    double* ops = (double*)(ws + P->ops_off);
    CUDA_TRY(mark(job, 1, s));
    CUDA_TRY(launch_eval_fp64(t, ops, 0, s));
    CUDA_TRY(mark(job, 2, s));
    CUDA_TRY(launch_contract_fp64(t, ops, part, s));
    CUDA_TRY(mark(job, 3, s));
    CUDA_TRY(launch_reduce(t, part, res, s));
  }
  CUDA_TRY(mark(job, 4, s));
  const int* fa = (const int*)(ws + P->o_fa);
  const int* fl = (const int*)(ws + P->o_fl);
  const int* aa = (const int*)(ws + P->o_aa);
  const int* al = (const int*)(ws + P->o_al);
  const unsigned cls[4] = {PSQ_S, PSQ_T, PSQ_V, PSQ_J2};
  for (int c = 0; c < 4; ++c) {
    if (!(mask & cls[c])) continue;
    const int n = c == 3 ? job->naux : job->nbf;
    const int* at = c == 3 ? aa : fa;
    const int* lo = c == 3 ? al : fl;
    // one-centre S and T from their closed forms (the basis shells and each function's shell)
    const bool closed = c < 2;
    CUDA_TRY(launch_assemble((int)cls[c], job->nat, n, 0, at, lo, nullptr, nullptr,
                             (const SrcEntry*)(ws + P->o_src[c]), (const int*)(ws + P->o_ptr[c]), nullptr,
                             closed ? (const DevShell*)(ws + P->o_bsh) : nullptr,
                             closed ? (const int*)(ws + P->o_fs) : nullptr, res, d_out[c], s));
  }
  if (mask & PSQ_J3)
    CUDA_TRY(launch_assemble(16, job->nat, job->nbf, job->naux, fa, fl, aa, al, nullptr, nullptr,
                             (const J3Src*)(ws + P->o_j3), nullptr, nullptr, res, d_out[4], s));
  CUDA_TRY(mark(job, -1, s));
  return PSQ_OK;
}

}  // namespace

extern "C" {

psq_status psq_job_autotune(psq_job* job, unsigned mask, void* d_workspace, size_t ws_bytes, double* d_out[5],
                            void* stream, int* work_split, float* best_ms) {
  if (!job) return fail(PSQ_ERR_ARG, "job is NULL");
  if (job->ctx->device < 0) return fail(PSQ_ERR_ARG, "the job's context has no device (planning only)");
  if (mask & ~31u) return fail(PSQ_ERR_ARG, "mask 0x%x has unknown bits", mask);
  if (mask == 0) return fail(PSQ_ERR_ARG, "mask is empty");
  if (!d_out) return fail(PSQ_ERR_ARG, "d_out is NULL");
  for (int c = 0; c < 5; ++c)
    if ((mask >> c) & 1 && !d_out[c]) return fail(PSQ_ERR_ARG, "output %d is NULL", c);
  if (!d_workspace || (uintptr_t)d_workspace % 256) return fail(PSQ_ERR_ARG, "workspace NULL or not 256-byte aligned");
  // candidates: work items per SM (mixed) or 8-CTA waves per SM (FP64)
  static const int kMixed[] = {2, 4, 6, 8, 16, 32};
  static const int kFp64[] = {2, 4, 8, 16};
  const bool mixed = job->prec == PSQ_MIXED;
  const int* cand = mixed ? kMixed : kFp64;
  const int n_cand = mixed ? 6 : 4;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(PSQ_ERR_CUDA, "cudaEventCreate failed");
  }
  const bool prof = job->prof_on;
  job->prof_on = false;  // the trial runs stay out of the launch timing record
  std::shared_ptr<Plan> best;
  float best_t = 0.0f;
  psq_status st = PSQ_OK;
  for (int k = 0; k < n_cand && st == PSQ_OK; ++k) {
    std::shared_ptr<Plan> p(new (std::nothrow) Plan());
    if (!p) { st = fail(PSQ_ERR_OOM, "plan allocation failed"); break; }
    p->work_split = cand[k];
    st = make_plan(job, mask, *p);
    if (st != PSQ_OK) break;
    if (p->ws_bytes > ws_bytes) continue;  // does not fit the caller's workspace
    char* ws = (char*)d_workspace;
    st = run_plan(job, p.get(), mask, ws, d_out, s);  // warm-up
    for (int r = 0; r < 3 && st == PSQ_OK; ++r) {
      if (r == 0 && cudaEventRecord(e0, s) != cudaSuccess) st = fail(PSQ_ERR_CUDA, "cudaEventRecord failed");
      if (st == PSQ_OK) st = run_plan(job, p.get(), mask, ws, d_out, s);
    }
    if (st != PSQ_OK) break;
    float ms = 0.0f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = fail(PSQ_ERR_CUDA, "timing a candidate failed");
      break;
    }
    ms /= 3.0f;
    if (!best || ms < best_t) {
      best_t = ms;
      best = std::move(p);
    }
  }
  job->prof_on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PSQ_OK) return st;
  if (!best) return fail(PSQ_ERR_OOM, "no candidate plan fits a workspace of %zu bytes", ws_bytes);
  const int chosen = best->work_split;
  {
    std::lock_guard<std::mutex> lk(job->mu);
    job->plans[mask] = std::move(best);
    job->work_split[mask] = chosen;
    // graphs captured with the previous plan of this mask are stale
    for (auto it = job->graphs.begin(); it != job->graphs.end();) {
      if (it->first.mask == mask) {
        cudaGraphExecDestroy(it->second);
        it = job->graphs.erase(it);
      } else {
        ++it;
      }
    }
  }
  if (work_split) *work_split = chosen;
  if (best_ms) *best_ms = best_t;
  return PSQ_OK;
}

psq_status psq_compute_graph(psq_job* job, unsigned mask, void* d_workspace, size_t ws_bytes, double* d_out[5],
                             void* stream) {
  if (!job) return fail(PSQ_ERR_ARG, "job is NULL");
  if (job->ctx->device < 0) return fail(PSQ_ERR_ARG, "the job's context has no device (planning only)");
  if (mask & ~31u) return fail(PSQ_ERR_ARG, "mask 0x%x has unknown bits", mask);
  if (mask == 0) return PSQ_OK;
  if (!d_out) return fail(PSQ_ERR_ARG, "d_out is NULL");
  psq_job::GraphKey key{};
  key.mask = mask;
  key.ws = d_workspace;
  for (int c = 0; c < 5; ++c) key.out[c] = ((mask >> c) & 1) ? d_out[c] : nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  auto it = job->graphs.find(key);
  if (it == job->graphs.end()) {
    // plan first (host work and the page-locked staging buffer stay out of the capture)
    Plan* P = nullptr;
    psq_status st = get_plan(job, mask, &P);
    if (st != PSQ_OK) return st;
    if (!d_workspace || ws_bytes < P->ws_bytes)
      return fail(PSQ_ERR_OOM, "workspace of %zu bytes given, %zu needed", ws_bytes, P->ws_bytes);
    if (!s) return fail(PSQ_ERR_ARG, "graph capture needs a non-default stream");
    CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    job->capturing = true;
    st = psq::compute_on(job, mask, d_workspace, ws_bytes, d_out, stream, true);
    job->capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &graph);
    if (st != PSQ_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ec != cudaSuccess) return fail(PSQ_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ec));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(PSQ_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
    it = job->graphs.emplace(key, exec).first;
  }
  CUDA_TRY(cudaGraphLaunch(it->second, s));
  return PSQ_OK;
}

psq_status psq_job_set_wave_budget(psq_job* job, size_t bytes) {
  if (!job) return fail(PSQ_ERR_ARG, "job is NULL");
  std::lock_guard<std::mutex> lk(job->mu);
  job->wave_bytes = bytes;
  job->plans.clear();
  for (auto& kv : job->graphs) cudaGraphExecDestroy(kv.second);
  job->graphs.clear();
  return PSQ_OK;
}

psq_status psq_job_test_stall(psq_job* job, int on) {
  if (!job) return fail(PSQ_ERR_ARG, "job is NULL");
  job->test_stall = on != 0;
  return PSQ_OK;
}

psq_status psq_job_set_wait_limit(psq_job* job, uint64_t ns) {
  if (!job) return fail(PSQ_ERR_ARG, "job is NULL");
  if (ns < 1 || ns > 60000000000ull) return fail(PSQ_ERR_ARG, "wait limit %llu ns out of range", (unsigned long long)ns);
  job->wait_ns = ns;
  return PSQ_OK;
}

psq_status psq_profile_enable(psq_job* job, int on) {
  if (!job) return fail(PSQ_ERR_ARG, "job is NULL");
  job->prof_on = on != 0;
  return PSQ_OK;
}

psq_status psq_profile_read(psq_job* job, double ms[8], int counts[8]) {
  if (!job || !ms || !counts) return fail(PSQ_ERR_ARG, "NULL argument");
  for (int k = 0; k < 8; ++k) { ms[k] = 0; counts[k] = 0; }
  for (size_t i = 0; i < job->prof.size(); ++i) {
    CUDA_TRY(cudaEventSynchronize(job->prof[i].ev));
  }
  for (size_t i = 0; i + 1 < job->prof.size(); ++i) {
    const int k = job->prof[i].kind;
    if (k < 0 || k >= 8) continue;
    float dt = 0;
    CUDA_TRY(cudaEventElapsedTime(&dt, job->prof[i].ev, job->prof[i + 1].ev));
    ms[k] += dt;
    counts[k] += 1;
  }
  for (auto& r : job->prof) job->ev_free.push_back(r.ev);
  job->prof.clear();
  return PSQ_OK;
}

psq_status psq_job_io_bytes(const psq_job* job, unsigned mask, size_t* h2d, size_t* d2h) {
  if (!job) return fail(PSQ_ERR_ARG, "job is NULL");
  if (mask & ~31u) return fail(PSQ_ERR_ARG, "mask 0x%x has unknown bits", mask);
  Plan* P = nullptr;
  psq_status st = get_plan(const_cast<psq_job*>(job), mask, &P);
  if (st != PSQ_OK) return st;
  size_t out = 0;
  const size_t nb = job->nbf, na = job->naux;
  if (mask & PSQ_S) out += nb * nb;
  if (mask & PSQ_T) out += nb * nb;
  if (mask & PSQ_V) out += nb * nb;
  if (mask & PSQ_J2) out += na * na;
  if (mask & PSQ_J3) out += na * nb * nb;
  if (h2d) *h2d = P->table_bytes;
  if (d2h) *d2h = out * sizeof(double);
  return PSQ_OK;
}

psq_status psq_compute_host(psq_job* job, unsigned mask, void* d_workspace, size_t ws_bytes, double* d_out[5],
                            double* h_out[5], void* stream) {
  psq_status st = psq_compute(job, mask, d_workspace, ws_bytes, d_out, stream);
  if (st != PSQ_OK) return st;
  if (!h_out) return fail(PSQ_ERR_ARG, "h_out is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  for (int c = 0; c < 5; ++c) {
    if (!((mask >> c) & 1)) continue;
    if (!h_out[c]) return fail(PSQ_ERR_ARG, "host output %d is NULL", c);
    size_t n = c < 3 ? (size_t)job->nbf * job->nbf
                     : (c == 3 ? (size_t)job->naux * job->naux : (size_t)job->naux * job->nbf * job->nbf);
    CUDA_TRY(cudaMemcpyAsync(h_out[c], d_out[c], n * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  return psq_check(job, mask, d_workspace, stream);
}

psq_status psq_check(psq_job* job, unsigned mask, void* d_workspace, void* stream) {
  if (!job) return fail(PSQ_ERR_ARG, "job is NULL");
  Plan* P = nullptr;
  psq_status st = get_plan(job, mask, &P);
  if (st != PSQ_OK) return st;
  if (!d_workspace) {  // the allocation-free entry point's scratch on the current device
    st = psq::noalloc_scratch(&d_workspace);
    if (st != PSQ_OK) return st;
  }
  int flag = 0;
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(&flag, (char*)d_workspace + P->o_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (flag) return fail(PSQ_ERR_TIMEOUT, "a bounded device wait expired (status word %d)", flag);
  return PSQ_OK;
}

psq_status psq_job_grid_info(const psq_job* job, int g, int* A, int* B, int* C, int64_t* n_points) {
  if (!job) return fail(PSQ_ERR_ARG, "job is NULL");
  Plan* P = nullptr;
  psq_status st = get_plan(const_cast<psq_job*>(job), PSQ_ALL, &P);
  if (st != PSQ_OK) return st;
  if (g < 0 || g >= (int)P->grids.size()) return fail(PSQ_ERR_ARG, "grid %d of %zu", g, P->grids.size());
  if (A) *A = P->grids[g].A;
  if (B) *B = P->grids[g].B;
  if (C) *C = P->grids[g].C;
  if (n_points) *n_points = P->grids[g].K;
  return PSQ_OK;
}

psq_status psq_job_grid_points(psq_job* job, int g, void* d_workspace, size_t ws_bytes, double* d_out,
                               void* stream) {
  if (!job || !d_out) return fail(PSQ_ERR_ARG, "NULL argument");
  if (job->ctx->device < 0) return fail(PSQ_ERR_ARG, "the job's context has no device (planning only)");
  Plan* P = nullptr;
  psq_status st = get_plan(job, PSQ_ALL, &P);
  if (st != PSQ_OK) return st;
  if (g < 0 || g >= (int)P->grids.size()) return fail(PSQ_ERR_ARG, "grid %d of %zu", g, P->grids.size());
  if (!d_workspace || ws_bytes < P->table_bytes)
    return fail(PSQ_ERR_OOM, "workspace of %zu bytes given, %zu needed", ws_bytes, P->table_bytes);
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)d_workspace;
  CUDA_TRY(cudaMemcpyAsync(ws, P->staging, P->table_bytes, cudaMemcpyHostToDevice, s));
  LaunchTables t = tables_at(*P, ws);
  t.n_elems = P->grids[g].K;
  CUDA_TRY(launch_grid_points(t, g, d_out, s));
  return PSQ_OK;
}

psq_status psq_job_grid_functions(psq_job* job, int g, int kind, void* d_workspace, size_t ws_bytes,
                                  double* d_out, int* rows, void* stream) {
  if (!job || !d_out) return fail(PSQ_ERR_ARG, "NULL argument");
  if (job->ctx->device < 0) return fail(PSQ_ERR_ARG, "the job's context has no device (planning only)");
  if (kind < 0 || kind > 3) return fail(PSQ_ERR_ARG, "kind %d", kind);
  Plan* P = nullptr;
  psq_status st = get_plan(job, PSQ_ALL, &P);
  if (st != PSQ_OK) return st;
  if (g < 0 || g >= (int)P->grids.size()) return fail(PSQ_ERR_ARG, "grid %d of %zu", g, P->grids.size());
  // one-grid table: the grid with only the requested rows
  DevGrid G = P->grids[g];
  G.op_off = 0;
  G.row_F = G.row_L = G.row_G = G.row_U = G.row_W = -1;
  int nrows = kind <= 1 ? G.nFA + G.nFB : G.nG;
  if (kind == 0) G.row_F = 0;
  if (kind == 1) G.row_L = 0;
  if (kind == 2) G.row_G = 0;
  if (kind == 3) G.row_U = 0;
  if (rows) *rows = nrows;
  const bool mixed = job->prec == PSQ_MIXED;
  std::vector<PointBlock> pb;
  for (int64_t p0 = 0; p0 < G.K; p0 += kPointsPerBlock) pb.push_back(PointBlock{0, 0, p0});
  // mixed path: node table of this grid, the FP64 row constants and the hi/lo operand rows
  const int n_nodes = (G.n_mu + G.nt_mu * G.n_sp) * G.q_mu + (G.n_nu + G.nt_nu * G.n_sp) * G.q_nu +
                      (G.n_phi + G.nt_phi * G.n_sp) * G.q_phi;
  std::vector<double> rc;
  if (mixed) row_constants(job, G, kind, rc);
  G.ld = mixed ? (int64_t)align_up((size_t)G.K, 128) : G.K;
  if (mixed) G.nt_off = 0;
  const size_t o_grid = 0, o_pb = align_up(sizeof(DevGrid), 256);
  size_t need = o_pb + align_up(sizeof(PointBlock) * pb.size(), 256);
  const size_t o_nodes = need;
  const size_t o_rc = o_nodes + (mixed ? align_up(sizeof(NodeEntry) * (size_t)n_nodes, 256) : 0);
  const size_t o_ops = o_rc + (mixed ? align_up(sizeof(double) * rc.size(), 256) : 0);
  if (mixed) need = o_ops + align_up(2 * sizeof(float) * (size_t)nrows * (size_t)G.ld, 256);
  if (!d_workspace || ws_bytes < P->table_bytes + need)
    return fail(PSQ_ERR_OOM, "workspace of %zu bytes given, %zu needed", ws_bytes, P->table_bytes + need);
  cudaStream_t s = (cudaStream_t)stream;
  char* ws = (char*)d_workspace;
  CUDA_TRY(cudaMemcpyAsync(ws, P->staging, P->table_bytes, cudaMemcpyHostToDevice, s));
  char* extra = ws + P->table_bytes;
  CUDA_TRY(cudaMemcpyAsync(extra + o_grid, &G, sizeof(G), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(extra + o_pb, pb.data(), sizeof(PointBlock) * pb.size(), cudaMemcpyHostToDevice, s));
  LaunchTables t = tables_at(*P, ws);
  t.grids = (const DevGrid*)(extra + o_grid);
  t.pblocks = (const PointBlock*)(extra + o_pb);
  t.n_pblocks = (int)pb.size();
  if (mixed) {
    if (!rc.empty())
      CUDA_TRY(cudaMemcpyAsync(extra + o_rc, rc.data(), sizeof(double) * rc.size(), cudaMemcpyHostToDevice, s));
    NodeEntry* nodes = (NodeEntry*)(extra + o_nodes);
    float* oh = (float*)(extra + o_ops);
    float* ol = oh + (size_t)nrows * G.ld;
    CUDA_TRY(launch_nodes(t.grids, 1, n_nodes, t.edges, nodes, s));
    CUDA_TRY(launch_eval_mixed(t, nodes, (const float2*)(ws + P->o_xi), oh, ol, s));
    CUDA_TRY(launch_combine_rows(oh, ol, (const double*)(extra + o_rc), nrows, G.K, G.ld, d_out, s));
  } else {
    CUDA_TRY(launch_eval_fp64(t, d_out, 0, s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));  // the host copies above live on this stack frame
  return PSQ_OK;
}

}  // extern "C"
