// Double-float ("double-word") arithmetic on pairs of FP32 numbers (hi + lo, |lo| <= ulp(hi)/2),
// about 48 significant bits, for the mixed path's function values and weights.
//
// Methods (published; written here from their definitions):
//  * Knuth's TwoSum and Dekker's Fast2Sum: the exact sum of two floats as a pair;
//  * the FMA-based exact product (the rounding error of a*b is fma(a, b, -a*b));
//  * the double-word sum, product and quotient built on them, in the forms analysed by
//    Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic building blocks
//    of double-word arithmetic", ACM TOMS 44 (2017): relative errors of a few units of 2^-48;
//  * Dekker's square root (one correction of the FP32 root by the exact residual);
//  * e^-x by additive range reduction with a three-part ln 2 / 64 (Cody and Waite), a 64-entry
//    table of 2^(-j/64) and the Taylor series of e^-r on |r| <= ln 2 / 128.
// Every step uses the _rn intrinsics so that no rounding is fused or reordered away.
//
// With PSQ_DF_HOST defined the same code compiles for the CPU (IEEE single arithmetic, the
// C library's fmaf), which the CPU tests use to check it against FP64 references.
#pragma once

#ifdef PSQ_DF_HOST
#include <cmath>
#include <cstring>
#define PSQ_DF_FN inline
namespace psq {
namespace dfa {
inline float __fadd_rn(float a, float b) { volatile float r = a + b; return r; }
inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
inline float __fmul_rn(float a, float b) { volatile float r = a * b; return r; }
inline float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
inline float __fdividef(float a, float b) { volatile float r = a / b; return r; }
inline float __int_as_float(int i) { float f; std::memcpy(&f, &i, 4); return f; }
struct float2 { float x, y; };
}  // namespace dfa
}  // namespace psq
#else
#include <cuda_runtime.h>
#define PSQ_DF_FN __device__ __forceinline__
#endif

namespace psq {
namespace dfa {

struct df {
  float h, l;
};

PSQ_DF_FN df mk(float h) { return {h, 0.0f}; }

// a + b exactly (Knuth).
PSQ_DF_FN df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// a + b exactly when |a| >= |b| or a == 0 (Dekker).
PSQ_DF_FN df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a * b exactly.
PSQ_DF_FN df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

PSQ_DF_FN df mul(df x, df y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return fast_two_sum(p, e);
}

PSQ_DF_FN df mul_f(df x, float f) {
  const float p = __fmul_rn(x.h, f);
  float e = __fmaf_rn(x.h, f, -p);
  e = __fmaf_rn(x.l, f, e);
  return fast_two_sum(p, e);
}

// Exact scaling by a power of two (no underflow below 2^-126 assumed).
PSQ_DF_FN df scale2(df x, float p2) { return {__fmul_rn(x.h, p2), __fmul_rn(x.l, p2)}; }

// Accurate sum (two TwoSums): safe under cancellation.
PSQ_DF_FN df add(df x, df y) {
  df s = two_sum(x.h, y.h);
  const df t = two_sum(x.l, y.l);
  s = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(s.h, __fadd_rn(s.l, t.l));
}

PSQ_DF_FN df neg(df x) { return {-x.h, -x.l}; }
PSQ_DF_FN df sub(df x, df y) { return add(x, neg(y)); }

PSQ_DF_FN df add_f(df x, float f) {
  const df s = two_sum(x.h, f);
  return fast_two_sum(s.h, __fadd_rn(x.l, s.l));
}

// x / d for a float d: FP32 quotient, then the exact residual x - q d divided once more.
PSQ_DF_FN df div_f(df x, float d) {
  const float q = __fdividef(x.h, d);
  const df p = two_prod(q, d);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.h, p.h), p.l), x.l);
  return fast_two_sum(q, __fdividef(r, d));
}

// x / k for a small positive integer k, with rcp[k] ~ 1/k (FP32): quotient from the table
// reciprocal, the exact residual x - q k divided once more (no SFU instruction).
PSQ_DF_FN df div_k(df x, int k, const float* rcp) {
  const float r = rcp[k];
  const float q = __fmul_rn(x.h, r);
  const df p = two_prod(q, (float)k);
  const float e = __fadd_rn(__fsub_rn(__fsub_rn(x.h, p.h), p.l), x.l);
  return fast_two_sum(q, __fmul_rn(e, r));
}

// x / y.
PSQ_DF_FN df div(df x, df y) {
  const float q = __fdividef(x.h, y.h);
  const df p = mul_f(y, q);
  const float r = __fadd_rn(__fsub_rn(x.h, p.h), __fsub_rn(x.l, p.l));
  return fast_two_sum(q, __fdividef(r, y.h));
}

PSQ_DF_FN df rcp(df y) { return div(mk(1.0f), y); }

// sqrt(x), x > 0 (Dekker): s = sqrtf(x_h), then s + (x - s^2) / (2 s) with x - s^2 exact.
PSQ_DF_FN df sqrt(df x) {
  const float s = sqrtf(x.h);
  const df p = two_prod(s, s);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.h, p.h), p.l), x.l);
  return fast_two_sum(s, __fdividef(r, __fmul_rn(2.0f, s)));
}

// x^n, n >= 0, by repeated products.
PSQ_DF_FN df pow_i(df x, int n) {
  df r = mk(1.0f);
  for (int i = 0; i < n; ++i) r = mul(r, x);
  return r;
}

// c x^n, the factor c taken first (with x < 1 no intermediate falls below the result).
PSQ_DF_FN df mul_pow(df c, df x, int n) {
  for (int i = 0; i < n; ++i) c = mul(c, x);
  return c;
}

PSQ_DF_FN double to_double(df x) { return (double)x.h + (double)x.l; }

// Constants of e^-x: ln 2 / 64 = kL1 + kL2 + kL3 with kL1 of 10 significant bits (k * kL1
// exact for k < 2^14), and 64 / ln 2 for the reduction index.  Set by the host.
struct ExpConsts {
  float inv, c1, c2, c3;
};

// e^-x for x >= 0.  tab[j] = 2^(-j/64) (hi, lo) for j = 0..63, in shared memory.
// x = k ln2/64 + r, |r| <= ln2/128, e^-x = 2^-(k/64) e^-r with k = 64 q + j.
PSQ_DF_FN df exp_neg(df x, const ExpConsts& c, const float2* tab) {
  if (!(x.h < 87.0f)) return mk(0.0f);  // below 1.7e-38: zero at this precision
  // nearest integer of x 64/ln2 (< 2^13) by the FP32 magic number 1.5 * 2^23
  const float kf = __fsub_rn(__fadd_rn(__fmul_rn(x.h, c.inv), 12582912.0f), 12582912.0f);
  const int k = (int)kf;
  // x - k c1 is exact (k c1 has at most 24 bits and lies within a factor 2 of x_h)
  df r = two_sum(__fsub_rn(x.h, __fmul_rn(kf, c.c1)), x.l);
  r = sub(r, two_prod(kf, c.c2));
  r = add_f(r, -__fmul_rn(kf, c.c3));
  // e^-r = 1 - r + r^2/2 - r^3/6 + r^4/24 - r^5/120 (next term < 2^-54)
  const float h = r.h;
  const float tail = __fmul_rn(__fmul_rn(__fmul_rn(h, h), h), fmaf(h, fmaf(h, -1.0f / 120.0f, 1.0f / 24.0f), -1.0f / 6.0f));
  df q = two_prod(h, h);
  q = fast_two_sum(q.h, __fmaf_rn(__fmul_rn(2.0f, h), r.l, q.l));
  q = scale2(q, 0.5f);
  df e = add_f(q, tail);
  e = sub(e, r);
  e = add_f(e, 1.0f);
  const float2 t = tab[k & 63];
  e = mul(e, df{t.x, t.y});
  return scale2(e, __int_as_float((127 - (k >> 6)) << 23));
}


// Sum of two values of one sign (no cancellation): one TwoSum.
PSQ_DF_FN df add_same(df x, df y) {
  const df s = two_sum(x.h, y.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}

// Unnormalised real harmonics Yu_lm(u) = Q_l^|m|(u_z) {Re, Im}(u_x + i u_y)^|m| (the norms K_lm
// are left to the FP64 row constants), index l*l + l + m, l <= lmax <= 6: Q_m^m = (2m-1)!!,
// Q_{m+1}^m = (2m+1) u_z Q_m^m, (l-m) Q_l^m = (2l-1) u_z Q_{l-1}^m - (l+m-1) Q_{l-2}^m.
PSQ_DF_FN void real_ylm(int lmax, df ux, df uy, df uz, df* Y, const float* rcp) {
  df C[7], S[7];
  C[0] = mk(1.0f);
  S[0] = mk(0.0f);
#pragma unroll 1
  for (int m = 1; m <= lmax; ++m) {
    C[m] = sub(mul(ux, C[m - 1]), mul(uy, S[m - 1]));
    S[m] = add(mul(ux, S[m - 1]), mul(uy, C[m - 1]));
  }
  float dfact = 1.0f;  // (2m-1)!!, exact in FP32 for m <= 6
#pragma unroll 1
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) dfact *= (float)(2 * m - 1);
    df q2 = mk(0.0f), q1 = mk(dfact);
#pragma unroll 1
    for (int l = m; l <= lmax; ++l) {
      df q;
      if (l == m) {
        q = mk(dfact);
      } else if (l == m + 1) {
        q = mul_f(uz, (float)(2 * m + 1) * dfact);
      } else {
        const df a = mul_f(mul(uz, q1), (float)(2 * l - 1));
        q = div_k(sub(a, mul_f(q2, (float)(l + m - 1))), l - m, rcp);
      }
      if (l > m) { q2 = q1; q1 = q; }
      const int base = l * l + l;
      if (m == 0) {
        Y[base] = q;
      } else {
        Y[base + m] = mul(q, C[m]);
        Y[base - m] = mul(q, S[m]);
      }
    }
  }
}

// Radial factors as functions of x = zeta r (the powers of zeta and the norms are left to the
// FP64 row constants):
//   kind 0 chi: x^(n-1) e^-x;  kind 1 lap chi: [(n(n-1) - l(l+1))/x^2 - 2n/x + 1] x^(n-1) e^-x;
//   kind 2 V^P: gamma(n+l+2, x)/x^(l+1) + Gamma(n-l+1, x) x^l, with the integer incomplete gamma
//   functions Gamma(k, x) = (k-1)! e^-x sum_{j<k} x^j/j! and, below x = k, the positive series
//   gamma(k, x) = x^k e^-x sum_j x^j / (k (k+1) ... (k+j)) (no cancellation); above, (k-1)! -
//   Gamma(k, x).  ex = e^-x, ix = 1/x; fact[k] = k! as (hi, lo); rcp[k] = 1/k in FP32 (k < 128).
PSQ_DF_FN df radial(int kind, int n, int l, df x, df ex, df ix, const float2* fact, const float* rcp) {
  if (ex.h == 0.0f) {
    // e^-x below FP32 range (x >= 87; grids of distant pairs reach x ~ 1e5, where the finite
    // sums below would overflow): the upper incomplete gamma terms vanish, V^P is the
    // multipole term (k-1)!/x^(l+1), chi and lap chi are 0
    if (kind != 2) return mk(0.0f);
    const int k1 = n + l + 2;
    return mul_pow(df{fact[k1 - 1].x, fact[k1 - 1].y}, ix, l + 1);
  }
  if (kind == 2) {
    const int k1 = n + l + 2, k2 = n - l + 1;
    df inner;
    if (x.h < (float)k1) {
      df t = div_k(mk(1.0f), k1, rcp), s = t;
      int j = 1;
#pragma unroll 1  // data-dependent trip counts: rolled loops keep the code small
      for (; j < 100; ++j) {  // double-float terms while they reach 2^-24 of the sum
        t = div_k(mul(t, x), k1 + j, rcp);
        s = add_same(s, t);
        if (t.h < 5.9604645e-8f * s.h) break;
      }
      float tf = t.h, sf = 0.0f;  // the rest in FP32 (each term below 2^-24 of the sum)
#pragma unroll 1
      for (++j; j < 400 && k1 + j < 128; ++j) {
        tf *= x.h * rcp[k1 + j];
        sf += tf;
        if (tf < 1e-17f * s.h) break;
      }
      s = add_f(s, sf);
      inner = mul(mul(pow_i(x, n + 1), ex), s);
    } else {
      df t = mk(1.0f), s = mk(1.0f);
#pragma unroll 1
      for (int j = 1; j < k1; ++j) {
        t = div_k(mul(t, x), j, rcp);
        s = add_same(s, t);
      }
      const df q = sub(mk(1.0f), mul(ex, s));  // regularised lower gamma, >= 1/2 for x >= k
      inner = mul_pow(mul(df{fact[k1 - 1].x, fact[k1 - 1].y}, q), ix, l + 1);
    }
    df t = mk(1.0f), s = mk(1.0f);
#pragma unroll 1
    for (int j = 1; j < k2; ++j) {
      t = div_k(mul(t, x), j, rcp);
      s = add_same(s, t);
    }
    const df outer = mul(mul(mul(df{fact[k2 - 1].x, fact[k2 - 1].y}, ex), s), pow_i(x, l));
    return add(inner, outer);
  }
  const df g = mul(pow_i(x, n - 1), ex);
  if (kind == 0) return g;
  const float A = (float)(n * (n - 1) - l * (l + 1));
  const df u = add_f(mul_f(ix, A), -2.0f * (float)n);
  return mul(add_f(mul(u, ix), 1.0f), g);
}

}  // namespace dfa
}  // namespace psq
