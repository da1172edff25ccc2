// CPU driver for the double-float arithmetic of the mixed path (psq_df.cuh built with
// PSQ_DF_HOST).  Reads one request per line from stdin and prints each result as
// "hi lo" pairs (%.9g each, so the floats round-trip):
//   exp x              e^-x
//   div a b            a / b
//   sqrt a             sqrt(a)
//   radial k n l x     radial factor of kind k (0 chi, 1 lap chi, 2 V^P) at x = zeta r
//   ylm L ux uy uz     the (L+1)^2 unnormalised real harmonics
// Inputs are FP64 numbers, split into (hi, lo) pairs.
#include <cmath>
#include <cstdio>
#include <iostream>
#include <sstream>
#include <string>

#define PSQ_DF_HOST
#include "psq_df.cuh"

using psq::dfa::df;

static df split(double v) {
  const float h = (float)v;
  return df{h, (float)(v - (double)h)};
}

static void put(df v) { std::printf(" %.9g %.9g", v.h, v.l); }

int main() {
  // constants as the library uploads them
  psq::dfa::float2 tab[64];
  for (int j = 0; j < 64; ++j) {
    const df t = split(std::exp2(-j / 64.0));
    tab[j] = {t.h, t.l};
  }
  const double l64 = 0.693147180559945309417232121458 / 64.0;
  int e2 = 0;
  std::frexp(l64, &e2);
  const double c1 = std::ldexp(std::nearbyint(std::ldexp(l64, 10 - e2)), e2 - 10);
  const float c2 = (float)(l64 - c1);
  const float c3 = (float)(l64 - c1 - (double)c2);
  const psq::dfa::ExpConsts ec{(float)(64.0 / 0.693147180559945309417232121458), (float)c1, c2, c3};
  psq::dfa::float2 fact[40];
  double f = 1.0;
  for (int k = 0; k < 40; ++k) {
    if (k > 0) f *= k;
    const df t = split(f);
    fact[k] = {t.h, t.l};
  }
  float rcp[128];
  rcp[0] = 0.0f;
  for (int k = 1; k < 128; ++k) rcp[k] = (float)(1.0 / k);
  std::string line;
  while (std::getline(std::cin, line)) {
    std::istringstream in(line);
    std::string op;
    in >> op;
    if (op == "exp") {
      double x;
      in >> x;
      put(psq::dfa::exp_neg(split(x), ec, tab));
    } else if (op == "div") {
      double a, b;
      in >> a >> b;
      put(psq::dfa::div(split(a), split(b)));
    } else if (op == "sqrt") {
      double a;
      in >> a;
      put(psq::dfa::sqrt(split(a)));
    } else if (op == "radial") {
      int k, n, l;
      double x;
      in >> k >> n >> l >> x;
      const df X = split(x);
      put(psq::dfa::radial(k, n, l, X, psq::dfa::exp_neg(X, ec, tab), psq::dfa::rcp(X), fact, rcp));
    } else if (op == "ylm") {
      int L;
      double ux, uy, uz;
      in >> L >> ux >> uy >> uz;
      df Y[49];
      psq::dfa::real_ylm(L, split(ux), split(uy), split(uz), Y, rcp);
      for (int i = 0; i < (L + 1) * (L + 1); ++i) put(Y[i]);
    } else {
      continue;
    }
    std::printf("\n");
  }
  return 0;
}
