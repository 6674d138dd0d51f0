// Host program (no GPU): the reverse mode of one M2L pair (m2l_pair_vjp) against
// central differences of the forward pair expression (m2l_pair with acc_finish) in
// long double, for every input (R, source m, Q, O and the target's O / m) of the
// four target / source variants.  Prints the worst relative error per variant and
// exits non-zero above the bound given as argv[1].
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>

#include "pair_vjp.cuh"

using namespace octo;
typedef long double LD;

template <bool FULL, bool TOCT>
static LD objective(const LD* x, const double* Lb) {
  Acc<LD> a;
  acc_zero(a);
  const LD* R = x;
  const LD m = x[3];
  const LD* Q = x + 4;
  const LD* O = x + 10;
  const LD* Oh = x + 20;
  const LD tOh[3] = {Oh[0] + Oh[3] + Oh[5], Oh[1] + Oh[6] + Oh[8], Oh[2] + Oh[7] + Oh[9]};
  const LD rinv = 1.0L / sqrtl(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
  m2l_pair<FULL, TOCT>(R[0], R[1], R[2], m, Q, O, Oh, tOh, rinv, a);
  acc_finish(a);
  LD s = Lb[0] * a.L0;
  for (int i = 0; i < 3; ++i) s += Lb[1 + i] * a.L1[i];
  if (FULL) {
    for (int i = 0; i < 6; ++i) s += Lb[4 + i] * a.L2[i];
    for (int i = 0; i < 10; ++i) s += Lb[10 + i] * a.L3[i];
  }
  for (int i = 0; i < 3; ++i) s += Lb[20 + i] * a.dg[i];
  return s;
}

template <bool FULL, bool TOCT>
static double worst(std::mt19937_64& rng, int trials) {
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  double w = 0.0;
  for (int t = 0; t < trials; ++t) {
    double x[30], Lb[23];
    for (double& v : x) v = U(rng);
    x[0] += 3.0, x[1] += 1.5, x[3] += 2.0;  // |R| away from 0, positive mass
    if (!TOCT)
      for (int i = 20; i < 30; ++i) x[i] = 0.0;
    for (double& v : Lb) v = U(rng);
    if (!FULL)
      for (int i = 4; i < 20; ++i) Lb[i] = 0.0;
    PairVJP g;
    m2l_pair_vjp<FULL, TOCT, true, true>(x[0], x[1], x[2], x[3], x + 4, x + 10, x + 20, Lb, g);
    double an[30];
    for (int i = 0; i < 3; ++i) an[i] = g.R[i];
    an[3] = g.m;
    for (int i = 0; i < 6; ++i) an[4 + i] = g.Q[i];
    for (int i = 0; i < 10; ++i) an[10 + i] = g.O[i];
    for (int i = 0; i < 10; ++i) an[20 + i] = TOCT ? g.Oh[i] : 0.0;
    for (int k = 0; k < (TOCT ? 30 : 20); ++k) {
      LD xp[30], xm[30];
      for (int i = 0; i < 30; ++i) xp[i] = xm[i] = x[i];
      const LD h = 1e-6L;
      xp[k] += h, xm[k] -= h;
      const LD fd = (objective<FULL, TOCT>(xp, Lb) - objective<FULL, TOCT>(xm, Lb)) / (2 * h);
      const double e = std::fabs((double)fd - an[k]) / (1e-3 + std::fabs((double)fd));
      if (e > w) w = e;
    }
  }
  return w;
}

int main(int argc, char** argv) {
  const double bound = argc > 1 ? std::atof(argv[1]) : 1e-8;
  std::mt19937_64 rng(7);
  const double w[4] = {worst<true, true>(rng, 100), worst<true, false>(rng, 100), worst<false, true>(rng, 100),
                       worst<false, false>(rng, 100)};
  std::printf("worst relative error: full+oct %.3e full %.3e oct %.3e leaf %.3e\n", w[0], w[1], w[2], w[3]);
  for (double v : w)
    if (!(v <= bound)) return 1;
  return 0;
}
