// Host program (no GPU): evaluates the device pair expression of the solver
// (m2l_pair + acc_finish, device.cuh) for records read from stdin, so that a test
// can compare it with the oracle.  Input per line: a flag (1 = refined target with
// L2/L3 and an octupole, 0 = leaf target), then target record A and source record B
// (20 values each: m, X(3), M2(6), M3(10), packed as in the multipole arrays).
// Output per line: the 23 local-expansion values (L0, L1(3), L2(6), L3(10), dg(3)),
// L2/L3 zero for a leaf target.
#include <cmath>
#include <cstdio>

#include "device.cuh"

using namespace octo;

template <bool FULL>
static void eval(const double* A, const double* B, double* out) {
  Acc<double> a;
  acc_zero(a);
  const double R0 = A[1] - B[1], R1 = A[2] - B[2], R2 = A[3] - B[3];
  const double rinv = 1.0 / std::sqrt(R0 * R0 + R1 * R1 + R2 * R2);
  double Oh[10], tOh[3];
  const double inv_m = 1.0 / A[0];
  for (int i = 0; i < 10; ++i) Oh[i] = FULL ? A[10 + i] * inv_m : 0.0;
  tOh[0] = Oh[0] + Oh[3] + Oh[5];
  tOh[1] = Oh[1] + Oh[6] + Oh[8];
  tOh[2] = Oh[2] + Oh[7] + Oh[9];
  m2l_pair<FULL, FULL>(R0, R1, R2, B[0], B + 4, B + 10, Oh, tOh, rinv, a);
  acc_finish(a);
  out[0] = a.L0;
  for (int i = 0; i < 3; ++i) out[1 + i] = a.L1[i], out[20 + i] = a.dg[i];
  for (int i = 0; i < 6; ++i) out[4 + i] = FULL ? a.L2[i] : 0.0;
  for (int i = 0; i < 10; ++i) out[10 + i] = FULL ? a.L3[i] : 0.0;
}

int main() {
  int full;
  double A[20], B[20], out[23];
  while (std::scanf("%d", &full) == 1) {
    for (double& v : A) std::scanf("%lf", &v);
    for (double& v : B) std::scanf("%lf", &v);
    if (full)
      eval<true>(A, B, out);
    else
      eval<false>(A, B, out);
    for (int i = 0; i < 23; ++i) std::printf("%.17g%c", out[i], i == 22 ? '\n' : ' ');
  }
  return 0;
}
