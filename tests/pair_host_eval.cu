// Host program (no GPU): evaluates the device pair expression of the solver
// (m2l_pair + acc_finish, device.cuh) for records read from stdin, so that a test
// can compare it with the oracle.  Input per line: a flag (1 = refined target with
// L2/L3 and an octupole, 0 = leaf target, 2 = refined target in float32 as the
// mixed-precision far field evaluates it), then target record A and source record B
// (20 values each: m, X(3), M2(6), M3(10), packed as in the multipole arrays).
// Output per line: the 23 local-expansion values (L0, L1(3), L2(6), L3(10), dg(3)),
// L2/L3 zero for a leaf target.
#include <cmath>
#include <cstdio>

#include "device.cuh"

using namespace octo;

template <bool FULL, typename T>
static void eval(const double* A, const double* B, double* out) {
  Acc<T> a;
  acc_zero(a);
  T b[20];
  for (int i = 0; i < 20; ++i) b[i] = (T)B[i];
  const T R0 = (T)A[1] - b[1], R1 = (T)A[2] - b[2], R2 = (T)A[3] - b[3];
  const T rinv = (T)1 / std::sqrt(R0 * R0 + R1 * R1 + R2 * R2);
  T Oh[10], tOh[3];
  const T inv_m = (T)1 / (T)A[0];
  for (int i = 0; i < 10; ++i) Oh[i] = FULL ? (T)A[10 + i] * inv_m : (T)0;
  tOh[0] = Oh[0] + Oh[3] + Oh[5];
  tOh[1] = Oh[1] + Oh[6] + Oh[8];
  tOh[2] = Oh[2] + Oh[7] + Oh[9];
  m2l_pair<FULL, FULL>(R0, R1, R2, b[0], b + 4, b + 10, Oh, tOh, rinv, a);
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
    if (full == 2)
      eval<true, float>(A, B, out);
    else if (full == 1)
      eval<true, double>(A, B, out);
    else
      eval<false, double>(A, B, out);
    for (int i = 0; i < 23; ++i) std::printf("%.17g%c", out[i], i == 22 ? '\n' : ' ');
  }
  return 0;
}
