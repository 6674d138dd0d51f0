// Host program (no GPU): evaluates the device pair expression of the solver
// (m2l_pair + acc_finish, device.cuh) for records read from stdin, so that a test
// can compare it with the oracle.  Input per line: a flag (1 = refined target with
// L2/L3 and an octupole, 0 = leaf target, 2 = refined target in float32 as the
// mixed-precision far field evaluates it; the paired float32 expression
// m2l_pair_x2 of pair_x2.cuh: 3 = refined target, source in lane 0 and lane 1
// masked to zero moments, 4 = the same with the lanes swapped, 5 = the source in
// both lanes, 6 = leaf target, lane 1 masked), then target record A and source
// record B (20 values each: m, X(3), M2(6), M3(10), packed as in the multipole
// arrays).  Output per line: the 23 local-expansion values (L0, L1(3), L2(6),
// L3(10), dg(3)), L2/L3 zero for a leaf target.
#include <cmath>
#include <cstdio>

#include "device.cuh"
#include "pair_x2.cuh"

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

struct LeafSums {  // the partial sums of a leaf target
  float L0, L1[3], dg[3];
};

// The paired expression: lane `src` (0, 1 or 2 = both) holds source B, the other
// lane B with zero mass and moments.
template <bool INTERIOR>
static void eval_x2(const double* A, const double* B, int src, double* out) {
  F2 R[3], m, Q[6], O[10];
  for (int i = 0; i < 3; ++i) {
    const float r = (float)A[1 + i] - (float)B[1 + i];
    R[i] = f2(r, r);
  }
  const float w0 = src != 1 ? 1.0f : 0.0f, w1 = src != 0 ? 1.0f : 0.0f;
  m = f2((float)B[0] * w0, (float)B[0] * w1);
  for (int i = 0; i < 6; ++i) Q[i] = f2((float)B[4 + i] * w0, (float)B[4 + i] * w1);
  for (int i = 0; i < 10; ++i) O[i] = f2((float)B[10 + i] * w0, (float)B[10 + i] * w1);
  const F2 rinv = rsqrt2(fma2(R[0], R[0], fma2(R[1], R[1], R[2] * R[2])));
  for (int i = 0; i < 23; ++i) out[i] = 0.0;
  if constexpr (INTERIOR) {
    float Oh[10], tOh[3];
    const float inv_m = 1.0f / (float)A[0];
    for (int i = 0; i < 10; ++i) Oh[i] = (float)A[10 + i] * inv_m;
    tOh[0] = Oh[0] + Oh[3] + Oh[5];
    tOh[1] = Oh[1] + Oh[6] + Oh[8];
    tOh[2] = Oh[2] + Oh[7] + Oh[9];
    Acc<float> a;
    acc_zero(a);
    m2l_pair_x2<true>(R[0], R[1], R[2], m, Q, O, Oh, tOh, rinv, a);
    acc_finish(a);
    out[0] = a.L0;
    for (int i = 0; i < 3; ++i) out[1 + i] = a.L1[i], out[20 + i] = a.dg[i];
    for (int i = 0; i < 6; ++i) out[4 + i] = a.L2[i];
    for (int i = 0; i < 10; ++i) out[10 + i] = a.L3[i];
  } else {
    LeafSums a = {0.0f, {0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
    m2l_pair_x2<false>(R[0], R[1], R[2], m, Q, O, nullptr, nullptr, rinv, a);
    out[0] = a.L0;
    for (int i = 0; i < 3; ++i) out[1 + i] = a.L1[i], out[20 + i] = a.dg[i];
  }
}

int main() {
  int full;
  double A[20], B[20], out[23];
  while (std::scanf("%d", &full) == 1) {
    for (double& v : A) std::scanf("%lf", &v);
    for (double& v : B) std::scanf("%lf", &v);
    if (full >= 3 && full <= 5)
      eval_x2<true>(A, B, full - 3, out);
    else if (full == 6)
      eval_x2<false>(A, B, 0, out);
    else if (full == 2)
      eval<true, float>(A, B, out);
    else if (full == 1)
      eval<true, double>(A, B, out);
    else
      eval<false, double>(A, B, out);
    for (int i = 0; i < 23; ++i) std::printf("%.17g%c", out[i], i == 22 ? '\n' : ' ');
  }
  return 0;
}
