// Packed symmetric Cartesian tensors of rank 0..5 and the derivative tensors
// D^(n) = grad^n (1/|R|), for the adjoint kernels.
//
// A rank-n component is identified by its exponents (a, b, c), a + b + c = n
// (the number of x, y and z indices).  Components of one rank are ordered by
// decreasing a, then decreasing b (for rank 2: xx, xy, xz, yy, yz, zz; rank 3:
// xxx, xxy, xxz, xyy, xyz, xzz, yyy, yyz, yzz, zzz - the order of the stored
// multipoles and local expansions).  All ranks 0..5 are concatenated (56 values).
// The index helpers are constexpr so that, inside fully unrolled loops, every
// index folds to a constant and the packed arrays stay in registers.
//
// D^(n) with exponents (a, b, c) follows from differentiating a radial function:
//   d^a_x d^b_y d^c_z F = sum_{i,j,k} H(a,i) H(b,j) H(c,k) x^(a-2i) y^(b-2j) z^(c-2k) F_{n-i-j-k},
//   H(a,i) = a! / (2^i i! (a-2i)!),  F_m = (r^-1 d/dr)^m (1/r) = (-1)^m (2m-1)!! r^-(2m+1).
#pragma once

namespace octo {
namespace sym {

constexpr int kNComp = 56;

__host__ __device__ constexpr int rank_off(int n) { return n * (n + 1) * (n + 2) / 6; }

// The helpers below are loop-free so that they fold to constants immediately
// inside the unrolled loops of the kernels (compile time stays short).
__host__ __device__ constexpr int rank_of(int q) {
  return q < 1 ? 0 : q < 4 ? 1 : q < 10 ? 2 : q < 20 ? 3 : q < 35 ? 4 : 5;
}

// position of the component with exponents (a, b, c): ranks before it, then
// (n - a)(n - a + 1) / 2 components with a larger x exponent, then decreasing b
__host__ __device__ constexpr int comp_index(int a, int b, int c) {
  return rank_off(a + b + c) + (b + c) * (b + c + 1) / 2 + c;
}

// m with m (m + 1) / 2 <= k < (m + 1)(m + 2) / 2, for k < 21
__host__ __device__ constexpr int tri_root(int k) {
  return k < 1 ? 0 : k < 3 ? 1 : k < 6 ? 2 : k < 10 ? 3 : k < 15 ? 4 : 5;
}

// exponent of axis d of component q
__host__ __device__ constexpr int ex(int q, int d) {
  return d == 0 ? rank_of(q) - tri_root(q - rank_off(rank_of(q)))
         : d == 1 ? tri_root(q - rank_off(rank_of(q))) -
                        (q - rank_off(rank_of(q)) - tri_root(q - rank_off(rank_of(q))) *
                                                        (tri_root(q - rank_off(rank_of(q))) + 1) / 2)
                  : q - rank_off(rank_of(q)) -
                        tri_root(q - rank_off(rank_of(q))) * (tri_root(q - rank_off(rank_of(q))) + 1) / 2;
}

__host__ __device__ constexpr double fact(int n) {
  return n <= 1 ? 1.0 : n == 2 ? 2.0 : n == 3 ? 6.0 : n == 4 ? 24.0 : n == 5 ? 120.0 : 720.0;
}

// copies of the component in the full tensor: n! / (a! b! c!)
__host__ __device__ constexpr double mult(int q) {
  return fact(rank_of(q)) / (fact(ex(q, 0)) * fact(ex(q, 1)) * fact(ex(q, 2)));
}

__host__ __device__ constexpr int up(int q, int d) {
  return comp_index(ex(q, 0) + (d == 0), ex(q, 1) + (d == 1), ex(q, 2) + (d == 2));
}

__host__ __device__ constexpr int down(int q, int d) {
  return ex(q, d) == 0 ? -1 : comp_index(ex(q, 0) - (d == 0), ex(q, 1) - (d == 1), ex(q, 2) - (d == 2));
}

// Hermite terms of component q: term k <-> (i, j, l)
__host__ __device__ constexpr int nterm(int q) { return (ex(q, 0) / 2 + 1) * (ex(q, 1) / 2 + 1) * (ex(q, 2) / 2 + 1); }
__host__ __device__ constexpr int term_i(int q, int k) { return k / ((ex(q, 1) / 2 + 1) * (ex(q, 2) / 2 + 1)); }
__host__ __device__ constexpr int term_j(int q, int k) { return (k / (ex(q, 2) / 2 + 1)) % (ex(q, 1) / 2 + 1); }
__host__ __device__ constexpr int term_l(int q, int k) { return k % (ex(q, 2) / 2 + 1); }
__host__ __device__ constexpr double hcoef(int a, int i) { return fact(a) / (fact(i) * fact(a - 2 * i) * (double)(1 << i)); }

// All D^(n), n = 0..5, packed, at R.
__device__ __forceinline__ void derivatives(double x, double y, double z, double* D) {
  const double r2 = fma(x, x, fma(y, y, z * z));
  double F[6];
  F[0] = 1.0 / sqrt(r2);
  const double ir2 = 1.0 / r2;
#pragma unroll
  for (int m = 1; m < 6; ++m) F[m] = -(2.0 * m - 1.0) * F[m - 1] * ir2;
  double px[6], py[6], pz[6];
  px[0] = py[0] = pz[0] = 1.0;
#pragma unroll
  for (int k = 1; k < 6; ++k) px[k] = px[k - 1] * x, py[k] = py[k - 1] * y, pz[k] = pz[k - 1] * z;
#pragma unroll
  for (int q = 0; q < kNComp; ++q) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < nterm(q)) {
        const int i = term_i(q, k), j = term_j(q, k), l = term_l(q, k);
        const int a = ex(q, 0), b = ex(q, 1), c = ex(q, 2);
        s += hcoef(a, i) * hcoef(b, j) * hcoef(c, l) * px[a - 2 * i] * py[b - 2 * j] * pz[c - 2 * l] *
             F[rank_of(q) - i - j - l];
      }
    D[q] = s;
  }
}

}  // namespace sym
}  // namespace octo
