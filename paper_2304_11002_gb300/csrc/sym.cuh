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

__host__ __device__ constexpr int rank_of(int q) {
  int n = 0;
  while (rank_off(n + 1) <= q) ++n;
  return n;
}

__host__ __device__ constexpr int comp_index(int a, int b, int c) {
  const int n = a + b + c;
  int idx = 0;
  for (int a2 = n; a2 > a; --a2) idx += n - a2 + 1;
  return rank_off(n) + idx + (n - a - b);
}

// exponent of axis d of component q
__host__ __device__ constexpr int ex(int q, int d) {
  const int n = rank_of(q);
  int k = q - rank_off(n);
  for (int a = n; a >= 0; --a) {
    const int cnt = n - a + 1;
    if (k < cnt) {
      const int b = n - a - k;
      return d == 0 ? a : (d == 1 ? b : n - a - b);
    }
    k -= cnt;
  }
  return -1;
}

__host__ __device__ constexpr double fact(int n) { return n <= 1 ? 1.0 : n * fact(n - 1); }

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
