// Device-side data layout and the per-pair arithmetic of the expansions.
//
// Layout in HBM (structure of arrays over all cells of all nodes; a cell's global
// index is dnode * 512 + local, local = a + 8 b + 64 c, nodes sorted by level):
//   mp   [20][NC]  m, X(3), M2 {xx,xy,xz,yy,yz,zz}, M3 {xxx,xxy,xxz,xyy,xyz,xzz,yyy,yyz,yzz,zzz}
//   loc  [23][NC]  L0, L1(3), L2(6), L3(10), dg(3)
// Leaf cells only ever use L0, L1 and dg (their expansion centre is the point
// itself), so their L2/L3 slots are never written.
#pragma once
#include <cstdint>

namespace octo {

constexpr int F_M = 0, F_X = 1, F_Q = 4, F_O = 10;          // multipole field offsets
constexpr int G_L0 = 0, G_L1 = 1, G_L2 = 4, G_L3 = 10, G_DG = 20;  // local-expansion offsets
constexpr int N_MP = 20, N_LOC = 23;

// Bits of the handle's device error word.  The adjoint's index checks use the low
// bits (see kernels_adjoint.cu); P2M sets kErrDensity for a density that is not
// finite and positive; kErrTimeout is set when a kernel's bounded wait for its own
// asynchronous copies ran out (the item's results are then incomplete).
constexpr int kErrDensity = 1 << 30;
constexpr int kErrTimeout = 1 << 29;

struct DevTree {
  int64_t NC;  // number of cells = n_nodes * 512
  int n_nodes;
  const int* level;
  const int* parent;
  const int* octant;
  const int* children;
  const int* nbr;      // [n][27]
  const int* leaf_id;  // leaf order index or -1
  const int* ijk;      // [n][3] node position within its level
  double origin[3];
  double h[16];        // cell width per level
  double h3[16];       // h^3 per level
};

// Float32 copy of the multipoles used by the mixed-precision far field, in units of
// the cell width h of the cell's level (so that float32 neither overflows nor
// underflows whatever the physical units): per cell the 20 values f = 0 .. 19
//   m, x = (X - c_node) / h (c_node = geometric centre of the node), Q / h^2, O / h^3
// (same field order as mp).  The two cells of an x-pair, (2X, b, c) and
// (2X + 1, b, c), share one record of ten float4 planes,
//   plane k = (f_2k(2X), f_2k(2X + 1), f_2k+1(2X), f_2k+1(2X + 1)),
//   mp32 float4 [n_nodes][10][256],
// so that one 16-byte load returns the same field of both cells as an aligned pair
// of registers: the operand layout of the paired float32 instructions with which
// the interior M2L takes two sources at once.  The 256 pair records of a node are in
// (b & 1, c & 1)-parity-major order (mp32_pair_slot), X fastest: the lanes of a
// parity-class warp hold consecutive (a >> 1, b >> 1, c >> 1), so at any stencil
// offset they read runs of consecutive 16-byte words of each plane, and the ten
// planes of a pair are one address plus constant offsets.
// Node centres of same-level neighbours differ by exactly 8 h per axis.
constexpr int kMp32Planes = 10;
constexpr int kMp32Pairs = 256;

__host__ __device__ __forceinline__ int mp32_pair_slot(int X, int b, int c) {
  return ((b & 1) + 2 * (c & 1)) * 64 + X + 4 * (b >> 1) + 16 * (c >> 1);
}

// Plane 0 of the record of cells (2X, b, c) and (2X + 1, b, c), 0 <= X < 4,
// 0 <= b, c < 8, of node `node`, as a float4 index.
__host__ __device__ __forceinline__ int64_t mp32_pair_base(int node, int X, int b, int c) {
  return (int64_t)node * (kMp32Planes * kMp32Pairs) + mp32_pair_slot(X, b, c);
}

// Float index of field f of local cell (a, b, c) of `node`.
__host__ __device__ __forceinline__ int64_t mp32_index(int node, int a, int b, int c, int f) {
  return 4 * (mp32_pair_base(node, a >> 1, b, c) + (int64_t)(f >> 1) * kMp32Pairs) + 2 * (f & 1) + (a & 1);
}

// Compensated float32 sum (Kahan): s holds the running sum, c the negative of the
// rounding error not yet added back; the exact sum is s - c to float32 working
// precision.
struct KF {
  float s, c;
  __host__ __device__ __forceinline__ KF& operator=(float v) {
    s = v;
    c = 0.0f;
    return *this;
  }
  __host__ __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __host__ __device__ __forceinline__ KF& operator+=(float x) {
    add(x);
    return *this;
  }
  __host__ __device__ __forceinline__ KF& operator-=(float x) {
    add(-x);
    return *this;
  }
  __host__ __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// 1/sqrt(x) in float64 for x > 0: a float32 hardware seed refined by one
// third-order Householder step (Newton iteration for x^-1/2 with the quadratic
// term of the binomial series): e = 1 - x y^2, y <- y (1 + e/2 + 3 e^2 / 8).
// The seed's relative error (~1e-7) cubes to below the float64 rounding unit.
__device__ __forceinline__ double rsqrt_f64(double x) {
  double y = (double)rsqrtf((float)x);
  double e = fma(-x * y, y, 1.0);
  double p = fma(e, 0.375, 0.5);
  return fma(y * e, p, y);
}

__device__ __forceinline__ float rsqrt_f32(float x) {
  float y = rsqrtf(x);
  // one Newton step to reach ~1 ulp (the hardware estimate is ~2 ulp)
  float e = fmaf(-x * y, y, 1.0f);
  return fmaf(y * 0.5f, e, y);
}

// Accumulators of one target cell.  L2/L3 carry only the R-polynomial parts; the
// Kronecker-delta parts are summed in W (L2) and V (L3) and added once at the end:
//   L2_ab = acc.L2_ab - delta_ab W,   W = sum m f1
//   L3_abc = acc.L3_abc - (delta_ab V_c + delta_ac V_b + delta_bc V_a),  V = sum m f2 R
template <typename T>
struct Acc {
  T L0, L1[3], L2[6], L3[10], dg[3], W, V[3];
};

template <typename A>
__host__ __device__ __forceinline__ void acc_zero(A& a) {
  a.L0 = 0;
  for (int i = 0; i < 3; ++i) a.L1[i] = 0, a.dg[i] = 0, a.V[i] = 0;
  for (int i = 0; i < 6; ++i) a.L2[i] = 0;
  for (int i = 0; i < 10; ++i) a.L3[i] = 0;
  a.W = 0;
}

// Angular-momentum correction of one far pair (target A, source B, R = X_A - X_B):
//   dg_A += (m_B O_A - m_A O_B):D4 / (6 m_A),
// written with Oh = O_A / m_A as ((m_B Oh - O_B):D4)/6 and, for a 3-tensor C,
//   (C:D4)_a = f4 R_a (C:RRR) + 3 f3 [(C.RR)_a + R_a (tC.R)] + 3 f2 tC_a,  tC_a = C_abb,
// from the source octupole's contractions with R (u = O_B.RR, sB = O_B:RRR, its
// trace vector t and tauB = t.R; the M2L terms use them too).  TOCT: the target
// has an octupole (interior cell); otherwise Oh = 0.
template <bool TOCT, typename T, typename A>
__host__ __device__ __forceinline__ void corr_pair(const T R0, const T R1, const T R2, const T m, const T xx,
                                                   const T xy2, const T xz2, const T yy, const T yz2, const T zz,
                                                   const T u0, const T u1, const T u2, const T sB, const T t0,
                                                   const T t1, const T t2, const T tauB, const T* Oh, const T* tOh,
                                                   const T f2, const T f3, const T f4, A& a) {
  T cS, cT, v0, v1, v2, w0, w1, w2;
  if constexpr (TOCT) {
    const T uA0 = Oh[0] * xx + Oh[1] * xy2 + Oh[2] * xz2 + Oh[3] * yy + Oh[4] * yz2 + Oh[5] * zz;
    const T uA1 = Oh[1] * xx + Oh[3] * xy2 + Oh[4] * xz2 + Oh[6] * yy + Oh[7] * yz2 + Oh[8] * zz;
    const T uA2 = Oh[2] * xx + Oh[4] * xy2 + Oh[5] * xz2 + Oh[7] * yy + Oh[8] * yz2 + Oh[9] * zz;
    const T sA = uA0 * R0 + uA1 * R1 + uA2 * R2;
    const T tauA = tOh[0] * R0 + tOh[1] * R1 + tOh[2] * R2;
    cS = m * sA - sB;
    cT = m * tauA - tauB;
    v0 = m * uA0 - u0;
    v1 = m * uA1 - u1;
    v2 = m * uA2 - u2;
    w0 = m * tOh[0] - t0;
    w1 = m * tOh[1] - t1;
    w2 = m * tOh[2] - t2;
  } else {
    cS = -sB;
    cT = -tauB;
    v0 = -u0;
    v1 = -u1;
    v2 = -u2;
    w0 = -t0;
    w1 = -t1;
    w2 = -t2;
  }
  const T kR = f4 * cS * (T)(1.0 / 6.0) + (T)0.5 * f3 * cT;
  const T k3 = (T)0.5 * f3, k2 = (T)0.5 * f2;
  a.dg[0] += kR * R0 + k3 * v0 + k2 * w0;
  a.dg[1] += kR * R1 + k3 * v1 + k2 * w1;
  a.dg[2] += kR * R2 + k3 * v2 + k2 * w2;
}

// One M2L contribution of source B (m, quadrupole Q, octupole O, all about its
// centre of mass) to target A, with R = X_A - X_B.  Truncation n + k <= 3:
//   L0  += -[ m D0 + Q:D2/2 - O:D3/6 ]
//   L1  += -[ m D1 + (Q:D3)/2 ]
//   L2  += -m D2,   L3 += -m D3
// with D^(n) = grad^n (1/|R|) written through the radial factors
// f0 = 1/r, f_{n+1} = -(2n+1) f_n / r^2:
//   D1 = f1 R, D2 = f2 RR + f1 I, D3 = f3 RRR + f2 (I R)_sym, D4 = f4 RRRR + f3 (I RR)_sym + f2 (I I)_sym,
// plus the angular-momentum correction (corr_pair) unless CORR is false (the
// caller then forms it separately, in float64).
// FULL: the target needs L2/L3 (interior cell).  TOCT: the target has an octupole.
template <bool FULL, bool TOCT, typename T, typename A, bool CORR = true>
__host__ __device__ __forceinline__ void m2l_pair(const T R0, const T R1, const T R2, const T m, const T* Q, const T* O,
                                                  const T* Oh, const T* tOh, T rinv, A& a) {
  const T ir2 = rinv * rinv;
  const T f0 = rinv;
  const T f1 = -rinv * ir2;
  const T f2 = (T)(-3.0) * f1 * ir2;
  const T f3 = (T)(-5.0) * f2 * ir2;
  const T f4 = (T)(-7.0) * f3 * ir2;
  const T xx = R0 * R0, xy = R0 * R1, xz = R0 * R2, yy = R1 * R1, yz = R1 * R2, zz = R2 * R2;
  const T xy2 = xy + xy, xz2 = xz + xz, yz2 = yz + yz;
  // quadrupole terms
  const T QR0 = Q[0] * R0 + Q[1] * R1 + Q[2] * R2;
  const T QR1 = Q[1] * R0 + Q[3] * R1 + Q[4] * R2;
  const T QR2 = Q[2] * R0 + Q[4] * R1 + Q[5] * R2;
  const T RQR = QR0 * R0 + QR1 * R1 + QR2 * R2;
  const T trQ = Q[0] + Q[3] + Q[5];
  // octupole terms: u = O.RR, s = O:RRR, t = trace vector, tau = t.R
  const T u0 = O[0] * xx + O[1] * xy2 + O[2] * xz2 + O[3] * yy + O[4] * yz2 + O[5] * zz;
  const T u1 = O[1] * xx + O[3] * xy2 + O[4] * xz2 + O[6] * yy + O[7] * yz2 + O[8] * zz;
  const T u2 = O[2] * xx + O[4] * xy2 + O[5] * xz2 + O[7] * yy + O[8] * yz2 + O[9] * zz;
  const T sB = u0 * R0 + u1 * R1 + u2 * R2;
  const T t0 = O[0] + O[3] + O[5], t1 = O[1] + O[6] + O[8], t2 = O[2] + O[7] + O[9];
  const T tauB = t0 * R0 + t1 * R1 + t2 * R2;
  // L0
  a.L0 -= m * f0 + (T)0.5 * (f2 * RQR + f1 * trQ) - (f3 * sB + (T)3.0 * f2 * tauB) * (T)(1.0 / 6.0);
  // L1
  const T c1 = m * f1 + (T)0.5 * (f3 * RQR + f2 * trQ);
  a.L1[0] -= c1 * R0 + f2 * QR0;
  a.L1[1] -= c1 * R1 + f2 * QR1;
  a.L1[2] -= c1 * R2 + f2 * QR2;
  if constexpr (FULL) {
    const T mf2 = m * f2;
    a.L2[0] -= mf2 * xx;
    a.L2[1] -= mf2 * xy;
    a.L2[2] -= mf2 * xz;
    a.L2[3] -= mf2 * yy;
    a.L2[4] -= mf2 * yz;
    a.L2[5] -= mf2 * zz;
    a.W += m * f1;
    const T mf3 = m * f3;
    const T g0 = mf3 * R0, g1 = mf3 * R1, g2 = mf3 * R2;
    a.L3[0] -= g0 * xx;
    a.L3[1] -= g0 * xy;
    a.L3[2] -= g0 * xz;
    a.L3[3] -= g0 * yy;
    a.L3[4] -= g0 * yz;
    a.L3[5] -= g0 * zz;
    a.L3[6] -= g1 * yy;
    a.L3[7] -= g1 * yz;
    a.L3[8] -= g1 * zz;
    a.L3[9] -= g2 * zz;
    a.V[0] += mf2 * R0;
    a.V[1] += mf2 * R1;
    a.V[2] += mf2 * R2;
  }
  if constexpr (CORR)
    corr_pair<TOCT>(R0, R1, R2, m, xx, xy2, xz2, yy, yz2, zz, u0, u1, u2, sB, t0, t1, t2, tauB, Oh, tOh, f2, f3, f4, a);
}

// Float64 accumulator of the correction alone (float64-correction variant of the
// mixed path).
struct DgAcc {
  double dg[3];
};

// The angular-momentum correction of one far pair on its own, in float64 from the
// float64 multipoles: R = X_A - X_B, source mass m and octupole O, target Oh = O_A /
// m_A and its trace vector tOh (TOCT), 1/|R| = rinv.
template <bool TOCT>
__host__ __device__ __forceinline__ void corr_pair_f64(const double R0, const double R1, const double R2,
                                                       const double m, const double* O, const double* Oh,
                                                       const double* tOh, const double rinv, DgAcc& a) {
  const double ir2 = rinv * rinv;
  const double f2 = 3.0 * rinv * ir2 * ir2;
  const double f3 = -5.0 * f2 * ir2;
  const double f4 = -7.0 * f3 * ir2;
  const double xx = R0 * R0, xy = R0 * R1, xz = R0 * R2, yy = R1 * R1, yz = R1 * R2, zz = R2 * R2;
  const double xy2 = xy + xy, xz2 = xz + xz, yz2 = yz + yz;
  const double u0 = O[0] * xx + O[1] * xy2 + O[2] * xz2 + O[3] * yy + O[4] * yz2 + O[5] * zz;
  const double u1 = O[1] * xx + O[3] * xy2 + O[4] * xz2 + O[6] * yy + O[7] * yz2 + O[8] * zz;
  const double u2 = O[2] * xx + O[4] * xy2 + O[5] * xz2 + O[7] * yy + O[8] * yz2 + O[9] * zz;
  const double sB = u0 * R0 + u1 * R1 + u2 * R2;
  const double t0 = O[0] + O[3] + O[5], t1 = O[1] + O[6] + O[8], t2 = O[2] + O[7] + O[9];
  const double tauB = t0 * R0 + t1 * R1 + t2 * R2;
  corr_pair<TOCT>(R0, R1, R2, m, xx, xy2, xz2, yy, yz2, zz, u0, u1, u2, sB, t0, t1, t2, tauB, Oh, tOh, f2, f3, f4, a);
}

// Adds the deferred Kronecker-delta parts into L2 / L3.
template <typename T>
__host__ __device__ __forceinline__ void acc_finish(Acc<T>& a) {
  a.L2[0] -= a.W;
  a.L2[3] -= a.W;
  a.L2[5] -= a.W;
  const T V0 = a.V[0], V1 = a.V[1], V2 = a.V[2];
  a.L3[0] -= (T)3.0 * V0;  // xxx
  a.L3[1] -= V1;           // xxy
  a.L3[2] -= V2;           // xxz
  a.L3[3] -= V0;           // xyy
  a.L3[5] -= V0;           // xzz
  a.L3[6] -= (T)3.0 * V1;  // yyy
  a.L3[7] -= V2;           // yyz
  a.L3[8] -= V1;           // yzz
  a.L3[9] -= (T)3.0 * V2;  // zzz
}

}  // namespace octo
