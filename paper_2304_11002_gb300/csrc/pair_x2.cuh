// Two far-field pairs at once in Blackwell's paired float32 instructions (add, mul,
// fma and sub on .f32x2 operands, sm_100 family): every F2 holds the same quantity
// of two source cells, one per lane, and one instruction computes both lanes, each
// rounded as its scalar counterpart.  The interior M2L is bound by instruction
// issue, not by the float32 pipe, so computing two sources per instruction moves
// its bound from issue to the pipe.  Compiled as host code (no GPU) the same
// functions compute each lane with the scalar float32 operation (the same
// rounding), so that a host test can check the expression.
#pragma once
#include <cmath>

#include "device.cuh"

namespace octo {

struct F2 {
  float2 v;
};

__host__ __device__ __forceinline__ F2 f2(float x, float y) { return F2{make_float2(x, y)}; }
__host__ __device__ __forceinline__ F2 bc(float s) { return F2{make_float2(s, s)}; }
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return F2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(*reinterpret_cast<unsigned long long*>(&a.v)),
      "l"(*reinterpret_cast<unsigned long long*>(&b.v)));
  return F2{*reinterpret_cast<float2*>(&r)};
}
#else  // host code (and device code for architectures without the paired instructions)
__host__ __device__ inline F2 operator+(F2 a, F2 b) { return f2(a.v.x + b.v.x, a.v.y + b.v.y); }
__host__ __device__ inline F2 operator*(F2 a, F2 b) { return f2(a.v.x * b.v.x, a.v.y * b.v.y); }
__host__ __device__ inline F2 fma2(F2 a, F2 b, F2 c) { return f2(fmaf(a.v.x, b.v.x, c.v.x), fmaf(a.v.y, b.v.y, c.v.y)); }
__host__ __device__ inline F2 operator-(F2 a, F2 b) { return f2(a.v.x - b.v.x, a.v.y - b.v.y); }
#endif

// acc += x.x * y.x + x.y * y.y (two float32 FMAs); acc -= likewise; acc -= x.x + x.y.
__host__ __device__ __forceinline__ void acc_fma(float& acc, F2 x, F2 y) {
  acc = fmaf(x.v.x, y.v.x, acc);
  acc = fmaf(x.v.y, y.v.y, acc);
}
__host__ __device__ __forceinline__ void acc_fms(float& acc, F2 x, F2 y) {
  acc = fmaf(-x.v.x, y.v.x, acc);
  acc = fmaf(-x.v.y, y.v.y, acc);
}
__host__ __device__ __forceinline__ void acc_sub(float& acc, F2 x) {
  acc -= x.v.x;
  acc -= x.v.y;
}

// 1/sqrt(x) per lane: the hardware estimate (host: 1 / sqrt) and one Newton step
// (rsqrt_f32).
__host__ __device__ __forceinline__ F2 rsqrt2(F2 x) {
#ifdef __CUDA_ARCH__
  const F2 y = f2(rsqrtf(x.v.x), rsqrtf(x.v.y));
#else
  const F2 y = f2(1.0f / std::sqrt(x.v.x), 1.0f / std::sqrt(x.v.y));
#endif
  const F2 e = fma2(bc(-1.0f) * x * y, y, bc(1.0f));
  return fma2(y * bc(0.5f), e, y);
}

// The M2L contribution of two sources (lanes of R, m, Q, O; R = X_A - X_B) to one
// target A, with the angular-momentum correction, summed into the scalar float32
// partials of `a` (both lanes): the same terms as m2l_pair followed by corr_pair
// (truncation n + k <= 3, paper Section IV-C; D^(n) through the radial factors
// f0 .. f4 with the Kronecker parts deferred to W and V).  INTERIOR: the target is
// an interior cell (L0 .. L3 and dg into Acc<float>; target octupole over mass Oh
// and its trace vector tOh); otherwise a leaf cell (L0, L1 and dg into
// LeafAcc<float>; no target octupole, Oh and tOh unused).  A lane whose m, Q and O
// are zero contributes exactly zero.
template <bool INTERIOR, typename A>
__host__ __device__ __forceinline__ void m2l_pair_x2(const F2 R0, const F2 R1, const F2 R2, const F2 m, const F2* Q,
                                            const F2* O, const float* Oh, const float* tOh, const F2 rinv, A& a) {
  const F2 ir2 = rinv * rinv;
  const F2 f0 = rinv;
  const F2 nf1 = rinv * ir2;                 // -f1
  const F2 h2 = bc(1.5f) * nf1 * ir2;        // f2 / 2  (f2 = -3 f1 / r^2)
  const F2 h3 = bc(-5.0f) * h2 * ir2;        // f3 / 2  (f3 = -5 f2 / r^2)
  const F2 s4 = bc(-7.0f / 3.0f) * h3 * ir2;  // f4 / 6  (f4 = -7 f3 / r^2)
  const F2 f2v = h2 + h2;
  const F2 xx = R0 * R0, xy = R0 * R1, xz = R0 * R2, yy = R1 * R1, yz = R1 * R2, zz = R2 * R2;
  const F2 xy2 = xy + xy, xz2 = xz + xz, yz2 = yz + yz;
  // source quadrupole: Q.R, R.Q.R, trace
  const F2 QR0 = fma2(Q[0], R0, fma2(Q[1], R1, Q[2] * R2));
  const F2 QR1 = fma2(Q[1], R0, fma2(Q[3], R1, Q[4] * R2));
  const F2 QR2 = fma2(Q[2], R0, fma2(Q[4], R1, Q[5] * R2));
  const F2 RQR = fma2(QR0, R0, fma2(QR1, R1, QR2 * R2));
  const F2 trQ = Q[0] + Q[3] + Q[5];
  // source octupole: u = O.RR, sB = O:RRR, trace vector t, tauB = t.R
  const F2 u0 = fma2(O[0], xx, fma2(O[1], xy2, fma2(O[2], xz2, fma2(O[3], yy, fma2(O[4], yz2, O[5] * zz)))));
  const F2 u1 = fma2(O[1], xx, fma2(O[3], xy2, fma2(O[4], xz2, fma2(O[6], yy, fma2(O[7], yz2, O[8] * zz)))));
  const F2 u2 = fma2(O[2], xx, fma2(O[4], xy2, fma2(O[5], xz2, fma2(O[7], yy, fma2(O[8], yz2, O[9] * zz)))));
  const F2 sB = fma2(u0, R0, fma2(u1, R1, u2 * R2));
  const F2 t0 = O[0] + O[3] + O[5], t1 = O[1] + O[6] + O[8], t2 = O[2] + O[7] + O[9];
  const F2 tauB = fma2(t0, R0, fma2(t1, R1, t2 * R2));
  // L0 -= m f0 + (f2 R.Q.R + f1 trQ) / 2 - (f3 sB + 3 f2 tauB) / 6
  //     = m f0 + h2 (R.Q.R - tauB) - (nf1 trQ) / 2 - (h3 sB) / 3
  const F2 e0 = fma2(m, f0, fma2(h2, RQR - tauB, fma2(bc(-0.5f), nf1 * trQ, bc(-1.0f / 3.0f) * h3 * sB)));
  acc_sub(a.L0, e0);
  // L1 -= c1 R + f2 Q.R,  c1 = m f1 + (f3 R.Q.R + f2 trQ) / 2 = h3 R.Q.R + h2 trQ - m nf1
  const F2 c1 = fma2(h3, RQR, h2 * trQ) - m * nf1;
  acc_sub(a.L1[0], fma2(c1, R0, f2v * QR0));
  acc_sub(a.L1[1], fma2(c1, R1, f2v * QR1));
  acc_sub(a.L1[2], fma2(c1, R2, f2v * QR2));
  if constexpr (!INTERIOR) {
    // correction without a target octupole: dg -= (s4 sB + h3 tauB) R + h3 u + h2 t
    const F2 nkR = fma2(s4, sB, h3 * tauB);
    acc_sub(a.dg[0], fma2(nkR, R0, fma2(h3, u0, h2 * t0)));
    acc_sub(a.dg[1], fma2(nkR, R1, fma2(h3, u1, h2 * t1)));
    acc_sub(a.dg[2], fma2(nkR, R2, fma2(h3, u2, h2 * t2)));
  } else {
    // L2 -= m f2 RR (W: deferred -delta m f1),  L3 -= m f3 RRR (V: deferred m f2 R)
    const F2 mf2 = m * f2v, mf3 = (m + m) * h3;
    acc_fms(a.L2[0], mf2, xx);
    acc_fms(a.L2[1], mf2, xy);
    acc_fms(a.L2[2], mf2, xz);
    acc_fms(a.L2[3], mf2, yy);
    acc_fms(a.L2[4], mf2, yz);
    acc_fms(a.L2[5], mf2, zz);
    acc_fms(a.W, m, nf1);
    const F2 g0 = mf3 * R0, g1 = mf3 * R1, g2 = mf3 * R2;
    acc_fms(a.L3[0], g0, xx);
    acc_fms(a.L3[1], g0, xy);
    acc_fms(a.L3[2], g0, xz);
    acc_fms(a.L3[3], g0, yy);
    acc_fms(a.L3[4], g0, yz);
    acc_fms(a.L3[5], g0, zz);
    acc_fms(a.L3[6], g1, yy);
    acc_fms(a.L3[7], g1, yz);
    acc_fms(a.L3[8], g1, zz);
    acc_fms(a.L3[9], g2, zz);
    acc_fma(a.V[0], mf2, R0);
    acc_fma(a.V[1], mf2, R1);
    acc_fma(a.V[2], mf2, R2);
    // angular-momentum correction (corr_pair with a target octupole):
    //   dg += kR R + h3 v + h2 w,  kR = f4 cS / 6 + f3 cT / 2,
    //   v = m uA - u, w = m tOh - t, cS = m sA - sB, cT = m tauA - tauB,
    //   uA = Oh.RR, sA = uA.R, tauA = tOh.R
    const F2 uA0 = fma2(bc(Oh[0]), xx, fma2(bc(Oh[1]), xy2, fma2(bc(Oh[2]), xz2,
                   fma2(bc(Oh[3]), yy, fma2(bc(Oh[4]), yz2, bc(Oh[5]) * zz)))));
    const F2 uA1 = fma2(bc(Oh[1]), xx, fma2(bc(Oh[3]), xy2, fma2(bc(Oh[4]), xz2,
                   fma2(bc(Oh[6]), yy, fma2(bc(Oh[7]), yz2, bc(Oh[8]) * zz)))));
    const F2 uA2 = fma2(bc(Oh[2]), xx, fma2(bc(Oh[4]), xy2, fma2(bc(Oh[5]), xz2,
                   fma2(bc(Oh[7]), yy, fma2(bc(Oh[8]), yz2, bc(Oh[9]) * zz)))));
    const F2 sA = fma2(uA0, R0, fma2(uA1, R1, uA2 * R2));
    const F2 tauA = fma2(bc(tOh[0]), R0, fma2(bc(tOh[1]), R1, bc(tOh[2]) * R2));
    const F2 cS = m * sA - sB;
    const F2 cT = m * tauA - tauB;
    const F2 kR = fma2(s4, cS, h3 * cT);  // f4 cS / 6 + f3 cT / 2
    const F2 v0 = m * uA0 - u0, v1 = m * uA1 - u1, v2 = m * uA2 - u2;
    const F2 w0 = m * bc(tOh[0]) - t0, w1 = m * bc(tOh[1]) - t1, w2 = m * bc(tOh[2]) - t2;
    const F2 d0 = fma2(kR, R0, fma2(h3, v0, h2 * w0));
    const F2 d1 = fma2(kR, R1, fma2(h3, v1, h2 * w1));
    const F2 d2 = fma2(kR, R2, fma2(h3, v2, h2 * w2));
    a.dg[0] += d0.v.x;
    a.dg[0] += d0.v.y;
    a.dg[1] += d1.v.x;
    a.dg[1] += d1.v.y;
    a.dg[2] += d2.v.x;
    a.dg[2] += d2.v.y;
  }
}

}  // namespace octo
