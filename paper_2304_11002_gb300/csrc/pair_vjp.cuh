// Reverse mode of the one-pair M2L expression m2l_pair (device.cuh), used by the
// adjoint of the float64 solve.  Kept apart from the forward's header: the forward
// kernels do not include it.
#pragma once
#include <type_traits>

#include "device.cuh"

namespace octo {

// Reverse mode of m2l_pair (vector-Jacobian product of one pair), statement by
// statement in the opposite order.  Given the adjoints of the target's local
// expansion as stored (Lb: L0, L1(3), L2(6), L3(10), dg(3); the deferred Kronecker
// parts W, V of acc_finish are folded in here), it returns dS/dR (R = X_T - X_S, the
// rinv dependence on R included) and, as requested, the source moments' adjoints
// (m, Q, O) and the adjoint of the target's Oh = O_T / m_T.  Float64 only.
template <typename T>
struct PairVJPT {
  T R[3], m, Q[6], O[10], Oh[10];
};
using PairVJP = PairVJPT<double>;

// T = double on the device; the host also instantiates it with an operation-counting
// scalar (the adjoint's algorithmic flops).
template <typename T>
struct NoDeduce {
  using type = T;
};

template <bool FULL, bool TOCT, bool WANT_SRC, bool WANT_OH, typename T = double>
__host__ __device__ __forceinline__ void m2l_pair_vjp(const T R0, const T R1, const T R2, const T m,
                                                      const typename NoDeduce<T>::type* Q,
                                                      const typename NoDeduce<T>::type* O,
                                                      const typename NoDeduce<T>::type* Oh,
                                                      const typename NoDeduce<T>::type* Lb, PairVJPT<T>& out) {
  // ---- forward intermediates
  T rinv;
#ifdef __CUDA_ARCH__
  if constexpr (std::is_same<T, double>::value)
    rinv = rsqrt_f64(fma(R0, R0, fma(R1, R1, R2 * R2)));  // as the forward kernels
  else
#endif
    rinv = T(1.0) / sqrt(R0 * R0 + R1 * R1 + R2 * R2);
  const T ir2 = rinv * rinv;
  const T f0 = rinv, f1 = -rinv * ir2, f2 = -3.0 * f1 * ir2, f3 = -5.0 * f2 * ir2, f4 = -7.0 * f3 * ir2;
  const T xx = R0 * R0, xy = R0 * R1, xz = R0 * R2, yy = R1 * R1, yz = R1 * R2, zz = R2 * R2;
  const T xy2 = xy + xy, xz2 = xz + xz, yz2 = yz + yz;
  const T QR0 = Q[0] * R0 + Q[1] * R1 + Q[2] * R2;
  const T QR1 = Q[1] * R0 + Q[3] * R1 + Q[4] * R2;
  const T QR2 = Q[2] * R0 + Q[4] * R1 + Q[5] * R2;
  const T RQR = QR0 * R0 + QR1 * R1 + QR2 * R2;
  const T trQ = Q[0] + Q[3] + Q[5];
  const T u0 = O[0] * xx + O[1] * xy2 + O[2] * xz2 + O[3] * yy + O[4] * yz2 + O[5] * zz;
  const T u1 = O[1] * xx + O[3] * xy2 + O[4] * xz2 + O[6] * yy + O[7] * yz2 + O[8] * zz;
  const T u2 = O[2] * xx + O[4] * xy2 + O[5] * xz2 + O[7] * yy + O[8] * yz2 + O[9] * zz;
  const T sB = u0 * R0 + u1 * R1 + u2 * R2;
  const T t0 = O[0] + O[3] + O[5], t1 = O[1] + O[6] + O[8], t2 = O[2] + O[7] + O[9];
  const T tauB = t0 * R0 + t1 * R1 + t2 * R2;
  const T c1 = m * f1 + 0.5 * (f3 * RQR + f2 * trQ);
  T uA0 = 0, uA1 = 0, uA2 = 0, tO0 = 0, tO1 = 0, tO2 = 0, sA = 0, tauA = 0;
  if constexpr (TOCT) {
    uA0 = Oh[0] * xx + Oh[1] * xy2 + Oh[2] * xz2 + Oh[3] * yy + Oh[4] * yz2 + Oh[5] * zz;
    uA1 = Oh[1] * xx + Oh[3] * xy2 + Oh[4] * xz2 + Oh[6] * yy + Oh[7] * yz2 + Oh[8] * zz;
    uA2 = Oh[2] * xx + Oh[4] * xy2 + Oh[5] * xz2 + Oh[7] * yy + Oh[8] * yz2 + Oh[9] * zz;
    tO0 = Oh[0] + Oh[3] + Oh[5], tO1 = Oh[1] + Oh[6] + Oh[8], tO2 = Oh[2] + Oh[7] + Oh[9];
    sA = uA0 * R0 + uA1 * R1 + uA2 * R2;
    tauA = tO0 * R0 + tO1 * R1 + tO2 * R2;
  }
  const T cS = TOCT ? m * sA - sB : -sB;
  const T cT = TOCT ? m * tauA - tauB : -tauB;
  const T v0 = TOCT ? m * uA0 - u0 : -u0, v1 = TOCT ? m * uA1 - u1 : -u1, v2 = TOCT ? m * uA2 - u2 : -u2;
  const T w0 = TOCT ? m * tO0 - t0 : -t0, w1 = TOCT ? m * tO1 - t1 : -t1, w2 = TOCT ? m * tO2 - t2 : -t2;
  const T kR = f4 * cS * (1.0 / 6.0) + 0.5 * f3 * cT;
  // ---- adjoints of the outputs
  const T* dgb = Lb + 20;
  T Rb0 = 0, Rb1 = 0, Rb2 = 0, mb = 0;
  T f0b = 0, f1b = 0, f2b = 0, f3b = 0, f4b = 0;
  T xxb = 0, xyb = 0, xzb = 0, yyb = 0, yzb = 0, zzb = 0, xy2b = 0, xz2b = 0, yz2b = 0;
  // dg_i += kR R_i + k3 v_i + k2 w_i,  k3 = f3 / 2, k2 = f2 / 2
  const T kRb = dgb[0] * R0 + dgb[1] * R1 + dgb[2] * R2;
  Rb0 += dgb[0] * kR, Rb1 += dgb[1] * kR, Rb2 += dgb[2] * kR;
  f3b += 0.5 * (dgb[0] * v0 + dgb[1] * v1 + dgb[2] * v2);
  f2b += 0.5 * (dgb[0] * w0 + dgb[1] * w1 + dgb[2] * w2);
  const T vb0 = 0.5 * f3 * dgb[0], vb1 = 0.5 * f3 * dgb[1], vb2 = 0.5 * f3 * dgb[2];
  const T wb0 = 0.5 * f2 * dgb[0], wb1 = 0.5 * f2 * dgb[1], wb2 = 0.5 * f2 * dgb[2];
  // kR = f4 cS / 6 + f3 cT / 2
  f4b += kRb * cS * (1.0 / 6.0);
  f3b += 0.5 * kRb * cT;
  const T cSb = kRb * f4 * (1.0 / 6.0), cTb = 0.5 * kRb * f3;
  // cS, cT, v, w  (source part: -sB, -tauB, -u, -t; target part with m)
  T sBb = -cSb, tauBb = -cTb, ub0 = -vb0, ub1 = -vb1, ub2 = -vb2, tb0 = -wb0, tb1 = -wb1, tb2 = -wb2;
  if constexpr (TOCT) {
    mb += cSb * sA + cTb * tauA + vb0 * uA0 + vb1 * uA1 + vb2 * uA2 + wb0 * tO0 + wb1 * tO1 + wb2 * tO2;
    const T sAb = cSb * m, tauAb = cTb * m;
    const T uAb0 = vb0 * m + sAb * R0, uAb1 = vb1 * m + sAb * R1, uAb2 = vb2 * m + sAb * R2;
    const T tOb0 = wb0 * m + tauAb * R0, tOb1 = wb1 * m + tauAb * R1, tOb2 = wb2 * m + tauAb * R2;
    Rb0 += sAb * uA0 + tauAb * tO0, Rb1 += sAb * uA1 + tauAb * tO1, Rb2 += sAb * uA2 + tauAb * tO2;
    xxb += uAb0 * Oh[0] + uAb1 * Oh[1] + uAb2 * Oh[2];
    xy2b += uAb0 * Oh[1] + uAb1 * Oh[3] + uAb2 * Oh[4];
    xz2b += uAb0 * Oh[2] + uAb1 * Oh[4] + uAb2 * Oh[5];
    yyb += uAb0 * Oh[3] + uAb1 * Oh[6] + uAb2 * Oh[7];
    yz2b += uAb0 * Oh[4] + uAb1 * Oh[7] + uAb2 * Oh[8];
    zzb += uAb0 * Oh[5] + uAb1 * Oh[8] + uAb2 * Oh[9];
    if constexpr (WANT_OH) {
      out.Oh[0] = uAb0 * xx + tOb0;
      out.Oh[1] = uAb0 * xy2 + uAb1 * xx + tOb1;
      out.Oh[2] = uAb0 * xz2 + uAb2 * xx + tOb2;
      out.Oh[3] = uAb0 * yy + uAb1 * xy2 + tOb0;
      out.Oh[4] = uAb0 * yz2 + uAb1 * xz2 + uAb2 * xy2;
      out.Oh[5] = uAb0 * zz + uAb2 * xz2 + tOb0;
      out.Oh[6] = uAb1 * yy + tOb1;
      out.Oh[7] = uAb1 * yz2 + uAb2 * yy + tOb2;
      out.Oh[8] = uAb1 * zz + uAb2 * yz2 + tOb1;
      out.Oh[9] = uAb2 * zz + tOb2;
    }
  }
  if constexpr (FULL) {
    // deferred Kronecker parts (acc_finish): L2 diag -= W, L3 -= V terms
    const T Wb = -(Lb[4] + Lb[7] + Lb[9]);
    const T Vb0 = -(3.0 * Lb[10] + Lb[13] + Lb[15]);
    const T Vb1 = -(Lb[11] + 3.0 * Lb[16] + Lb[18]);
    const T Vb2 = -(Lb[12] + Lb[17] + 3.0 * Lb[19]);
    const T mf2 = m * f2, mf3 = m * f3;
    const T g0 = mf3 * R0, g1 = mf3 * R1, g2 = mf3 * R2;
    // V_i += mf2 R_i
    T mf2b = Vb0 * R0 + Vb1 * R1 + Vb2 * R2;
    Rb0 += Vb0 * mf2, Rb1 += Vb1 * mf2, Rb2 += Vb2 * mf2;
    // L3 -= g (x) RR
    const T* L3b = Lb + 10;
    const T gb0 = -(L3b[0] * xx + L3b[1] * xy + L3b[2] * xz + L3b[3] * yy + L3b[4] * yz + L3b[5] * zz);
    const T gb1 = -(L3b[6] * yy + L3b[7] * yz + L3b[8] * zz);
    const T gb2 = -(L3b[9] * zz);
    xxb -= L3b[0] * g0;
    xyb -= L3b[1] * g0;
    xzb -= L3b[2] * g0;
    yyb -= L3b[3] * g0 + L3b[6] * g1;
    yzb -= L3b[4] * g0 + L3b[7] * g1;
    zzb -= L3b[5] * g0 + L3b[8] * g1 + L3b[9] * g2;
    const T mf3b = gb0 * R0 + gb1 * R1 + gb2 * R2;
    Rb0 += gb0 * mf3, Rb1 += gb1 * mf3, Rb2 += gb2 * mf3;
    mb += mf3b * f3;
    f3b += mf3b * m;
    // W += m f1
    mb += Wb * f1;
    f1b += Wb * m;
    // L2 -= mf2 RR
    const T* L2b = Lb + 4;
    mf2b -= L2b[0] * xx + L2b[1] * xy + L2b[2] * xz + L2b[3] * yy + L2b[4] * yz + L2b[5] * zz;
    xxb -= L2b[0] * mf2;
    xyb -= L2b[1] * mf2;
    xzb -= L2b[2] * mf2;
    yyb -= L2b[3] * mf2;
    yzb -= L2b[4] * mf2;
    zzb -= L2b[5] * mf2;
    mb += mf2b * f2;
    f2b += mf2b * m;
  }
  // L1_i -= c1 R_i + f2 QR_i
  const T c1b = -(Lb[1] * R0 + Lb[2] * R1 + Lb[3] * R2);
  Rb0 -= Lb[1] * c1, Rb1 -= Lb[2] * c1, Rb2 -= Lb[3] * c1;
  f2b -= Lb[1] * QR0 + Lb[2] * QR1 + Lb[3] * QR2;
  T QRb0 = -Lb[1] * f2, QRb1 = -Lb[2] * f2, QRb2 = -Lb[3] * f2;
  // c1 = m f1 + (f3 RQR + f2 trQ) / 2
  mb += c1b * f1;
  f1b += c1b * m;
  f3b += 0.5 * c1b * RQR;
  f2b += 0.5 * c1b * trQ;
  T RQRb = 0.5 * c1b * f3, trQb = 0.5 * c1b * f2;
  // L0 -= m f0 + (f2 RQR + f1 trQ) / 2 - (f3 sB + 3 f2 tauB) / 6
  const T e = -Lb[0];
  mb += e * f0;
  f0b += e * m;
  f2b += 0.5 * e * RQR - 0.5 * e * tauB;
  RQRb += 0.5 * e * f2;
  f1b += 0.5 * e * trQ;
  trQb += 0.5 * e * f1;
  f3b -= e * sB * (1.0 / 6.0);
  sBb -= e * f3 * (1.0 / 6.0);
  tauBb -= 0.5 * e * f2;
  // tauB = t . R,  sB = u . R
  tb0 += tauBb * R0, tb1 += tauBb * R1, tb2 += tauBb * R2;
  Rb0 += tauBb * t0 + sBb * u0, Rb1 += tauBb * t1 + sBb * u1, Rb2 += tauBb * t2 + sBb * u2;
  ub0 += sBb * R0, ub1 += sBb * R1, ub2 += sBb * R2;
  // u = O : RR (monomial adjoints; source octupole adjoints below)
  xxb += ub0 * O[0] + ub1 * O[1] + ub2 * O[2];
  xy2b += ub0 * O[1] + ub1 * O[3] + ub2 * O[4];
  xz2b += ub0 * O[2] + ub1 * O[4] + ub2 * O[5];
  yyb += ub0 * O[3] + ub1 * O[6] + ub2 * O[7];
  yz2b += ub0 * O[4] + ub1 * O[7] + ub2 * O[8];
  zzb += ub0 * O[5] + ub1 * O[8] + ub2 * O[9];
  // RQR = QR . R,  QR = Q R
  QRb0 += RQRb * R0, QRb1 += RQRb * R1, QRb2 += RQRb * R2;
  Rb0 += RQRb * QR0 + QRb0 * Q[0] + QRb1 * Q[1] + QRb2 * Q[2];
  Rb1 += RQRb * QR1 + QRb0 * Q[1] + QRb1 * Q[3] + QRb2 * Q[4];
  Rb2 += RQRb * QR2 + QRb0 * Q[2] + QRb1 * Q[4] + QRb2 * Q[5];
  if constexpr (WANT_SRC) {
    out.m = mb;
    out.Q[0] = QRb0 * R0 + trQb;
    out.Q[1] = QRb0 * R1 + QRb1 * R0;
    out.Q[2] = QRb0 * R2 + QRb2 * R0;
    out.Q[3] = QRb1 * R1 + trQb;
    out.Q[4] = QRb1 * R2 + QRb2 * R1;
    out.Q[5] = QRb2 * R2 + trQb;
    out.O[0] = ub0 * xx + tb0;
    out.O[1] = ub0 * xy2 + ub1 * xx + tb1;
    out.O[2] = ub0 * xz2 + ub2 * xx + tb2;
    out.O[3] = ub0 * yy + ub1 * xy2 + tb0;
    out.O[4] = ub0 * yz2 + ub1 * xz2 + ub2 * xy2;
    out.O[5] = ub0 * zz + ub2 * xz2 + tb0;
    out.O[6] = ub1 * yy + tb1;
    out.O[7] = ub1 * yz2 + ub2 * yy + tb2;
    out.O[8] = ub1 * zz + ub2 * yz2 + tb1;
    out.O[9] = ub2 * zz + tb2;
  }
  // monomials and doubled cross terms
  xyb += 2.0 * xy2b, xzb += 2.0 * xz2b, yzb += 2.0 * yz2b;
  Rb0 += 2.0 * R0 * xxb + R1 * xyb + R2 * xzb;
  Rb1 += R0 * xyb + 2.0 * R1 * yyb + R2 * yzb;
  Rb2 += R0 * xzb + R1 * yzb + 2.0 * R2 * zzb;
  // radial factors: f4 = -7 f3 ir2, f3 = -5 f2 ir2, f2 = -3 f1 ir2, f1 = -rinv ir2, f0 = rinv
  T ir2b = -7.0 * f4b * f3;
  f3b += -7.0 * f4b * ir2;
  ir2b += -5.0 * f3b * f2;
  f2b += -5.0 * f3b * ir2;
  ir2b += -3.0 * f2b * f1;
  f1b += -3.0 * f2b * ir2;
  T rinvb = -f1b * ir2 + f0b;
  ir2b += -f1b * rinv;
  rinvb += 2.0 * rinv * ir2b;
  // rinv = (R . R)^(-1/2): d rinv / d R = -R rinv^3 = f1 R
  Rb0 += rinvb * f1 * R0, Rb1 += rinvb * f1 * R1, Rb2 += rinvb * f1 * R2;
  out.R[0] = Rb0, out.R[1] = Rb1, out.R[2] = Rb2;
}

}  // namespace octo
