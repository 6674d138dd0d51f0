// Cross-level pairs: a leaf cell and a cell of a finer refined region (both
// directions are listed).  One warp per target cell, lanes striding over its
// partners, a fixed butterfly reduction at the end (deterministic).  M2L partners
// come first in each list, then P2P partners (exact point-mass interaction, always
// float64).  Mixed precision runs the M2L part in float32 with compensated sums,
// operands scaled to the target's cell width.
#include "kernels.h"

namespace octo {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <bool FULL, bool MIXED>
__global__ void __launch_bounds__(128) k_cross_w(DevTree t, CrossList xl, const double* __restrict__ mp,
                                                 double* __restrict__ loc) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wid >= xl.n_targets) return;  // whole warp exits together
  const int64_t NC = t.NC;
  const int64_t tgt = xl.targets[wid];
  const int lvl = t.level[tgt / 512];
  const double h = t.h[lvl], ih = 1.0 / h, ih2 = ih * ih, ih3 = ih2 * ih;
  const double XA0 = mp[(F_X + 0) * NC + tgt], XA1 = mp[(F_X + 1) * NC + tgt], XA2 = mp[(F_X + 2) * NC + tgt];
  double Oh[10], tOh[3];
  if (FULL) {
    const double inv_m = 1.0 / mp[tgt];
    for (int k = 0; k < 10; ++k) Oh[k] = mp[(F_O + k) * NC + tgt] * inv_m;
    tOh[0] = Oh[0] + Oh[3] + Oh[5];
    tOh[1] = Oh[1] + Oh[6] + Oh[8];
    tOh[2] = Oh[2] + Oh[7] + Oh[9];
  }
  Acc<double> d;
  acc_zero(d);
  const int64_t e0 = xl.start[wid], em = xl.mid[wid], e1 = xl.start[wid + 1];
  if (MIXED) {
    // far partners in float32, operands in units of the target's cell width
    float Oh32[10], tOh32[3];
    for (int k = 0; k < 10; ++k) Oh32[k] = FULL ? (float)(Oh[k] * ih3) : 0.0f;
    for (int k = 0; k < 3; ++k) tOh32[k] = FULL ? (float)(tOh[k] * ih3) : 0.0f;
    Acc<KF> acc;
    acc_zero(acc);
    for (int64_t e = e0 + lane; e < em; e += 32) {
      const int64_t src = xl.sources[e];
      const float R0 = (float)((XA0 - mp[(F_X + 0) * NC + src]) * ih);
      const float R1 = (float)((XA1 - mp[(F_X + 1) * NC + src]) * ih);
      const float R2 = (float)((XA2 - mp[(F_X + 2) * NC + src]) * ih);
      float Q[6], O[10];
      for (int k = 0; k < 6; ++k) Q[k] = (float)(mp[(F_Q + k) * NC + src] * ih2);
      for (int k = 0; k < 10; ++k) O[k] = (float)(mp[(F_O + k) * NC + src] * ih3);
      const float rinv = rsqrt_f32(fmaf(R0, R0, fmaf(R1, R1, R2 * R2)));
      m2l_pair<FULL, FULL>(R0, R1, R2, (float)mp[src], Q, O, Oh32, tOh32, rinv, acc);
    }
    const double ih4 = ih2 * ih2;
    d.L0 = acc.L0.value() * ih;
    for (int k = 0; k < 3; ++k) {
      d.L1[k] = acc.L1[k].value() * ih2;
      d.dg[k] = acc.dg[k].value() * ih2;
      d.V[k] = acc.V[k].value() * ih4;
    }
    for (int k = 0; k < 6; ++k) d.L2[k] = acc.L2[k].value() * ih3;
    for (int k = 0; k < 10; ++k) d.L3[k] = acc.L3[k].value() * ih4;
    d.W = acc.W.value() * ih3;
  } else {
    for (int64_t e = e0 + lane; e < em; e += 32) {
      const int64_t src = xl.sources[e];
      const double R0 = XA0 - mp[(F_X + 0) * NC + src];
      const double R1 = XA1 - mp[(F_X + 1) * NC + src];
      const double R2 = XA2 - mp[(F_X + 2) * NC + src];
      double Q[6], O[10];
      for (int k = 0; k < 6; ++k) Q[k] = mp[(F_Q + k) * NC + src];
      for (int k = 0; k < 10; ++k) O[k] = mp[(F_O + k) * NC + src];
      const double rinv = rsqrt_f64(fma(R0, R0, fma(R1, R1, R2 * R2)));
      m2l_pair<FULL, FULL>(R0, R1, R2, mp[src], Q, O, Oh, tOh, rinv, d);
    }
  }
  // near partners: exact point masses (both cells are leaves), float64
  for (int64_t e = em + lane; e < e1; e += 32) {
    const int64_t src = xl.sources[e];
    const double R0 = XA0 - mp[(F_X + 0) * NC + src];
    const double R1 = XA1 - mp[(F_X + 1) * NC + src];
    const double R2 = XA2 - mp[(F_X + 2) * NC + src];
    const double rinv = rsqrt_f64(fma(R0, R0, fma(R1, R1, R2 * R2)));
    const double mr = mp[src] * rinv, mr3 = mr * rinv * rinv;
    d.L0 -= mr;
    d.L1[0] += mr3 * R0;
    d.L1[1] += mr3 * R1;
    d.L1[2] += mr3 * R2;
  }
  d.L0 = warp_sum(d.L0);
  for (int k = 0; k < 3; ++k) d.L1[k] = warp_sum(d.L1[k]), d.dg[k] = warp_sum(d.dg[k]);
  if (FULL) {
    for (int k = 0; k < 6; ++k) d.L2[k] = warp_sum(d.L2[k]);
    for (int k = 0; k < 10; ++k) d.L3[k] = warp_sum(d.L3[k]);
    for (int k = 0; k < 3; ++k) d.V[k] = warp_sum(d.V[k]);
    d.W = warp_sum(d.W);
  }
  if (lane == 0) {
    loc[G_L0 * NC + tgt] += d.L0;
    for (int k = 0; k < 3; ++k) loc[(G_L1 + k) * NC + tgt] += d.L1[k], loc[(G_DG + k) * NC + tgt] += d.dg[k];
    if (FULL) {
      acc_finish(d);
      for (int k = 0; k < 6; ++k) loc[(G_L2 + k) * NC + tgt] += d.L2[k];
      for (int k = 0; k < 10; ++k) loc[(G_L3 + k) * NC + tgt] += d.L3[k];
    }
  }
}

}  // namespace

cudaError_t launch_cross_list(const DevTree& t, const CrossList& xl, bool full, const double* mp, double* loc,
                              bool mixed, cudaStream_t s) {
  if (xl.n_targets == 0) return cudaSuccess;
  const int blocks = (int)(((int64_t)xl.n_targets * 32 + 127) / 128);
  if (full) {
    if (mixed)
      k_cross_w<true, true><<<blocks, 128, 0, s>>>(t, xl, mp, loc);
    else
      k_cross_w<true, false><<<blocks, 128, 0, s>>>(t, xl, mp, loc);
  } else {
    if (mixed)
      k_cross_w<false, true><<<blocks, 128, 0, s>>>(t, xl, mp, loc);
    else
      k_cross_w<false, false><<<blocks, 128, 0, s>>>(t, xl, mp, loc);
  }
  return cudaGetLastError();
}

}  // namespace octo
