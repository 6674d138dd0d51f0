// Tabulated cross-level pairs (two leaf cells one level apart; see kernels_boundary.cu):
// the per-slice body shared by k_cross_cells and the cross items of the persistent
// interaction kernel, so that both compute the same sums in the same order.
#pragma once
#include "kernels.h"

namespace octo {
namespace cross {

__device__ __forceinline__ double flip_sign(double x, int64_t bit) {
  return __longlong_as_double(__double_as_longlong(x) ^ (bit << 63));
}

// The kernel table (n_rows x 4 doubles) into shared memory, by the whole block.
__device__ __forceinline__ void stage_table(const CrossCells& xc, double2* tab2) {
  const double2* __restrict__ gt = reinterpret_cast<const double2*>(xc.table);
  for (int i = threadIdx.x; i < 2 * xc.n_rows; i += blockDim.x) tab2[i] = gt[i];
}

// Unscaled sums (S0 = sum m k0, S1..S3 = sum +-m k1..k3) of the target of lane
// `lane` in slice s; all 32 lanes of the warp call it together.
__device__ __forceinline__ void slice_sums(const CrossCells& xc, const double2* tab2, const double* __restrict__ mp,
                                           int s, int lane, double S[4]) {
  const int64_t o0 = xc.slice_off[s];
  const int64_t width = (xc.slice_off[s + 1] - o0) >> 5;  // a multiple of 4
  const int64_t* __restrict__ ent = xc.entries + o0 + lane;
  double S0 = 0.0, S1 = 0.0, S2 = 0.0, S3 = 0.0;
  int64_t en[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) en[u] = __ldcs(ent + 32 * u);
  for (int64_t k = 0; k < width; k += 4) {
    int64_t e[4];
    double m[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) e[u] = en[u];
    if (k + 4 < width) {  // next group's entries, in flight during this group
#pragma unroll
      for (int u = 0; u < 4; ++u) en[u] = __ldcs(ent + 32 * (k + 4 + u));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) m[u] = __ldg(mp + (e[u] >> 20));
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int row = (int)(e[u] & 0xffff);
      const double2 a = tab2[2 * row], b = tab2[2 * row + 1];
      S0 = fma(m[u], a.x, S0);
      S1 = fma(flip_sign(m[u], (e[u] >> 16) & 1), a.y, S1);
      S2 = fma(flip_sign(m[u], (e[u] >> 17) & 1), b.x, S2);
      S3 = fma(flip_sign(m[u], (e[u] >> 18) & 1), b.y, S3);
    }
  }
  S[0] = S0, S[1] = S1, S[2] = S2, S[3] = S3;
}

// Adds the sums of slot `slot` (= slice * 32 + lane) to its target's local
// expansion (phi = L0: -S0 / h; L1: +S1..S3 / h^2); padding slots have no target.
__device__ __forceinline__ void apply(const DevTree& t, const CrossCells& xc, int64_t slot, const double S[4],
                                      double* __restrict__ loc) {
  const int64_t tg = xc.targets[slot];
  if (tg < 0) return;
  const int64_t NC = t.NC;
  const double ih = 1.0 / t.h[t.level[tg >> 9]], ih2 = ih * ih;
  loc[G_L0 * NC + tg] -= S[0] * ih;
  loc[(G_L1 + 0) * NC + tg] += S[1] * ih2;
  loc[(G_L1 + 1) * NC + tg] += S[2] * ih2;
  loc[(G_L1 + 2) * NC + tg] += S[3] * ih2;
}

}  // namespace cross
}  // namespace octo
