// Cross-level pairs: a leaf cell and a cell of a finer refined region (both
// directions are listed).
//
// k_cross_cells: pairs of two leaf cells one level apart.  A leaf cell's multipole
// is a point mass at the cell centre, so M2L and P2P of such a pair are the same
// exact term, and the centre offset takes few values (odd multiples of half the
// finer cell width): the kernel reads the offset's row of a small table (shared
// memory) and does four float64 fused multiply-adds per pair.  One thread per
// target cell, targets in SELL-32 slices (a warp's 32 targets have similar partner
// counts; entry k of the 32 lanes is one coalesced 256-byte load); a persistent
// grid of warps claims slices, widest first, from a counter reset before every
// launch.  Each target is owned by one thread, so the result is deterministic.
//
// k_cross_w (everything else: deeper level differences, refined cells): one warp
// per target cell, lanes striding over its partners, a fixed butterfly reduction at
// the end (deterministic).  M2L partners come first in each list, then P2P partners
// (exact point-mass interaction, always float64).  Mixed precision runs the M2L part
// in float32 with compensated sums, operands scaled to the target's cell width.
#include "cross.cuh"

namespace octo {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kCrossCellsThreads = 256;
using cross::flip_sign;

__global__ void __launch_bounds__(kCrossCellsThreads) k_cross_cells(DevTree t, CrossCells xc,
                                                                    const double* __restrict__ mp,
                                                                    double* __restrict__ loc) {
  extern __shared__ double2 tab2[];  // n_rows x 4 doubles
  cross::stage_table(xc, tab2);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (;;) {
    // the next slice, claimed by the warp (slices are sorted widest first)
    int s = 0;
    if (lane == 0) s = atomicAdd(xc.counter, 1);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (s >= xc.n_slices) return;
    double S[4];
    cross::slice_sums(xc, tab2, mp, s, lane, S);
    cross::apply(t, xc, (int64_t)s * 32 + lane, S, loc);
  }
}

// Second half of the cross items of the persistent interaction kernel: the sums
// they left per slot (xcf [4][n_slices * 32]) into the targets' local expansions.
__global__ void k_cross_apply(DevTree t, CrossCells xc, const double* __restrict__ xcf, double* __restrict__ loc) {
  const int64_t n_slots = (int64_t)xc.n_slices * 32;
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= n_slots) return;
  const double S[4] = {xcf[slot], xcf[n_slots + slot], xcf[2 * n_slots + slot], xcf[3 * n_slots + slot]};
  cross::apply(t, xc, slot, S, loc);
}

// Adjoint of k_cross_cells (gather form).  Both directions of every pair are in
// the list, so the partners Y of list target X are the cells X was a source for.
// With fixed leaf centres only X's mass matters:
//   d S / d m_X = sum_Y [ -Lb0_Y / |R| + Lb1_Y . (x_Y - x_X) / |R|^3 ],
// and in the table's units (v = c_X - c_Y, row of the entry X <- Y, h = h_X)
//   1 / |R| = row0 / h,   (x_Y - x_X)_k / |R|^3 = -sign(v_k) row_k / h^2.
__global__ void __launch_bounds__(kCrossCellsThreads) k_cross_cells_adjoint(DevTree t, CrossCells xc,
                                                                            const double* __restrict__ locb,
                                                                            double* __restrict__ mpb) {
  extern __shared__ double2 tab2[];
  const double2* __restrict__ gt = reinterpret_cast<const double2*>(xc.table);
  for (int i = threadIdx.x; i < 2 * xc.n_rows; i += blockDim.x) tab2[i] = gt[i];
  __syncthreads();
  const int64_t NC = t.NC;
  const int lane = threadIdx.x & 31;
  for (;;) {
    int s = 0;
    if (lane == 0) s = atomicAdd(xc.counter, 1);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (s >= xc.n_slices) return;
    const int64_t o0 = xc.slice_off[s];
    const int64_t width = (xc.slice_off[s + 1] - o0) >> 5;
    const int64_t* __restrict__ ent = xc.entries + o0 + lane;
    double S0 = 0.0, S1 = 0.0;
    for (int64_t k = 0; k < width; k += 2) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int64_t e = __ldcs(ent + 32 * (k + u));
        const int64_t y = e >> 20;
        const int row = (int)(e & 0xffff);
        const double2 a = tab2[2 * row], b = tab2[2 * row + 1];
        const double b0 = __ldg(locb + G_L0 * NC + y);
        const double bx = __ldg(locb + (G_L1 + 0) * NC + y), by = __ldg(locb + (G_L1 + 1) * NC + y),
                     bz = __ldg(locb + (G_L1 + 2) * NC + y);
        S0 = fma(b0, a.x, S0);
        S1 = fma(flip_sign(bx, (e >> 16) & 1), a.y, S1);
        S1 = fma(flip_sign(by, (e >> 17) & 1), b.x, S1);
        S1 = fma(flip_sign(bz, (e >> 18) & 1), b.y, S1);
      }
    }
    const int64_t X = xc.targets[(int64_t)s * 32 + lane];
    if (X >= 0) {
      const double ih = 1.0 / t.h[t.level[X >> 9]];
      mpb[X] -= S0 * ih + S1 * ih * ih;
    }
  }
}

// C64 (mixed only): the correction of the far pairs in float64 from the float64
// multipoles, summed in float64 (measurement variant).
template <bool FULL, bool MIXED, bool C64 = false>
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
    DgAcc d64 = {{0.0, 0.0, 0.0}};
    for (int64_t e = e0 + lane; e < em; e += 32) {
      const int64_t src = xl.sources[e];
      const float R0 = (float)((XA0 - mp[(F_X + 0) * NC + src]) * ih);
      const float R1 = (float)((XA1 - mp[(F_X + 1) * NC + src]) * ih);
      const float R2 = (float)((XA2 - mp[(F_X + 2) * NC + src]) * ih);
      float Q[6], O[10];
      for (int k = 0; k < 6; ++k) Q[k] = (float)(mp[(F_Q + k) * NC + src] * ih2);
      for (int k = 0; k < 10; ++k) O[k] = (float)(mp[(F_O + k) * NC + src] * ih3);
      const float rinv = rsqrt_f32(fmaf(R0, R0, fmaf(R1, R1, R2 * R2)));
      m2l_pair<FULL, FULL, float, Acc<KF>, !C64>(R0, R1, R2, (float)mp[src], Q, O, Oh32, tOh32, rinv, acc);
      if constexpr (C64) {
        const double S0 = XA0 - mp[(F_X + 0) * NC + src], S1 = XA1 - mp[(F_X + 1) * NC + src],
                     S2 = XA2 - mp[(F_X + 2) * NC + src];
        double O64[10];
        for (int k = 0; k < 10; ++k) O64[k] = mp[(F_O + k) * NC + src];
        corr_pair_f64<FULL>(S0, S1, S2, mp[src], O64, Oh, tOh, rsqrt_f64(fma(S0, S0, fma(S1, S1, S2 * S2))), d64);
      }
    }
    const double ih4 = ih2 * ih2;
    d.L0 = acc.L0.value() * ih;
    for (int k = 0; k < 3; ++k) {
      d.L1[k] = acc.L1[k].value() * ih2;
      d.dg[k] = C64 ? d64.dg[k] : acc.dg[k].value() * ih2;
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

cudaError_t cross_cells_blocks_per_sm(const CrossCells& xc, int* blocks) {
  const size_t smem = sizeof(double) * 4 * (size_t)xc.n_rows;
  cudaError_t e = cudaSuccess;
  if (smem > 48 * 1024) e = cudaFuncSetAttribute(k_cross_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_cross_cells, kCrossCellsThreads, smem);
  return e;
}

cudaError_t launch_cross_cells(const DevTree& t, const CrossCells& xc, const double* mp, double* loc, int grid,
                               cudaStream_t s) {
  if (xc.n_slices == 0) return cudaSuccess;
  const size_t smem = sizeof(double) * 4 * (size_t)xc.n_rows;
  cudaError_t e = cudaMemsetAsync(xc.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_cross_cells<<<grid, kCrossCellsThreads, smem, s>>>(t, xc, mp, loc);
  return cudaGetLastError();
}

cudaError_t launch_cross_apply(const DevTree& t, const CrossCells& xc, const double* xcf, double* loc,
                               cudaStream_t s) {
  if (xc.n_slices == 0) return cudaSuccess;
  const int64_t n_slots = (int64_t)xc.n_slices * 32;
  k_cross_apply<<<(unsigned)((n_slots + 255) / 256), 256, 0, s>>>(t, xc, xcf, loc);
  return cudaGetLastError();
}

cudaError_t launch_cross_cells_adjoint(const DevTree& t, const CrossCells& xc, const double* locb, double* mpb,
                                       int grid, cudaStream_t s) {
  if (xc.n_slices == 0) return cudaSuccess;
  const size_t smem = sizeof(double) * 4 * (size_t)xc.n_rows;
  cudaError_t e = cudaFuncSetAttribute(k_cross_cells_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaMemsetAsync(xc.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_cross_cells_adjoint<<<grid, kCrossCellsThreads, smem, s>>>(t, xc, locb, mpb);
  return cudaGetLastError();
}

cudaError_t launch_cross_list(const DevTree& t, const CrossList& xl, bool full, const double* mp, double* loc,
                              bool mixed, cudaStream_t s, bool corr64) {
  if (xl.n_targets == 0) return cudaSuccess;
  const int blocks = (int)(((int64_t)xl.n_targets * 32 + 127) / 128);
  if (mixed && corr64) {
    if (full)
      k_cross_w<true, true, true><<<blocks, 128, 0, s>>>(t, xl, mp, loc);
    else
      k_cross_w<false, true, true><<<blocks, 128, 0, s>>>(t, xl, mp, loc);
  } else if (full) {
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
