// Work items of the same-level interaction phase, as device functions run by a
// block of 256 threads (4 parity classes of one node: half = 0 -> cells with even
// z, half = 1 -> odd z).  They are called both by the per-kind kernels and by the
// persistent work-queue kernel (kernels_interact.cu).
//
//  interior item: all same-level M2L into the cells of a refined node (the
//                 parity stencil, sources in the 26 neighbours), results stored;
//  leaf item:     the leaf-leaf pairs of a leaf node as a convolution with the
//                 tabulated point-mass kernel (far stencil + near offsets, mass
//                 halo in shared memory), plus the M2L from refined same-level
//                 neighbours (refinement boundary), results stored.
#pragma once
#include <type_traits>

#include "halo.h"
#include "kernels.h"
#include "pair_x2.cuh"
#include "tma.cuh"

namespace octo {
namespace items {

constexpr int kThreads = 256;

__host__ __device__ __forceinline__ void cell_of(int half, int tid, int& p, int& zh, int& a, int& b, int& c) {
  const int w = tid >> 5, lane = tid & 31;
  p = half * 4 + (w >> 1);
  zh = w & 1;
  const int q = (zh << 5) + lane;
  a = 2 * (q & 3) + (p & 1);
  b = 2 * ((q >> 2) & 3) + ((p >> 1) & 1);
  c = 2 * (q >> 4) + (p >> 2);
}

__host__ __device__ __forceinline__ void unpack(int e, int& dx, int& dy, int& dz) {
  dx = (int)(int8_t)(e & 0xff);
  dy = (int)(int8_t)((e >> 8) & 0xff);
  dz = (int)(int8_t)((e >> 16) & 0xff);
}

// ------------------------------------------------------------ interior, float64
__device__ __forceinline__ void interior_f64(const DevTree& t, int node, int half, const Stencils& st,
                                             const double* __restrict__ mp, double* __restrict__ loc) {
  int p, zh, a, b, c;
  cell_of(half, threadIdx.x, p, zh, a, b, c);
  const int lvl = t.level[node];
  const int64_t NC = t.NC;
  const int64_t tgt = (int64_t)node * 512 + a + 8 * b + 64 * c;
  const double XA0 = mp[(F_X + 0) * NC + tgt], XA1 = mp[(F_X + 1) * NC + tgt], XA2 = mp[(F_X + 2) * NC + tgt];
  double Oh[10], tOh[3];
  {
    const double inv_m = 1.0 / mp[tgt];
    for (int i = 0; i < 10; ++i) Oh[i] = mp[(F_O + i) * NC + tgt] * inv_m;
    tOh[0] = Oh[0] + Oh[3] + Oh[5];
    tOh[1] = Oh[1] + Oh[6] + Oh[8];
    tOh[2] = Oh[2] + Oh[7] + Oh[9];
  }
  const int* tab = lvl == 0 ? st.root : st.parity + p * st.n_st;
  const int ntab = lvl == 0 ? st.n_root : st.n_st;
  const int* nb = t.nbr + 27 * node;
  Acc<double> acc;
  acc_zero(acc);
  for (int s = 0; s < ntab; ++s) {
    int dx, dy, dz;
    unpack(__ldg(tab + s), dx, dy, dz);
    const int sa = a + dx, sb = b + dy, sc = c + dz;
    const int snode = __ldg(nb + ((sa >> 3) + 1) + 3 * ((sb >> 3) + 1) + 9 * ((sc >> 3) + 1));
    if (snode < 0) continue;
    const int64_t src = (int64_t)snode * 512 + (sa & 7) + 8 * (sb & 7) + 64 * (sc & 7);
    const double R0 = XA0 - __ldg(mp + (F_X + 0) * NC + src);
    const double R1 = XA1 - __ldg(mp + (F_X + 1) * NC + src);
    const double R2 = XA2 - __ldg(mp + (F_X + 2) * NC + src);
    const double m = __ldg(mp + src);
    double Q[6], O[10];
    for (int i = 0; i < 6; ++i) Q[i] = __ldg(mp + (F_Q + i) * NC + src);
    for (int i = 0; i < 10; ++i) O[i] = __ldg(mp + (F_O + i) * NC + src);
    const double rinv = rsqrt_f64(fma(R0, R0, fma(R1, R1, R2 * R2)));
    m2l_pair<true, true>(R0, R1, R2, m, Q, O, Oh, tOh, rinv, acc);
  }
  acc_finish(acc);
  loc[G_L0 * NC + tgt] = acc.L0;
  for (int i = 0; i < 3; ++i) loc[(G_L1 + i) * NC + tgt] = acc.L1[i];
  for (int i = 0; i < 6; ++i) loc[(G_L2 + i) * NC + tgt] = acc.L2[i];
  for (int i = 0; i < 10; ++i) loc[(G_L3 + i) * NC + tgt] = acc.L3[i];
  for (int i = 0; i < 3; ++i) loc[(G_DG + i) * NC + tgt] = acc.dg[i];
}

// ------------------------------------------------------------ interior, float32
// Positions relative to node centres in cell widths: R = x_A - (x_B + 8 o) for a
// source in neighbour slot o.  Accumulation: the pair terms of st.acc_block (16, 32
// or 64; 32 by default) stencil entries are summed in plain float32 (fused multiply-adds); each partial sum then
// gets its deferred Kronecker parts (acc_finish is linear) and is added by an
// error-free transformation (TwoSum) into a float32 (sum, compensation) pair per
// field, kept in shared memory; sum + compensation is converted to float64 once, at
// the end.  A partial holds few terms, so its rounding error stays a few float32
// ulps of the partial, and the pairs add only the compensation's own rounding (a
// float32 ulp of an already float32-ulp-sized error): the accuracy of a compensated
// float32 sum at about a fifth of the instructions, with no float64 arithmetic
// inside the loop (the float64 pipe stays free for the near-field items that share
// the SM) and the 27 partials as the only accumulator registers.
constexpr int kInteriorFields = N_LOC;

// Shared memory of an interior item: one float2 (sum, compensation) per field and
// thread, field-major ([field][thread]), so that a warp's accesses are contiguous.
__host__ __device__ constexpr size_t interior_smem_bytes() { return sizeof(float2) * kInteriorFields * kThreads; }

// s + c <- s + c + p with the rounding error of s + p kept exactly in c's update
// (Knuth's TwoSum: six float32 additions, no branch, valid for any magnitudes).
__device__ __forceinline__ void two_sum_into(float2& sc, float p) {
  const float s = sc.x + p;
  const float bp = s - sc.x;
  const float err = (sc.x - (s - bp)) + (p - bp);
  sc.x = s;
  sc.y += err;
}

__device__ __forceinline__ void flush_partial(Acc<float>& a, float2* __restrict__ sc) {
  acc_finish(a);
  two_sum_into(sc[G_L0 * kThreads], a.L0);
  for (int i = 0; i < 3; ++i) two_sum_into(sc[(G_L1 + i) * kThreads], a.L1[i]);
  for (int i = 0; i < 6; ++i) two_sum_into(sc[(G_L2 + i) * kThreads], a.L2[i]);
  for (int i = 0; i < 10; ++i) two_sum_into(sc[(G_L3 + i) * kThreads], a.L3[i]);
  for (int i = 0; i < 3; ++i) two_sum_into(sc[(G_DG + i) * kThreads], a.dg[i]);
  acc_zero(a);
}

// The float32 record of one cell (a, b, c) of `node` (see device.cuh), field by field.
__device__ __forceinline__ void load_mp32_cell(const float* __restrict__ mp32, int node, int a, int b, int c,
                                               float& m, float x[3], float Q[6], float O[10]) {
  const float* r = mp32 + mp32_index(node, a, b, c, 0);
  auto f = [&](int k) { return __ldg(r + 4 * kMp32Pairs * (k >> 1) + 2 * (k & 1)); };
  m = f(F_M);
  for (int i = 0; i < 3; ++i) x[i] = f(F_X + i);
  for (int i = 0; i < 6; ++i) Q[i] = f(F_Q + i);
  for (int i = 0; i < 10; ++i) O[i] = f(F_O + i);
}

// The float32 records of the x-pair of cells at float4 index base (mp32_pair_base):
// ten 16-byte loads, every field as an F2 (lane 0: cell 2X, lane 1: cell 2X + 1).
__device__ __forceinline__ void load_mp32_pair(const float* __restrict__ mp32, int64_t base, F2& m, F2 x[3],
                                               F2 Q[6], F2 O[10]) {
  const float4* r = reinterpret_cast<const float4*>(mp32) + base;
  float4 v[kMp32Planes];
#pragma unroll
  for (int k = 0; k < kMp32Planes; ++k) v[k] = __ldg(r + k * kMp32Pairs);
  F2 f[N_MP];
#pragma unroll
  for (int k = 0; k < kMp32Planes; ++k) {
    f[2 * k] = f2(v[k].x, v[k].y);
    f[2 * k + 1] = f2(v[k].z, v[k].w);
  }
  m = f[F_M];
  for (int i = 0; i < 3; ++i) x[i] = f[F_X + i];
  for (int i = 0; i < 6; ++i) Q[i] = f[F_Q + i];
  for (int i = 0; i < 10; ++i) O[i] = f[F_O + i];
}

// One x-pair of float32 source records at `base` with the stencil-membership mask
// of a pair entry applied (a lane not in the stencil gets zero mass and moments),
// and the separation R = X_A - X_B to target position xA, the pair's node being
// offset by (ox, oy, oz) nodes from the target's.
__device__ __forceinline__ void pair_sources(const float* __restrict__ mp32, int64_t base, int mask,
                                             const float xA[3], int ox, int oy, int oz, F2& m, F2 Q[6],
                                             F2 O[10], F2& R0, F2& R1, F2& R2, F2& rinv) {
  F2 x[3];
  load_mp32_pair(mp32, base, m, x, Q, O);
  if (mask != 3) {
    const F2 w = f2(mask & 1 ? 1.0f : 0.0f, mask & 2 ? 1.0f : 0.0f);
    m = m * w;
    for (int i = 0; i < 6; ++i) Q[i] = Q[i] * w;
    for (int i = 0; i < 10; ++i) O[i] = O[i] * w;
  }
  const float c0 = xA[0] - 8.0f * (float)ox, c1 = xA[1] - 8.0f * (float)oy, c2 = xA[2] - 8.0f * (float)oz;
  R0 = f2(c0 - x[0].v.x, c0 - x[0].v.y);
  R1 = f2(c1 - x[1].v.x, c1 - x[1].v.y);
  R2 = f2(c2 - x[2].v.x, c2 - x[2].v.y);
  rinv = rsqrt2(fma2(R0, R0, fma2(R1, R1, R2 * R2)));
}

// Target cell and stencil range of a thread of an interior item.  split 1: part =
// half (0, 1) of the node, thread = cell (cell_of), all entries.  split 2: part =
// quarter (0..3) of the node = parity classes 2 part and 2 part + 1 (warps 0-3 and
// 4-7 hold the same 128 cells, one stencil half each); still one parity class per
// warp.
__host__ __device__ __forceinline__ void interior_cell(int split, int part, int tid, int ntab, int& p, int& a,
                                                       int& b, int& c, int& s_begin, int& s_end) {
  int zh;
  if (split == 2) {
    const int w = (tid >> 5) & 3, lane = tid & 31;
    p = 2 * part + (w >> 1);
    zh = w & 1;
    const int q = (zh << 5) + lane;
    a = 2 * (q & 3) + (p & 1);
    b = 2 * ((q >> 2) & 3) + ((p >> 1) & 1);
    c = 2 * (q >> 4) + (p >> 2);
    const int h = (ntab + 1) >> 1;
    s_begin = tid < 128 ? 0 : h;
    s_end = tid < 128 ? h : ntab;
  } else {
    cell_of(part, tid, p, zh, a, b, c);
    s_begin = 0;
    s_end = ntab;
  }
}

// C64: the angular-momentum correction of every pair is formed in float64 from the
// float64 multipoles (mp) and summed in float64, beside the float32 pair without it
// (a measurement variant of the mixed path; per-kind launches, split 1 only).
// BLK: stencil entries per float32 partial sum; SPLIT: 1 or 2 (see interior_cell).
// The kernels are instantiated per shape (a runtime choice inside one kernel made
// the 80-register variants spill).  Contains a block-wide barrier when SPLIT == 2
// (every thread reaches it).
template <bool C64, int BLK, int SPLIT>
__device__ __forceinline__ void interior_f32(const DevTree& t, int node, int part, const Stencils& st,
                                             const float* __restrict__ mp32, double* __restrict__ loc,
                                             unsigned char* smem, const double* __restrict__ mp) {
  const int lvl = t.level[node];
  const int ntab = lvl == 0 ? st.n_root : st.n_st;
  constexpr int split = SPLIT;
  int p, a, b, c, s_begin, s_end;
  interior_cell(split, part, threadIdx.x, ntab, p, a, b, c, s_begin, s_end);
  const int64_t NC = t.NC;
  const int64_t tgt = (int64_t)node * 512 + a + 8 * b + 64 * c;
  double XA64[3], Oh64[10], tOh64[3];
  DgAcc d64 = {{0.0, 0.0, 0.0}};
  if constexpr (C64) {
    for (int i = 0; i < 3; ++i) XA64[i] = mp[(F_X + i) * NC + tgt];
    const double inv_m = 1.0 / mp[tgt];
    for (int i = 0; i < 10; ++i) Oh64[i] = mp[(F_O + i) * NC + tgt] * inv_m;
    tOh64[0] = Oh64[0] + Oh64[3] + Oh64[5];
    tOh64[1] = Oh64[1] + Oh64[6] + Oh64[8];
    tOh64[2] = Oh64[2] + Oh64[7] + Oh64[9];
  }
  float mA, xA[3], QA[6], Oh[10], tOh[3];
  load_mp32_cell(mp32, node, a, b, c, mA, xA, QA, Oh);
  {
    const float inv_m = 1.0f / mA;
    for (int i = 0; i < 10; ++i) Oh[i] *= inv_m;
    tOh[0] = Oh[0] + Oh[3] + Oh[5];
    tOh[1] = Oh[1] + Oh[6] + Oh[8];
    tOh[2] = Oh[2] + Oh[7] + Oh[9];
  }
  const int* tab = lvl == 0 ? st.root : st.parity + p * st.n_st;
  const int* nb = t.nbr + 27 * node;
  float2* sc = reinterpret_cast<float2*>(smem) + threadIdx.x;
  for (int f = 0; f < kInteriorFields; ++f) sc[f * kThreads] = make_float2(0.0f, 0.0f);
  Acc<float> part_sum;
  acc_zero(part_sum);
  for (int s0 = s_begin; s0 < s_end; s0 += BLK) {
    const int s1 = min(s0 + BLK, s_end);
    for (int s = s0; s < s1; ++s) {
      int dx, dy, dz;
      unpack(__ldg(tab + s), dx, dy, dz);
      const int sa = a + dx, sb = b + dy, sc = c + dz;
      const int ox = sa >> 3, oy = sb >> 3, oz = sc >> 3;
      const int snode = __ldg(nb + (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1));
      if (snode < 0) continue;
      float m, x[3], Q[6], O[10];
      load_mp32_cell(mp32, snode, sa & 7, sb & 7, sc & 7, m, x, Q, O);
      const float R0 = xA[0] - (x[0] + 8.0f * (float)ox);
      const float R1 = xA[1] - (x[1] + 8.0f * (float)oy);
      const float R2 = xA[2] - (x[2] + 8.0f * (float)oz);
      const float rinv = rsqrt_f32(fmaf(R0, R0, fmaf(R1, R1, R2 * R2)));
      m2l_pair<true, true, float, Acc<float>, !C64>(R0, R1, R2, m, Q, O, Oh, tOh, rinv, part_sum);
      if constexpr (C64) {
        const int64_t src = (int64_t)snode * 512 + (sa & 7) + 8 * (sb & 7) + 64 * (sc & 7);
        const double S0 = XA64[0] - __ldg(mp + (F_X + 0) * NC + src);
        const double S1 = XA64[1] - __ldg(mp + (F_X + 1) * NC + src);
        const double S2 = XA64[2] - __ldg(mp + (F_X + 2) * NC + src);
        double O64[10];
        for (int i = 0; i < 10; ++i) O64[i] = __ldg(mp + (F_O + i) * NC + src);
        corr_pair_f64<true>(S0, S1, S2, __ldg(mp + src), O64, Oh64, tOh64,
                            rsqrt_f64(fma(S0, S0, fma(S1, S1, S2 * S2))), d64);
      }
    }
    flush_partial(part_sum, sc);
  }
  if constexpr (split == 2) {  // the second stencil half's (sum, compensation) pairs join the first's
    __syncthreads();
    if (threadIdx.x >= 128) return;
    for (int f = 0; f < kInteriorFields; ++f) {
      const float2 o = sc[f * kThreads + 128];
      two_sum_into(sc[f * kThreads], o.x);
      sc[f * kThreads].y += o.y;
    }
  }
  // sum + compensation in float64; unit cell width -> physical units: L_n scales
  // with h^-(n+1), dg with h^-2
  const double ih = 1.0 / t.h[lvl], ih2 = ih * ih, ih3 = ih2 * ih, ih4 = ih2 * ih2;
  auto out = [&](int f, double scale) {
    const float2 v = sc[f * kThreads];
    loc[f * NC + tgt] = ((double)v.x + (double)v.y) * scale;
  };
  out(G_L0, ih);
  for (int i = 0; i < 3; ++i) out(G_L1 + i, ih2);
  for (int i = 0; i < 6; ++i) out(G_L2 + i, ih3);
  for (int i = 0; i < 10; ++i) out(G_L3 + i, ih4);
  if constexpr (C64) {
    for (int i = 0; i < 3; ++i) loc[(G_DG + i) * NC + tgt] = d64.dg[i];  // physical units already
  } else {
    for (int i = 0; i < 3; ++i) out(G_DG + i, ih2);
  }
}

// The mixed path's interior M2L in paired float32 instructions: the stencil of the
// thread's parity class grouped into aligned x-pairs of source cells (st.pair, see
// build_pair_tables), each pair one iteration that loads the two cells' records
// with ten 16-byte loads (the pair layout of mp32) and computes both M2L pairs at
// once (m2l_pair_x2).  A stencil entry whose x-partner is not in the stencil is a
// pair with one lane masked to zero mass and moments.  Same targets, partial-sum
// blocks (BLK stencil entries, BLK / 2 pairs), compensated flush and split as
// interior_f32.  Contains a block-wide barrier when SPLIT == 2.
template <int BLK, int SPLIT>
__device__ __forceinline__ void interior_f32x2(const DevTree& t, int node, int part, const Stencils& st,
                                               const float* __restrict__ mp32, double* __restrict__ loc,
                                               unsigned char* smem) {
  static_assert(BLK % 2 == 0, "pairs per partial sum");
  const int lvl = t.level[node];
  const int ntab = lvl == 0 ? st.n_pair_root : st.n_pair;
  int p, a, b, c, s_begin, s_end;
  interior_cell(SPLIT, part, threadIdx.x, ntab, p, a, b, c, s_begin, s_end);
  const int64_t NC = t.NC;
  const int64_t tgt = (int64_t)node * 512 + a + 8 * b + 64 * c;
  float mA, xA[3], QA[6], Oh[10], tOh[3];
  load_mp32_cell(mp32, node, a, b, c, mA, xA, QA, Oh);
  {
    const float inv_m = 1.0f / mA;
    for (int i = 0; i < 10; ++i) Oh[i] *= inv_m;
    tOh[0] = Oh[0] + Oh[3] + Oh[5];
    tOh[1] = Oh[1] + Oh[6] + Oh[8];
    tOh[2] = Oh[2] + Oh[7] + Oh[9];
  }
  const int* tab = lvl == 0 ? st.pair_root + p * st.n_pair_root : st.pair + p * st.n_pair;
  const int* nb = t.nbr + 27 * node;
  float2* sc = reinterpret_cast<float2*>(smem) + threadIdx.x;
  for (int f = 0; f < kInteriorFields; ++f) sc[f * kThreads] = make_float2(0.0f, 0.0f);
  Acc<float> part_sum;
  acc_zero(part_sum);
  for (int s0 = s_begin; s0 < s_end; s0 += BLK / 2) {
    const int s1 = min(s0 + BLK / 2, s_end);
    for (int s = s0; s < s1; ++s) {
      const int e = __ldg(tab + s);
      int dx, dy, dz;
      unpack(e, dx, dy, dz);
      const int sa = a + dx, sb = b + dy, sc_ = c + dz;  // sa even: cells sa, sa + 1
      const int ox = sa >> 3, oy = sb >> 3, oz = sc_ >> 3;
      const int snode = __ldg(nb + (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1));
      if (snode < 0) continue;
      F2 m, Q[6], O[10], R0, R1, R2, rinv;
      pair_sources(mp32, mp32_pair_base(snode, (sa & 7) >> 1, sb & 7, sc_ & 7), (e >> 24) & 3, xA, ox, oy, oz, m, Q,
                   O, R0, R1, R2, rinv);
      m2l_pair_x2<true>(R0, R1, R2, m, Q, O, Oh, tOh, rinv, part_sum);
    }
    flush_partial(part_sum, sc);
  }
  if constexpr (SPLIT == 2) {  // the second stencil half's (sum, compensation) pairs join the first's
    __syncthreads();
    if (threadIdx.x >= 128) return;
    for (int f = 0; f < kInteriorFields; ++f) {
      const float2 o = sc[f * kThreads + 128];
      two_sum_into(sc[f * kThreads], o.x);
      sc[f * kThreads].y += o.y;
    }
  }
  // sum + compensation in float64; unit cell width -> physical units: L_n scales
  // with h^-(n+1), dg with h^-2
  const double ih = 1.0 / t.h[lvl], ih2 = ih * ih, ih3 = ih2 * ih, ih4 = ih2 * ih2;
  auto out = [&](int f, double scale) {
    const float2 v = sc[f * kThreads];
    loc[f * NC + tgt] = ((double)v.x + (double)v.y) * scale;
  };
  out(G_L0, ih);
  for (int i = 0; i < 3; ++i) out(G_L1 + i, ih2);
  for (int i = 0; i < 6; ++i) out(G_L2 + i, ih3);
  for (int i = 0; i < 10; ++i) out(G_L3 + i, ih4);
  for (int i = 0; i < 3; ++i) out(G_DG + i, ih2);
}

// ------------------------------------------------------------ leaf item
// Shared memory of a leaf item: the far halo (float32 in the mixed path, float64
// otherwise), and at least 512 x 7 doubles (the boundary results are exchanged
// through it).  Mixed path: then, per warp, two staging buffers of one table block
// (kLeafTableBlockBytes each) and their two mbarriers.  The near item of the mixed
// path needs the near float64 halo.
__host__ __device__ inline size_t leaf_halo_bytes(const Stencils& st, bool mixed) {
  const HaloGeom gf = far_geom(st.radius, mixed);
  const size_t halo = (mixed ? sizeof(float) : sizeof(double)) * 8 * (size_t)gf.PQ;
  const size_t b = halo > sizeof(double) * 512 * 7 ? halo : sizeof(double) * 512 * 7;
  return (b + 127) & ~(size_t)127;
}
constexpr int kLeafWarps = kThreads / 32;
__host__ __device__ inline size_t leaf_smem_bytes(const Stencils& st, bool mixed) {
  return leaf_halo_bytes(st, mixed) +
         (mixed ? (size_t)kLeafWarps * (2 * kLeafTableBlockBytes + 2 * sizeof(uint64_t)) : 0);
}

__host__ __device__ inline size_t near_smem_bytes(const Stencils& st) {
  return sizeof(double) * 8 * (size_t)near_geom(st.near_radius).PQ;
}


// Accumulator of a leaf target (m2l_pair<false, ...> touches only L0, L1, dg).
template <typename T>
struct LeafAcc {
  T L0, L1[3], dg[3];
};

// Compensated merge of float32 partial sums into acc (Acc<KF>); zeroes the partials.
template <typename A>
__device__ __forceinline__ void leaf_merge(A& acc, LeafAcc<float>& p) {
  acc.L0.add(p.L0);
  p.L0 = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    acc.L1[i].add(p.L1[i]);
    acc.dg[i].add(p.dg[i]);
    p.L1[i] = 0.0f;
    p.dg[i] = 0.0f;
  }
}

// boundary_pairs of the mixed path (float32 correction) by x-pairs of source cells:
// the per-cell lists grouped like the interior stencils (st.cell_pair, see
// build_cell_pair_lists), two sources per iteration in paired float32 instructions,
// st.acc_block / 2 pairs per float32 partial sum.
template <typename A>
__device__ __forceinline__ void boundary_pairs_x2(const DevTree& t, int node, int l, const Stencils& st,
                                                  const float* __restrict__ mp32, A& acc) {
  const int a = l & 7, b = (l >> 3) & 7, c = l >> 6;
  const int* nb = t.nbr + 27 * node;
  float xA[3];
  for (int i = 0; i < 3; ++i) xA[i] = __ldg(mp32 + mp32_index(node, a, b, c, F_X + i));
  LeafAcc<float> part = {0.0f, {0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
  int n_part = 0;
  // the lanes advance through their (slot, pair) lists independently, as in
  // boundary_pairs
  int o = -1, e = 0, e1 = 0, sn = -1, ox = 0, oy = 0, oz = 0;
  for (;;) {
    while (e == e1 && o < 27) {
      if (++o == 27) break;
      sn = nb[o];
      if (sn < 0 || t.children[8 * sn] < 0) continue;  // refined neighbours only
      ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
      e = __ldg(st.cell_pair_off + l * 27 + o), e1 = __ldg(st.cell_pair_off + l * 27 + o + 1);
    }
    if (o == 27) break;
    const int en = __ldg(st.cell_pair + e);
    int dx, dy, dz;
    unpack(en, dx, dy, dz);
    const int sa = a + dx, sb = b + dy, sc = c + dz;  // sa even
    F2 m, Q[6], O[10], R0, R1, R2, rinv;
    pair_sources(mp32, mp32_pair_base(sn, (sa & 7) >> 1, sb & 7, sc & 7), (en >> 24) & 3, xA, ox, oy, oz, m, Q, O,
                 R0, R1, R2, rinv);
    m2l_pair_x2<false>(R0, R1, R2, m, Q, O, nullptr, nullptr, rinv, part);
    if (++n_part == st.acc_block / 2) {
      leaf_merge(acc, part);
      n_part = 0;
    }
    ++e;
  }
  leaf_merge(acc, part);
}

// M2L from refined same-level neighbours into leaf cell l of a leaf node (leaf
// target: L0, L1, dg).  The per-cell entry lists hold only offsets whose source
// lies in the neighbour slot, so every iteration of every lane is a valid pair.
// Mixed path: plain float32 partial sums of st.acc_block pairs merged into the
// compensated sums of acc (Acc<KF>).
template <bool MIXED, typename A, bool C64 = false>
__device__ __forceinline__ void boundary_pairs(const DevTree& t, int node, int l, const Stencils& st,
                                               const double* __restrict__ mp, const float* __restrict__ mp32,
                                               A& acc, DgAcc* d64 = nullptr) {
  if constexpr (MIXED && !C64) {
    boundary_pairs_x2(t, node, l, st, mp32, acc);
    return;
  }
  using T = typename std::conditional<MIXED, float, double>::type;
  const int64_t NC = t.NC;
  const int a = l & 7, b = (l >> 3) & 7, c = l >> 6;
  const int64_t tgt = (int64_t)node * 512 + l;
  const int* nb = t.nbr + 27 * node;
  T xA0, xA1, xA2;
  if constexpr (MIXED) {
    xA0 = __ldg(mp32 + mp32_index(node, a, b, c, F_X + 0));
    xA1 = __ldg(mp32 + mp32_index(node, a, b, c, F_X + 1));
    xA2 = __ldg(mp32 + mp32_index(node, a, b, c, F_X + 2));
  } else {
    xA0 = mp[(F_X + 0) * NC + tgt], xA1 = mp[(F_X + 1) * NC + tgt], xA2 = mp[(F_X + 2) * NC + tgt];
  }
  const T zero10[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  // mixed path: partial sums of L0, L1, dg (the only fields a leaf target gets)
  LeafAcc<float> part = {0.0f, {0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
  int n_part = 0;
  // One flat walk over the (refined neighbour slot, entry) pairs of this cell: the
  // lanes of a warp (cells of similar total load) advance to their next slot
  // independently, so a warp runs as many iterations as its busiest lane rather
  // than the sum over slots of the per-slot maxima.  Each cell still takes its
  // pairs in slot order, then entry order.
  int o = -1, e = 0, e1 = 0, sn = -1, ox = 0, oy = 0, oz = 0;
  for (;;) {
    while (e == e1 && o < 27) {  // next refined neighbour slot of this cell
      if (++o == 27) break;
      sn = nb[o];
      if (sn < 0 || t.children[8 * sn] < 0) continue;  // refined neighbours only
      ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
      e = __ldg(st.cell_ent_off + l * 27 + o), e1 = __ldg(st.cell_ent_off + l * 27 + o + 1);
    }
    if (o == 27) break;
    {
      int dx, dy, dz;
      unpack(__ldg(st.cell_ent + e), dx, dy, dz);
      const int sa = a + dx, sb = b + dy, sc = c + dz;
      const int64_t src = (int64_t)sn * 512 + (sa & 7) + 8 * (sb & 7) + 64 * (sc & 7);
      T R0, R1, R2, m, Q[6], O[10], rinv;
      if constexpr (MIXED) {
        float x[3];
        load_mp32_cell(mp32, sn, sa & 7, sb & 7, sc & 7, m, x, Q, O);
        R0 = xA0 - (x[0] + 8.0f * (float)ox);
        R1 = xA1 - (x[1] + 8.0f * (float)oy);
        R2 = xA2 - (x[2] + 8.0f * (float)oz);
        rinv = rsqrt_f32(fmaf(R0, R0, fmaf(R1, R1, R2 * R2)));
      } else {
        R0 = xA0 - __ldg(mp + (F_X + 0) * NC + src);
        R1 = xA1 - __ldg(mp + (F_X + 1) * NC + src);
        R2 = xA2 - __ldg(mp + (F_X + 2) * NC + src);
        m = __ldg(mp + src);
        for (int i = 0; i < 6; ++i) Q[i] = __ldg(mp + (F_Q + i) * NC + src);
        for (int i = 0; i < 10; ++i) O[i] = __ldg(mp + (F_O + i) * NC + src);
        rinv = rsqrt_f64(fma(R0, R0, fma(R1, R1, R2 * R2)));
      }
      if constexpr (MIXED) {
        m2l_pair<false, false, float, LeafAcc<float>, !C64>(R0, R1, R2, m, Q, O, zero10, zero10, rinv, part);
        if constexpr (C64) {
          const double S0 = mp[(F_X + 0) * NC + tgt] - __ldg(mp + (F_X + 0) * NC + src);
          const double S1 = mp[(F_X + 1) * NC + tgt] - __ldg(mp + (F_X + 1) * NC + src);
          const double S2 = mp[(F_X + 2) * NC + tgt] - __ldg(mp + (F_X + 2) * NC + src);
          double O64[10];
          for (int i = 0; i < 10; ++i) O64[i] = __ldg(mp + (F_O + i) * NC + src);
          corr_pair_f64<false>(S0, S1, S2, __ldg(mp + src), O64, nullptr, nullptr,
                               rsqrt_f64(fma(S0, S0, fma(S1, S1, S2 * S2))), *d64);
        }
        if (++n_part == st.acc_block) {
          leaf_merge(acc, part);
          n_part = 0;
        }
      } else {
        m2l_pair<false, false>(R0, R1, R2, m, Q, O, zero10, zero10, rinv, acc);
      }
    }
    ++e;
  }
  if constexpr (MIXED) leaf_merge(acc, part);
}

// Stages the masses of the leaf same-level neighbourhood of `node` (cells within
// border g.r of the node) into a parity-split halo; refined or missing neighbours
// contribute zero.  nleaf: the 27 neighbours (or the node itself) if leaves, else -1.
template <typename T>
__device__ __forceinline__ void stage_halo(const HaloGeom& g, const int* nleaf, const double* __restrict__ mp,
                                           T* halo) {
  // one halo row (fixed y, z) per warp and step, lanes along x (consecutive cells of
  // a neighbour's row are contiguous in memory); kRows rows of loads in flight
  constexpr int kRows = 4;
  const int H = 2 * g.G, R = g.r, n_rows = H * H;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  for (int x0 = 0; x0 < H; x0 += 32) {
    const int hx = x0 + lane;
    const int x = hx - R;
    for (int r0 = warp; r0 < n_rows; r0 += kRows * n_warps) {
      double m[kRows];
#pragma unroll
      for (int u = 0; u < kRows; ++u) {
        const int r = r0 + u * n_warps;
        m[u] = 0.0;
        if (r < n_rows && hx < H) {
          const int y = r % H - R, z = r / H - R;
          const int sn = nleaf[((x >> 3) + 1) + 3 * ((y >> 3) + 1) + 9 * ((z >> 3) + 1)];
          if (sn >= 0) m[u] = __ldg(mp + (int64_t)sn * 512 + (x & 7) + 8 * (y & 7) + 64 * (z & 7));
        }
      }
#pragma unroll
      for (int u = 0; u < kRows; ++u) {
        const int r = r0 + u * n_warps;
        if (r < n_rows && hx < H) halo[halo_index(g, hx, r % H, r / H)] = (T)m[u];
      }
    }
  }
}

// stage_halo of the mixed path, from the float32 masses of mp32 (the float32
// rounding of mp's masses, the same values): each lane loads the two masses of an
// x-pair of cells (8 bytes) for one halo row, the two halves of a warp take two
// rows, and each lane keeps kRowPairs loads in flight, so that a block stages its
// halo in a few round trips to L2.
__device__ __forceinline__ void stage_halo_mixed(const HaloGeom& g, const int* nleaf, const float* __restrict__ mp32,
                                                 float* halo) {
  constexpr int kRowPairs = 6;
  const int R = g.r, H = 2 * g.G, n_rows = H * H;
  const int x_first = (-R) & ~1;               // even x of the first pair (floor)
  const int n_pairs = (7 + R - x_first) / 2 + 1;  // pairs covering x in [-R, 7 + R]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
  const int q = lane & 15, sub = lane >> 4;
  const int x = x_first + 2 * q;
  for (int r0 = 2 * warp + sub; r0 < n_rows; r0 += 2 * n_warps * kRowPairs) {
    float2 m[kRowPairs];
#pragma unroll
    for (int u = 0; u < kRowPairs; ++u) {
      const int r = r0 + u * 2 * n_warps;
      m[u] = make_float2(0.0f, 0.0f);
      if (r < n_rows && q < n_pairs) {
        const int y = r % H - R, z = r / H - R;
        const int sn = nleaf[((x >> 3) + 1) + 3 * ((y >> 3) + 1) + 9 * ((z >> 3) + 1)];
        if (sn >= 0) m[u] = __ldg(reinterpret_cast<const float2*>(mp32 + mp32_index(sn, x & 7, y & 7, z & 7, F_M)));
      }
    }
#pragma unroll
    for (int u = 0; u < kRowPairs; ++u) {
      const int r = r0 + u * 2 * n_warps;
      if (r < n_rows && q < n_pairs) {
        const int hx = x + R, hy = r % H, hz = r / H;
        if (hx >= 0) halo[halo_index(g, hx, hy, hz)] = m[u].x;
        if (hx + 1 < H) halo[halo_index(g, hx + 1, hy, hz)] = m[u].y;
      }
    }
  }
}

// Leaf neighbour table of `node` into shared memory; returns whether any same-level
// neighbour is refined (block-uniform).  Ends with a barrier.
__device__ __forceinline__ bool load_leaf_neighbours(const DevTree& t, int node, int* nleaf) {
  __syncthreads();  // the previous item may still read shared memory
  bool refined = false;
  if (threadIdx.x < 27) {
    const int sn = t.nbr[27 * node + threadIdx.x];
    refined = sn >= 0 && t.children[8 * sn] >= 0;
    nleaf[threadIdx.x] = sn >= 0 && !refined ? sn : -1;
  }
  return __syncthreads_or(refined) != 0;
}

// Local index of the q-th (q = 0, 1) cell owned by thread tid in a leaf item.
// Mixed path: warp w holds parity class w, lane (i, j, kh) the cells
// (2i + pa, 2j + pb, 2 (2 kh + q) + pc), adjacent planes of the parity class.
// Float64 path: cell_of(q, tid).
template <bool MIXED>
__host__ __device__ __forceinline__ int leaf_cell(int q, int tid) {
  if (MIXED) {
    const int p = tid >> 5, lane = tid & 31;
    const int a = 2 * (lane & 3) + (p & 1), b = 2 * ((lane >> 2) & 3) + ((p >> 1) & 1);
    const int c = 2 * (2 * (lane >> 4) + q) + (p >> 2);
    return a + 8 * b + 64 * c;
  }
  int p, zh, a, b, c;
  cell_of(q, tid, p, zh, a, b, c);
  return a + 8 * b + 64 * c;
}

// One leaf node per block (both halves): stage the halo once, then every thread
// computes its cell of each half.  Mixed path: the float32 far field only (the
// float64 near field is the separate near item, so that the two can run side by
// side on an SM); float64 path: far and near field.
template <bool MIXED, bool C64 = false>
__device__ __forceinline__ void leaf_item(const DevTree& t, int node, const Stencils& st,
                                          const double* __restrict__ mp, const float* __restrict__ mp32,
                                          double* __restrict__ loc, unsigned char* smem) {
  const HaloGeom gf = far_geom(st.radius, MIXED);
  __shared__ int nleaf[27];
  const bool any_refined = load_leaf_neighbours(t, node, nleaf);
  float* halo32 = reinterpret_cast<float*>(smem);
  double* halo64 = reinterpret_cast<double*>(smem);
  if (MIXED)
    stage_halo_mixed(gf, nleaf, mp32, halo32);
  else
    stage_halo(gf, nleaf, mp, halo64);
  __syncthreads();
  const int lvl = t.level[node];
  const int n_far = lvl == 0 ? st.n_root : st.n_st;
  const double ih = 1.0 / t.h[lvl], ih2 = ih * ih;
  double L0[2], L1[2][3];  // the thread's two cells (see leaf_cell)
  if (MIXED) {
    // warp w = parity class w; lane (i, j, kh) owns the cells of parity planes 2 kh
    // and 2 kh + 1 (leaf_cell).  The warp's stencil is a list of z-columns (runs of
    // entries d, d + 2 e_z, ... whose sources are consecutive planes of one parity
    // block): along a column the lane's first cell reads masses M_0 .. M_{L-1} and
    // its second cell M_1 .. M_L, so one shared-memory load serves both cells, and
    // each entry is four paired float32 FMAs (both cells' L0, L1 from the duplicated
    // mass and the entry's kernel row).  The table streams through shared memory in
    // blocks (kLeafTableBlockBytes: column headers, then kernel rows), each fetched
    // by one bulk asynchronous copy (TMA) issued a block ahead into the other of two
    // buffers; each block is one float32 partial sum, merged into compensated sums.
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nblk = lvl == 0 ? st.root_blocks : st.far_blocks;
    const unsigned char* gtab = reinterpret_cast<const unsigned char*>(st.leaf_blocks) +
                                ((lvl == 0 ? (size_t)8 * st.far_blocks + (size_t)w * st.root_blocks
                                           : (size_t)w * st.far_blocks) *
                                 kLeafTableBlockBytes);
    unsigned char* sbuf = smem + leaf_halo_bytes(st, true) + (size_t)w * 2 * kLeafTableBlockBytes;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + leaf_halo_bytes(st, true) +
                                                (size_t)kLeafWarps * 2 * kLeafTableBlockBytes) +
                    2 * w;
    const int lane_f = (lane & 3) + gf.PY * ((lane >> 2) & 3) + gf.PZ * 2 * (lane >> 4);
    const int PZ = gf.PZ;
    KF f[2][4];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k) f[q][k] = 0.0f;
    if (lane == 0 && nblk > 0) {
      tma::mbar_init(bar);
      tma::mbar_init(bar + 1);
      tma::fence_mbar_init();
      tma::fence_proxy_async();  // earlier items wrote this shared memory
      tma::mbar_expect_tx(bar, kLeafTableBlockBytes);
      tma::copy_g2s(sbuf, gtab, kLeafTableBlockBytes, bar);
    }
    __syncwarp();
    bool ok = true;
    int b = 0;
    for (; b < nblk; ++b) {
      if (lane == 0 && b + 1 < nblk) {  // the next block into the other buffer
        unsigned char* nb = sbuf + ((b + 1) & 1) * kLeafTableBlockBytes;
        tma::fence_proxy_async();
        tma::mbar_expect_tx(bar + ((b + 1) & 1), kLeafTableBlockBytes);
        tma::copy_g2s(nb, gtab + (size_t)(b + 1) * kLeafTableBlockBytes, kLeafTableBlockBytes, bar + ((b + 1) & 1));
      }
      ok = __all_sync(0xffffffffu, tma::mbar_wait(bar + (b & 1), (b >> 1) & 1));
      if (!ok) break;
      const int* hdr = reinterpret_cast<const int*>(sbuf + (b & 1) * kLeafTableBlockBytes);
      const float4* ks = reinterpret_cast<const float4*>(hdr + kLeafBlock);
      // (L0, L1x), (L1y, L1z) of cells A and B; two sets, even and odd chunks, for
      // two independent FMA chains per sum
      F2 acc[2][4] = {{bc(0.0f), bc(0.0f), bc(0.0f), bc(0.0f)}, {bc(0.0f), bc(0.0f), bc(0.0f), bc(0.0f)}};
      // chunks of C entries, fully unrolled: the chunk's C + 1 masses (cell A reads
      // M_0 .. M_{C-1}, cell B M_1 .. M_C), then four paired FMAs per entry
      auto chunks = [&](auto c_, auto n_) {
        constexpr int C = decltype(c_)::value, N = decltype(n_)::value;
#pragma unroll
        for (int ci = 0; ci < N; ++ci) {
          const float* src = halo32 + lane_f + (hdr[ci] & 0xfffff);
          F2 M[C + 1];
#pragma unroll
          for (int u = 0; u <= C; ++u) M[u] = bc(src[u * PZ]);
          F2* a = acc[ci & 1];
#pragma unroll
          for (int u = 0; u < C; ++u) {
            const float4 k = ks[C * ci + u];
            const F2 k01 = f2(k.x, k.y), k23 = f2(k.z, k.w);
            a[0] = fma2(M[u], k01, a[0]);
            a[1] = fma2(M[u], k23, a[1]);
            a[2] = fma2(M[u + 1], k01, a[2]);
            a[3] = fma2(M[u + 1], k23, a[3]);
          }
        }
      };
      switch (hdr[0] >> 20) {  // warp-uniform chunk length of this block (0: empty)
        case 3: chunks(std::integral_constant<int, 3>(), std::integral_constant<int, 10>()); break;
        case 2: chunks(std::integral_constant<int, 2>(), std::integral_constant<int, 16>()); break;
        case 1: chunks(std::integral_constant<int, 1>(), std::integral_constant<int, 32>()); break;
      }
      const F2 A01 = acc[0][0] + acc[1][0], A23 = acc[0][1] + acc[1][1];
      const F2 B01 = acc[0][2] + acc[1][2], B23 = acc[0][3] + acc[1][3];
      f[0][0].add(A01.v.x), f[0][1].add(A01.v.y), f[0][2].add(A23.v.x), f[0][3].add(A23.v.y);
      f[1][0].add(B01.v.x), f[1][1].add(B01.v.y), f[1][2].add(B23.v.x), f[1][3].add(B23.v.y);
      __syncwarp();  // every lane has read this buffer before it is refilled
    }
    if (!ok) {
      // a copy did not complete in time: report it, let the copies in flight land
      // (bounded), and leave this item's far field incomplete
      if (lane == 0) atomicOr(st.err, kErrTimeout);
      tma::mbar_wait(bar + (b & 1), (b >> 1) & 1);
      if (b + 1 < nblk) tma::mbar_wait(bar + ((b + 1) & 1), ((b + 1) >> 1) & 1);
    }
    // every phase of both barriers has completed: invalidate them, so that the next
    // leaf item of this block can initialise them again and other items may reuse
    // the memory
    __syncwarp();
    if (lane == 0 && nblk > 0) {
      tma::mbar_inval(bar);
      tma::mbar_inval(bar + 1);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      L0[q] = f[q][0].value() * ih;
      for (int i = 0; i < 3; ++i) L1[q][i] = f[q][1 + i].value() * ih2;
    }
  } else {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      int p, zh, a, b, c;
      cell_of(half, threadIdx.x, p, zh, a, b, c);
      const int2* __restrict__ far = (lvl == 0 ? st.leaf_root : st.leaf_far) + p * n_far;
      const int2* __restrict__ nr = st.leaf_near + p * st.n_near;
      const int lane_f = (a >> 1) + gf.PY * (b >> 1) + gf.PZ * (c >> 1);
      double s0 = 0, s1 = 0, s2 = 0, s3 = 0;  // unit cell width
      for (int s = 0; s < n_far; ++s) {
        const int2 e = __ldg(far + s);
        const double m = halo64[lane_f + e.x];
        const double2* kp = reinterpret_cast<const double2*>(st.kappa + e.y);
        const double2 ka = __ldg(kp), kb = __ldg(kp + 1);
        s0 = fma(m, ka.x, s0);
        s1 = fma(m, ka.y, s1);
        s2 = fma(m, kb.x, s2);
        s3 = fma(m, kb.y, s3);
      }
      for (int s = 0; s < st.n_near; s += 2) {  // (d, -d) pairs, as in near_item
        const int2 e = __ldg(nr + s), f = __ldg(nr + s + 1);
        const double mp_ = halo64[lane_f + e.x], mm = halo64[lane_f + f.x];
        const double2* kp = reinterpret_cast<const double2*>(st.kappa + e.y);
        const double2 ka = __ldg(kp), kb = __ldg(kp + 1);
        const double sum = mp_ + mm, dif = mp_ - mm;
        s0 = fma(sum, ka.x, s0);
        s1 = fma(dif, ka.y, s1);
        s2 = fma(dif, kb.x, s2);
        s3 = fma(dif, kb.y, s3);
      }
      L0[half] = s0 * ih;
      L1[half][0] = s1 * ih2;
      L1[half][1] = s2 * ih2;
      L1[half][2] = s3 * ih2;
    }
  }
  double dg[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  if (any_refined) {  // block-uniform
    // Boundary pairs: the node's cells in decreasing order of load, in groups of 32
    // (one cell per lane, similar loads within a warp), claimed by the warps one
    // group at a time from a shared counter, heaviest first, so that the block
    // waits for about max(heaviest group, total / warps) rather than for one warp
    // holding several heavy groups.  The results go back to the owning threads
    // through shared memory (the halo is no longer needed).
    __shared__ int next_group;
    if (threadIdx.x == 0) next_group = 0;
    __syncthreads();
    double* res = reinterpret_cast<double*>(smem);  // [512][7]
    const int lane = threadIdx.x & 31;
    for (;;) {
      int g = 0;
      if (lane == 0) g = atomicAdd(&next_group, 1);
      g = __shfl_sync(0xffffffffu, g, 0);
      if (g >= 512 / 32) break;
      const int lb = st.bnd_perm[(int64_t)st.bnd_index[node] * 512 + g * 32 + lane];
      double v[7];
      if constexpr (MIXED) {
        Acc<KF> acc;
        acc_zero(acc);
        DgAcc d64 = {{0.0, 0.0, 0.0}};
        boundary_pairs<true, Acc<KF>, C64>(t, node, lb, st, mp, mp32, acc, &d64);
        v[0] = acc.L0.value() * ih;
        for (int i = 0; i < 3; ++i)
          v[1 + i] = acc.L1[i].value() * ih2, v[4 + i] = C64 ? d64.dg[i] : acc.dg[i].value() * ih2;
      } else {
        Acc<double> acc;
        acc_zero(acc);
        boundary_pairs<false>(t, node, lb, st, mp, mp32, acc);
        v[0] = acc.L0;
        for (int i = 0; i < 3; ++i) v[1 + i] = acc.L1[i], v[4 + i] = acc.dg[i];
      }
      for (int i = 0; i < 7; ++i) res[lb * 7 + i] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int l = leaf_cell<MIXED>(q, threadIdx.x);
      L0[q] += res[l * 7];
      for (int i = 0; i < 3; ++i) L1[q][i] += res[l * 7 + 1 + i], dg[q][i] = res[l * 7 + 4 + i];
    }
  }
  const int64_t NC = t.NC;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int64_t tgt = (int64_t)node * 512 + leaf_cell<MIXED>(q, threadIdx.x);
    loc[G_L0 * NC + tgt] = L0[q];
    for (int i = 0; i < 3; ++i) loc[(G_L1 + i) * NC + tgt] = L1[q][i], loc[(G_DG + i) * NC + tgt] = dg[q][i];
  }
}

// Near item of the mixed path: the float64 near-field (P2P) sums of the 512 cells
// of one leaf node, from a float64 halo of the near radius, into
// nearf [4][NL] (leaf cell order; L0 and L1 in physical units), which L2P adds.
// Its work is float64 fused multiply-adds only, so it fills the float64 pipe while
// the float32 items of the same SM use the FMA pipe.
__device__ __forceinline__ void near_item(const DevTree& t, int node, const Stencils& st,
                                          const double* __restrict__ mp, double* __restrict__ nearf, int64_t NL,
                                          unsigned char* smem) {
  const HaloGeom gn = near_geom(st.near_radius);
  __shared__ int nleaf_n[27];
  load_leaf_neighbours(t, node, nleaf_n);
  double* halo = reinterpret_cast<double*>(smem);
  stage_halo(gn, nleaf_n, mp, halo);
  __syncthreads();
  const int lvl = t.level[node];
  const double ih = 1.0 / t.h[lvl], ih2 = ih * ih;
  const int64_t lid = t.leaf_id[node];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    int p, zh, a, b, c;
    cell_of(half, threadIdx.x, p, zh, a, b, c);
    const int2* __restrict__ nr = st.leaf_near + p * st.n_near;
    const int lane = (a >> 1) + gn.PY * (b >> 1) + gn.PZ * (c >> 1);
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    // entries come in (d, -d) pairs; kappa(-d) = (kappa0(d), -kappa1(d)), so a pair
    // takes one sum and one difference of its masses and four fused multiply-adds
    // (six float64 operations for two pairs instead of eight)
#pragma unroll 2
    for (int s = 0; s < st.n_near; s += 2) {
      const int2 e = __ldg(nr + s), f = __ldg(nr + s + 1);
      const double mp_ = halo[lane + e.x], mm = halo[lane + f.x];
      const double2* kp = reinterpret_cast<const double2*>(st.kappa + e.y);
      const double2 ka = __ldg(kp), kb = __ldg(kp + 1);
      const double sum = mp_ + mm, dif = mp_ - mm;
      s0 = fma(sum, ka.x, s0);
      s1 = fma(dif, ka.y, s1);
      s2 = fma(dif, kb.x, s2);
      s3 = fma(dif, kb.y, s3);
    }
    const int64_t k = lid * 512 + a + 8 * b + 64 * c;
    nearf[k] = s0 * ih;
    nearf[NL + k] = s1 * ih2;
    nearf[2 * NL + k] = s2 * ih2;
    nearf[3 * NL + k] = s3 * ih2;
  }
}

}  // namespace items
}  // namespace octo
