// Mixed-precision far field: the same-level M2L into interior cells and the
// leaf-leaf M2L part of the leaf convolution run in float32 with Kahan-compensated
// sums folded into float64 at the end; the leaf P2P near field stays in float64.
// Operands are in cell-width units of their level (see device.cuh), so the float32
// range is independent of the physical units, and results are scaled back by
// 1 / h^(n+1) in float64.
#include "kernels.h"

namespace octo {

namespace {

__device__ __forceinline__ void parity_cell32(int cls0, int tid, int& p, int& a, int& b, int& c) {
  const int w = tid >> 5, lane = tid & 31;
  p = cls0 + (w >> 1);
  const int q = ((w & 1) << 5) + lane;
  a = 2 * (q & 3) + (p & 1);
  b = 2 * ((q >> 2) & 3) + ((p >> 1) & 1);
  c = 2 * (q >> 4) + (p >> 2);
}

__device__ __forceinline__ void unpack32(int e, int& dx, int& dy, int& dz) {
  dx = (int)(int8_t)(e & 0xff);
  dy = (int)(int8_t)((e >> 8) & 0xff);
  dz = (int)(int8_t)((e >> 16) & 0xff);
}

// Interior targets, all same-level sources in the parity stencil.  The relative
// position uses node-centre coordinates: R = x_A - (x_B + 8 o) for a source in
// neighbour slot o (cell-width units).
__global__ void __launch_bounds__(256) k_m2l_f32(DevTree t, const int* __restrict__ nodes, Stencils st,
                                                  const float* __restrict__ mp32, double* __restrict__ loc) {
  const int node = nodes[blockIdx.x >> 1];
  int p, a, b, c;
  parity_cell32((blockIdx.x & 1) * 4, threadIdx.x, p, a, b, c);
  const int lvl = t.level[node];
  const int64_t NC = t.NC;
  const int64_t tgt = (int64_t)node * 512 + a + 8 * b + 64 * c;
  const float xA0 = mp32[(F_X + 0) * NC + tgt], xA1 = mp32[(F_X + 1) * NC + tgt], xA2 = mp32[(F_X + 2) * NC + tgt];
  float Oh[10], tOh[3];
  {
    const float inv_m = 1.0f / mp32[tgt];
    for (int i = 0; i < 10; ++i) Oh[i] = mp32[(F_O + i) * NC + tgt] * inv_m;
    tOh[0] = Oh[0] + Oh[3] + Oh[5];
    tOh[1] = Oh[1] + Oh[6] + Oh[8];
    tOh[2] = Oh[2] + Oh[7] + Oh[9];
  }
  const int* tab = lvl == 0 ? st.root : st.parity + p * st.n_st;
  const int ntab = lvl == 0 ? st.n_root : st.n_st;
  const int* nb = t.nbr + 27 * node;
  Acc<KF> acc;
  acc_zero(acc);
  for (int s = 0; s < ntab; ++s) {
    int dx, dy, dz;
    unpack32(__ldg(tab + s), dx, dy, dz);
    const int sa = a + dx, sb = b + dy, sc = c + dz;
    const int ox = sa >> 3, oy = sb >> 3, oz = sc >> 3;
    const int snode = __ldg(nb + (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1));
    if (snode < 0) continue;
    const int64_t src = (int64_t)snode * 512 + (sa & 7) + 8 * (sb & 7) + 64 * (sc & 7);
    const float R0 = xA0 - (__ldg(mp32 + (F_X + 0) * NC + src) + 8.0f * (float)ox);
    const float R1 = xA1 - (__ldg(mp32 + (F_X + 1) * NC + src) + 8.0f * (float)oy);
    const float R2 = xA2 - (__ldg(mp32 + (F_X + 2) * NC + src) + 8.0f * (float)oz);
    const float m = __ldg(mp32 + src);
    float Q[6], O[10];
    for (int i = 0; i < 6; ++i) Q[i] = __ldg(mp32 + (F_Q + i) * NC + src);
    for (int i = 0; i < 10; ++i) O[i] = __ldg(mp32 + (F_O + i) * NC + src);
    const float rinv = rsqrt_f32(fmaf(R0, R0, fmaf(R1, R1, R2 * R2)));
    m2l_pair<true, true>(R0, R1, R2, m, Q, O, Oh, tOh, rinv, acc);
  }
  // fold into float64, add the deferred delta terms, undo the cell-width scaling
  Acc<double> d;
  d.L0 = acc.L0.value();
  for (int i = 0; i < 3; ++i) d.L1[i] = acc.L1[i].value(), d.dg[i] = acc.dg[i].value(), d.V[i] = acc.V[i].value();
  for (int i = 0; i < 6; ++i) d.L2[i] = acc.L2[i].value();
  for (int i = 0; i < 10; ++i) d.L3[i] = acc.L3[i].value();
  d.W = acc.W.value();
  acc_finish(d);
  const double ih = 1.0 / t.h[lvl], ih2 = ih * ih, ih3 = ih2 * ih, ih4 = ih2 * ih2;
  loc[G_L0 * NC + tgt] = d.L0 * ih;
  for (int i = 0; i < 3; ++i) loc[(G_L1 + i) * NC + tgt] = d.L1[i] * ih2;
  for (int i = 0; i < 6; ++i) loc[(G_L2 + i) * NC + tgt] = d.L2[i] * ih3;
  for (int i = 0; i < 10; ++i) loc[(G_L3 + i) * NC + tgt] = d.L3[i] * ih4;
  for (int i = 0; i < 3; ++i) loc[(G_DG + i) * NC + tgt] = d.dg[i] * ih2;
}

// Leaf convolution, mixed: the far part (parity or root stencil) sums m * kappa
// in float32 with Kahan compensation from a float32 mass halo; the near part (P2P)
// sums in float64 from a float64 halo of the near radius.
__global__ void __launch_bounds__(512) k_leaf_conv_mixed(DevTree t, const int* __restrict__ nodes, Stencils st,
                                                         const double* __restrict__ mp, double* __restrict__ loc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int node = nodes[blockIdx.x];
  const int R = st.radius, H = 8 + 2 * R, H2 = H * H, W = 2 * R + 1;
  const int RN = st.near_radius, HN = 8 + 2 * RN, HN2 = HN * HN, WN = 2 * R + 1;
  double* halo64 = reinterpret_cast<double*>(smem);
  float* halo32 = reinterpret_cast<float*>(smem + sizeof(double) * HN2 * HN);
  const int* nb = t.nbr + 27 * node;
  for (int i = threadIdx.x; i < H2 * H; i += blockDim.x) {
    const int hx = i % H - R, hy = (i / H) % H - R, hz = i / H2 - R;
    const int slot = ((hx >> 3) + 1) + 3 * ((hy >> 3) + 1) + 9 * ((hz >> 3) + 1);
    const int sn = nb[slot];
    double m = 0.0;
    if (sn >= 0 && t.children[8 * sn] < 0) m = mp[(int64_t)sn * 512 + (hx & 7) + 8 * (hy & 7) + 64 * (hz & 7)];
    halo32[i] = (float)m;
    if (hx >= -RN && hx < 8 + RN && hy >= -RN && hy < 8 + RN && hz >= -RN && hz < 8 + RN)
      halo64[(hx + RN) + HN * (hy + RN) + HN2 * (hz + RN)] = m;
  }
  __syncthreads();
  int p, a, b, c;
  parity_cell32(0, threadIdx.x, p, a, b, c);
  const int lvl = t.level[node];
  const int kbase = R + W * R + W * W * R;
  // far part, float32 compensated
  KF f0, f1, f2, f3;
  f0 = 0.0f;
  f1 = 0.0f;
  f2 = 0.0f;
  f3 = 0.0f;
  {
    const int base = (a + R) + H * (b + R) + H2 * (c + R);
    const int* tab = lvl == 0 ? st.root : st.parity + p * st.n_st;
    const int ntab = lvl == 0 ? st.n_root : st.n_st;
    for (int s = 0; s < ntab; ++s) {
      int dx, dy, dz;
      unpack32(__ldg(tab + s), dx, dy, dz);
      const float m = halo32[base + dx + H * dy + H2 * dz];
      const float4 k = __ldg(st.kappa32 + kbase + dx + W * dy + W * W * dz);
      f0.add(m * k.x);
      f1.add(m * k.y);
      f2.add(m * k.z);
      f3.add(m * k.w);
    }
  }
  // near part, float64
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  {
    const int base = (a + RN) + HN * (b + RN) + HN2 * (c + RN);
    (void)WN;
    for (int s = 0; s < st.n_near; ++s) {
      int dx, dy, dz;
      unpack32(__ldg(st.near_ + s), dx, dy, dz);
      const double m = halo64[base + dx + HN * dy + HN2 * dz];
      const double2* kp = reinterpret_cast<const double2*>(st.kappa + kbase + dx + W * dy + W * W * dz);
      const double2 ka = __ldg(kp), kb = __ldg(kp + 1);
      s0 = fma(m, ka.x, s0);
      s1 = fma(m, ka.y, s1);
      s2 = fma(m, kb.x, s2);
      s3 = fma(m, kb.y, s3);
    }
  }
  const double ih = 1.0 / t.h[lvl];
  const int64_t NC = t.NC;
  const int64_t tgt = (int64_t)node * 512 + a + 8 * b + 64 * c;
  loc[G_L0 * NC + tgt] = (s0 + f0.value()) * ih;
  loc[(G_L1 + 0) * NC + tgt] = (s1 + f1.value()) * (ih * ih);
  loc[(G_L1 + 1) * NC + tgt] = (s2 + f2.value()) * (ih * ih);
  loc[(G_L1 + 2) * NC + tgt] = (s3 + f3.value()) * (ih * ih);
  loc[(G_DG + 0) * NC + tgt] = 0.0;
  loc[(G_DG + 1) * NC + tgt] = 0.0;
  loc[(G_DG + 2) * NC + tgt] = 0.0;
}

}  // namespace

cudaError_t configure_kernels_mixed() {
  return cudaFuncSetAttribute(k_leaf_conv_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_m2l_interior_f32(const DevTree& t, const int* nodes, int n, const Stencils& st, const float* mp32,
                                    double* loc, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_m2l_f32<<<2 * n, 256, 0, s>>>(t, nodes, st, mp32, loc);
  return cudaGetLastError();
}

cudaError_t launch_leaf_conv_mixed(const DevTree& t, const int* nodes, int n, const Stencils& st, const double* mp,
                                   double* loc, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int H = 8 + 2 * st.radius, HN = 8 + 2 * st.near_radius;
  const size_t smem = sizeof(double) * HN * HN * HN + sizeof(float) * H * H * H;
  k_leaf_conv_mixed<<<n, 512, smem, s>>>(t, nodes, st, mp, loc);
  return cudaGetLastError();
}

}  // namespace octo
