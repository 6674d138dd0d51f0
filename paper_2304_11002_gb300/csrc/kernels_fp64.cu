// Tree passes of the solve (paper Section VII-C): bottom-up (P2M, M2M) and
// top-down (L2L with L2P fused at leaf nodes), in float64 for both precision
// modes.  The same-level interactions are in items.cuh / kernels_interact.cu and
// kernels_boundary.cu.
#include "kernels.h"

namespace octo {

namespace {

// ---------------------------------------------------------------- init / P2M
__global__ void k_init_leaf(DevTree t, const int* __restrict__ nodes, double* __restrict__ mp,
                            float* __restrict__ mp32) {
  const int node = nodes[blockIdx.x];
  const double h = t.h[t.level[node]];
  const int64_t NC = t.NC;
  const int* ijk = t.ijk;
  for (int l = threadIdx.x; l < 512; l += blockDim.x) {
    const int64_t cell = (int64_t)node * 512 + l;
    const int a = l & 7, b = (l >> 3) & 7, c = l >> 6;
    mp[(F_X + 0) * NC + cell] = t.origin[0] + h * ((double)(8 * ijk[3 * node + 0] + a) + 0.5);
    mp[(F_X + 1) * NC + cell] = t.origin[1] + h * ((double)(8 * ijk[3 * node + 1] + b) + 0.5);
    mp[(F_X + 2) * NC + cell] = t.origin[2] + h * ((double)(8 * ijk[3 * node + 2] + c) + 0.5);
    for (int f = F_Q; f < N_MP; ++f) mp[f * NC + cell] = 0.0;
    if (mp32) {  // cell centre relative to the node centre, in cell widths (exact)
      float* r = mp32 + mp32_index(node, a, b, c, 0);  // field f at r + mp32_index(.., f) - mp32_index(.., 0)
      for (int f = 0; f < N_MP; ++f) {
        const float v = f == F_X + 0 ? (float)a - 3.5f : f == F_X + 1 ? (float)b - 3.5f : f == F_X + 2 ? (float)c - 3.5f : 0.0f;
        r[4 * kMp32Pairs * (f >> 1) + 2 * (f & 1)] = v;
      }
    }
  }
}

// P2M: a leaf cell is one monopole m = rho h^3 at its centre (Section IV-C).
// The density must be finite and positive (centres of mass divide by the mass):
// any other value sets kErrDensity in *err, read back by octo_fmm_stats and
// octo_fmm_forces_host.  The check changes no result.  Blocks of 256 threads run
// two full passes over the 512 cells, so every warp votes with all lanes.
__global__ void k_p2m(DevTree t, const int* __restrict__ nodes, const double* __restrict__ rho,
                      double* __restrict__ mp, float* __restrict__ mp32, int* __restrict__ err) {
  const int node = nodes[blockIdx.x];
  const double h3 = t.h3[t.level[node]];
  const int64_t lid = t.leaf_id[node];
  for (int l = threadIdx.x; l < 512; l += blockDim.x) {
    const double r = rho[lid * 512 + l];
    const double m = r * h3;
    mp[(int64_t)node * 512 + l] = m;
    if (mp32) mp32[mp32_index(node, l & 7, (l >> 3) & 7, l >> 6, F_M)] = (float)m;
    const bool bad = !(r > 0.0 && isfinite(r));  // NaN, <= 0 or +inf
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kErrDensity);
  }
}

// ---------------------------------------------------------------- M2M
// Parent cell from its 2x2x2 child cells (parallel-axis rule about the centre of
// mass): m = sum m_c, X = sum m_c X_c / m, d_c = X_c - X,
// M2 = sum (M2_c + m_c d d), M3 = sum (M3_c + 3 sym(M2_c d) + m_c d d d).
// One thread per parent cell, blocks of 64 threads (eight per node): the pass is
// float64-bound, and a coarse level of one or a few nodes then still spreads over
// eight SMs per node instead of two.  Registers capped at the same 80 as three
// 256-thread blocks per SM; the children loop of the moments stays rolled.
constexpr int kM2MThreads = 64;
__global__ void __launch_bounds__(kM2MThreads, 12) k_m2m(DevTree t, int node_begin, double* __restrict__ mp,
                                                        float* __restrict__ mp32) {
  const int node = node_begin + (blockIdx.x >> 3);
  if (t.children[8 * node] < 0) return;
  const int l = ((blockIdx.x & 7) * kM2MThreads) + threadIdx.x;
  const int a = l & 7, b = (l >> 3) & 7, c = l >> 6;
  const int o = (a >> 2) + 2 * (b >> 2) + 4 * (c >> 2);
  const int ch = t.children[8 * node + o];
  // a leaf child node's cells are point masses (P2M): their moments are zero, so
  // they are neither read nor added
  const bool leaf_child = t.children[8 * ch] < 0;
  const int64_t NC = t.NC;
  // child cell e = ex + 2 ey + 4 ez of this parent cell
  const int64_t c0 = (int64_t)ch * 512 + 2 * (a & 3) + 8 * 2 * (b & 3) + 64 * 2 * (c & 3);
  auto child = [c0](int e) { return c0 + (e & 1) + 8 * ((e >> 1) & 1) + 64 * (e >> 2); };
  double m = 0, X0 = 0, X1 = 0, X2 = 0;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int64_t ce = child(e);
    const double mc = mp[ce];
    m += mc;
    X0 += mc * mp[(F_X + 0) * NC + ce];
    X1 += mc * mp[(F_X + 1) * NC + ce];
    X2 += mc * mp[(F_X + 2) * NC + ce];
  }
  X0 /= m;
  X1 /= m;
  X2 /= m;
  double Q[6] = {0, 0, 0, 0, 0, 0}, O[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (leaf_child) {
    // point-mass children: M2 = sum m d d, M3 = sum m d d d (the general expressions
    // below with zero child moments and their zero terms left out; fused
    // multiply-adds may round differently)
#pragma unroll 1
    for (int e = 0; e < 8; ++e) {
      const int64_t ce = child(e);
      const double mc = mp[ce];
      const double d0 = mp[(F_X + 0) * NC + ce] - X0;
      const double d1 = mp[(F_X + 1) * NC + ce] - X1;
      const double d2 = mp[(F_X + 2) * NC + ce] - X2;
      const double md0 = mc * d0, md1 = mc * d1, md2 = mc * d2;
      Q[0] += md0 * d0;
      Q[1] += md0 * d1;
      Q[2] += md0 * d2;
      Q[3] += md1 * d1;
      Q[4] += md1 * d2;
      Q[5] += md2 * d2;
      O[0] += md0 * d0 * d0;
      O[1] += md0 * d0 * d1;
      O[2] += md0 * d0 * d2;
      O[3] += md0 * d1 * d1;
      O[4] += md0 * d1 * d2;
      O[5] += md0 * d2 * d2;
      O[6] += md1 * d1 * d1;
      O[7] += md1 * d1 * d2;
      O[8] += md1 * d2 * d2;
      O[9] += md2 * d2 * d2;
    }
  } else {
#pragma unroll 1
  for (int e = 0; e < 8; ++e) {
    const int64_t ce = child(e);
    const double mc = mp[ce];
    const double d0 = mp[(F_X + 0) * NC + ce] - X0;
    const double d1 = mp[(F_X + 1) * NC + ce] - X1;
    const double d2 = mp[(F_X + 2) * NC + ce] - X2;
    double q[6];
    for (int i = 0; i < 6; ++i) q[i] = mp[(F_Q + i) * NC + ce];
    double oc[10];
    for (int i = 0; i < 10; ++i) oc[i] = mp[(F_O + i) * NC + ce];
    const double md0 = mc * d0, md1 = mc * d1, md2 = mc * d2;
    Q[0] += q[0] + md0 * d0;
    Q[1] += q[1] + md0 * d1;
    Q[2] += q[2] + md0 * d2;
    Q[3] += q[3] + md1 * d1;
    Q[4] += q[4] + md1 * d2;
    Q[5] += q[5] + md2 * d2;
    // 3 sym(q d)_abc = q_ab d_c + q_ac d_b + q_bc d_a
    O[0] += oc[0] + 3.0 * q[0] * d0 + md0 * d0 * d0;                    // xxx
    O[1] += oc[1] + q[0] * d1 + 2.0 * q[1] * d0 + md0 * d0 * d1;        // xxy
    O[2] += oc[2] + q[0] * d2 + 2.0 * q[2] * d0 + md0 * d0 * d2;        // xxz
    O[3] += oc[3] + 2.0 * q[1] * d1 + q[3] * d0 + md0 * d1 * d1;        // xyy
    O[4] += oc[4] + q[1] * d2 + q[2] * d1 + q[4] * d0 + md0 * d1 * d2;  // xyz
    O[5] += oc[5] + 2.0 * q[2] * d2 + q[5] * d0 + md0 * d2 * d2;        // xzz
    O[6] += oc[6] + 3.0 * q[3] * d1 + md1 * d1 * d1;                    // yyy
    O[7] += oc[7] + q[3] * d2 + 2.0 * q[4] * d1 + md1 * d1 * d2;        // yyz
    O[8] += oc[8] + 2.0 * q[4] * d2 + q[5] * d1 + md1 * d2 * d2;        // yzz
    O[9] += oc[9] + 3.0 * q[5] * d2 + md2 * d2 * d2;                    // zzz
  }
  }
  const int64_t pc = (int64_t)node * 512 + l;
  mp[pc] = m;
  mp[(F_X + 0) * NC + pc] = X0;
  mp[(F_X + 1) * NC + pc] = X1;
  mp[(F_X + 2) * NC + pc] = X2;
  for (int i = 0; i < 6; ++i) mp[(F_Q + i) * NC + pc] = Q[i];
  for (int i = 0; i < 10; ++i) mp[(F_O + i) * NC + pc] = O[i];
  if (mp32) {  // float32 copy in cell-width units (see device.cuh)
    const int lv = t.level[node];
    const double h = t.h[lv], ih = 1.0 / h, ih2 = ih * ih, ih3 = ih2 * ih;
    const double c0 = t.origin[0] + h * (8.0 * t.ijk[3 * node + 0] + 4.0);
    const double c1 = t.origin[1] + h * (8.0 * t.ijk[3 * node + 1] + 4.0);
    const double c2 = t.origin[2] + h * (8.0 * t.ijk[3 * node + 2] + 4.0);
    float v[N_MP];
    v[F_M] = (float)m;
    v[F_X + 0] = (float)((X0 - c0) * ih);
    v[F_X + 1] = (float)((X1 - c1) * ih);
    v[F_X + 2] = (float)((X2 - c2) * ih);
    for (int i = 0; i < 6; ++i) v[F_Q + i] = (float)(Q[i] * ih2);
    for (int i = 0; i < 10; ++i) v[F_O + i] = (float)(O[i] * ih3);
    float* r = mp32 + mp32_index(node, a, b, c, 0);
    for (int f = 0; f < N_MP; ++f) r[4 * kMp32Pairs * (f >> 1) + 2 * (f & 1)] = v[f];
  }
}

// ---------------------------------------------------------------- L2L + L2P
// Child expansion += parent expansion shifted by delta = X_child - X_parent
// (exact for the cubic Taylor polynomial), dg carried down unshifted.  At leaf
// nodes the result is evaluated at the cell itself (L2P):
//   phi = L0,  g = -L1 + dg  (plus the near-field sums when they are kept apart).
// One thread per cell, 128-thread blocks (four per node) with three resident per
// SM: the polynomial shift keeps ~160 float64 registers live, which 256-thread
// blocks at two per SM (128 registers) spilled.
constexpr int kL2LThreads = 128;
__global__ void __launch_bounds__(kL2LThreads, 3) k_l2l(DevTree t, int node_begin, const double* __restrict__ mp,
                                                       double* __restrict__ loc, double* __restrict__ phi,
                                                       double* __restrict__ g, int64_t NL,
                                                       const double* __restrict__ nearf) {
  const int node = node_begin + (blockIdx.x >> 2);
  const int l = ((blockIdx.x & 3) * kL2LThreads) + threadIdx.x;
  const int64_t NC = t.NC;
  const int64_t cell = (int64_t)node * 512 + l;
  const bool leaf = t.children[8 * node] < 0;
  double L0 = loc[G_L0 * NC + cell];
  double L1[3], L2[6], L3[10], dg[3];
  for (int i = 0; i < 3; ++i) L1[i] = loc[(G_L1 + i) * NC + cell], dg[i] = loc[(G_DG + i) * NC + cell];
  if (!leaf) {
    for (int i = 0; i < 6; ++i) L2[i] = loc[(G_L2 + i) * NC + cell];
    for (int i = 0; i < 10; ++i) L3[i] = loc[(G_L3 + i) * NC + cell];
  }
  const int par = t.parent[node];
  if (par >= 0) {
    const int o = t.octant[node];
    const int a = l & 7, b = (l >> 3) & 7, c = l >> 6;
    const int64_t pc = (int64_t)par * 512 + (4 * (o & 1) + (a >> 1)) + 8 * (4 * ((o >> 1) & 1) + (b >> 1)) +
                       64 * (4 * (o >> 2) + (c >> 1));
    const double d0 = mp[(F_X + 0) * NC + cell] - mp[(F_X + 0) * NC + pc];
    const double d1 = mp[(F_X + 1) * NC + cell] - mp[(F_X + 1) * NC + pc];
    const double d2 = mp[(F_X + 2) * NC + cell] - mp[(F_X + 2) * NC + pc];
    double P1[3], P2[6], P3[10];
    const double P0 = loc[G_L0 * NC + pc];
    for (int i = 0; i < 3; ++i) P1[i] = loc[(G_L1 + i) * NC + pc];
    for (int i = 0; i < 6; ++i) P2[i] = loc[(G_L2 + i) * NC + pc];
    for (int i = 0; i < 10; ++i) P3[i] = loc[(G_L3 + i) * NC + pc];
    for (int i = 0; i < 3; ++i) dg[i] += loc[(G_DG + i) * NC + pc];
    // (L3 . d)_ab
    const double T0 = P3[0] * d0 + P3[1] * d1 + P3[2] * d2;  // xx
    const double T1 = P3[1] * d0 + P3[3] * d1 + P3[4] * d2;  // xy
    const double T2 = P3[2] * d0 + P3[4] * d1 + P3[5] * d2;  // xz
    const double T3 = P3[3] * d0 + P3[6] * d1 + P3[7] * d2;  // yy
    const double T4 = P3[4] * d0 + P3[7] * d1 + P3[8] * d2;  // yz
    const double T5 = P3[5] * d0 + P3[8] * d1 + P3[9] * d2;  // zz
    // (L3 . d d)_a and (L2 . d)_a
    const double U0 = T0 * d0 + T1 * d1 + T2 * d2;
    const double U1 = T1 * d0 + T3 * d1 + T4 * d2;
    const double U2 = T2 * d0 + T4 * d1 + T5 * d2;
    const double S0 = P2[0] * d0 + P2[1] * d1 + P2[2] * d2;
    const double S1 = P2[1] * d0 + P2[3] * d1 + P2[4] * d2;
    const double S2 = P2[2] * d0 + P2[4] * d1 + P2[5] * d2;
    L0 += P0 + (P1[0] * d0 + P1[1] * d1 + P1[2] * d2) + 0.5 * (S0 * d0 + S1 * d1 + S2 * d2) +
          (U0 * d0 + U1 * d1 + U2 * d2) * (1.0 / 6.0);
    L1[0] += P1[0] + S0 + 0.5 * U0;
    L1[1] += P1[1] + S1 + 0.5 * U1;
    L1[2] += P1[2] + S2 + 0.5 * U2;
    if (!leaf) {
      L2[0] += P2[0] + T0;
      L2[1] += P2[1] + T1;
      L2[2] += P2[2] + T2;
      L2[3] += P2[3] + T3;
      L2[4] += P2[4] + T4;
      L2[5] += P2[5] + T5;
      for (int i = 0; i < 10; ++i) L3[i] += P3[i];
    }
  }
  if (leaf) {
    const int64_t k = (int64_t)t.leaf_id[node] * 512 + l;
    if (nearf) {  // near-field sums kept apart by the mixed-precision interaction phase
      L0 += nearf[k];
      for (int i = 0; i < 3; ++i) L1[i] += nearf[(1 + i) * NL + k];
    }
    phi[k] = L0;
    for (int i = 0; i < 3; ++i) g[i * NL + k] = -L1[i] + dg[i];
  } else {
    loc[G_L0 * NC + cell] = L0;
    for (int i = 0; i < 3; ++i) loc[(G_L1 + i) * NC + cell] = L1[i], loc[(G_DG + i) * NC + cell] = dg[i];
    for (int i = 0; i < 6; ++i) loc[(G_L2 + i) * NC + cell] = L2[i];
    for (int i = 0; i < 10; ++i) loc[(G_L3 + i) * NC + cell] = L3[i];
  }
}

}  // namespace

// ---------------------------------------------------------------- launchers
cudaError_t launch_init_leaf(const DevTree& t, const int* leaf_nodes, int n, double* mp, float* mp32,
                             cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_init_leaf<<<n, 256, 0, s>>>(t, leaf_nodes, mp, mp32);
  return cudaGetLastError();
}

cudaError_t launch_p2m(const DevTree& t, const int* leaf_nodes, int n, const double* rho, double* mp, float* mp32,
                       int* err, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_p2m<<<n, 256, 0, s>>>(t, leaf_nodes, rho, mp, mp32, err);
  return cudaGetLastError();
}

cudaError_t launch_m2m(const DevTree& t, int b, int e, double* mp, float* mp32, cudaStream_t s) {
  if (e <= b) return cudaSuccess;
  k_m2m<<<(512 / kM2MThreads) * (e - b), kM2MThreads, 0, s>>>(t, b, mp, mp32);
  return cudaGetLastError();
}

cudaError_t launch_l2l(const DevTree& t, int b, int e, const double* mp, double* loc, double* phi, double* g,
                       int64_t NL, const double* nearf, cudaStream_t s) {
  if (e <= b) return cudaSuccess;
  k_l2l<<<(512 / kL2LThreads) * (e - b), kL2LThreads, 0, s>>>(t, b, mp, loc, phi, g, NL, nearf);
  return cudaGetLastError();
}

}  // namespace octo
