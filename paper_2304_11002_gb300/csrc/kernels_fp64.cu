// Float64 kernels of the three solve phases (paper Section VII-C): bottom-up
// (P2M, M2M), same-level interactions (M2L with the angular-momentum correction,
// the leaf-level monopole convolution that also carries P2P, cross-level pairs)
// and top-down (L2L with L2P fused at leaf nodes).
#include "kernels.h"

namespace octo {

namespace {

// Cell (a, b, c) handled by thread `tid` of a block covering `ncls` parity classes
// starting at class `cls0`: each warp holds 32 cells of one parity class
// (p = px + 2 py + 4 pz, 64 cells per class per node), so stencil offsets are
// warp-uniform.
__device__ __forceinline__ void parity_cell(int cls0, int tid, int& p, int& a, int& b, int& c) {
  const int w = tid >> 5, lane = tid & 31;
  p = cls0 + (w >> 1);
  const int q = ((w & 1) << 5) + lane;
  a = 2 * (q & 3) + (p & 1);
  b = 2 * ((q >> 2) & 3) + ((p >> 1) & 1);
  c = 2 * (q >> 4) + (p >> 2);
}

__device__ __forceinline__ void unpack(int e, int& dx, int& dy, int& dz) {
  dx = (int)(int8_t)(e & 0xff);
  dy = (int)(int8_t)((e >> 8) & 0xff);
  dz = (int)(int8_t)((e >> 16) & 0xff);
}

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
      mp32[(F_X + 0) * NC + cell] = (float)a - 3.5f;
      mp32[(F_X + 1) * NC + cell] = (float)b - 3.5f;
      mp32[(F_X + 2) * NC + cell] = (float)c - 3.5f;
      for (int f = F_Q; f < N_MP; ++f) mp32[f * NC + cell] = 0.0f;
    }
  }
}

// P2M: a leaf cell is one monopole m = rho h^3 at its centre (Section IV-C).
__global__ void k_p2m(DevTree t, const int* __restrict__ nodes, const double* __restrict__ rho,
                      double* __restrict__ mp, float* __restrict__ mp32) {
  const int node = nodes[blockIdx.x];
  const double h3 = t.h3[t.level[node]];
  const int64_t lid = t.leaf_id[node];
  for (int l = threadIdx.x; l < 512; l += blockDim.x) {
    const double m = rho[lid * 512 + l] * h3;
    mp[(int64_t)node * 512 + l] = m;
    if (mp32) mp32[(int64_t)node * 512 + l] = (float)m;
  }
}

// ---------------------------------------------------------------- M2M
// Parent cell from its 2x2x2 child cells (parallel-axis rule about the centre of
// mass): m = sum m_c, X = sum m_c X_c / m, d_c = X_c - X,
// M2 = sum (M2_c + m_c d d), M3 = sum (M3_c + 3 sym(M2_c d) + m_c d d d).
__global__ void __launch_bounds__(256) k_m2m(DevTree t, int node_begin, double* __restrict__ mp,
                                             float* __restrict__ mp32) {
  const int node = node_begin + (blockIdx.x >> 1);
  if (t.children[8 * node] < 0) return;
  const int l = ((blockIdx.x & 1) << 8) + threadIdx.x;
  const int a = l & 7, b = (l >> 3) & 7, c = l >> 6;
  const int o = (a >> 2) + 2 * (b >> 2) + 4 * (c >> 2);
  const int ch = t.children[8 * node + o];
  const int64_t NC = t.NC;
  int64_t cc[8];
  for (int e = 0; e < 8; ++e) {
    const int ca = 2 * (a & 3) + (e & 1), cb = 2 * (b & 3) + ((e >> 1) & 1), cz = 2 * (c & 3) + (e >> 2);
    cc[e] = (int64_t)ch * 512 + ca + 8 * cb + 64 * cz;
  }
  double m = 0, X0 = 0, X1 = 0, X2 = 0;
  for (int e = 0; e < 8; ++e) m += mp[cc[e]];
  for (int e = 0; e < 8; ++e) {
    const double mc = mp[cc[e]];
    X0 += mc * mp[(F_X + 0) * NC + cc[e]];
    X1 += mc * mp[(F_X + 1) * NC + cc[e]];
    X2 += mc * mp[(F_X + 2) * NC + cc[e]];
  }
  X0 /= m;
  X1 /= m;
  X2 /= m;
  double Q[6] = {0, 0, 0, 0, 0, 0}, O[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int e = 0; e < 8; ++e) {
    const double mc = mp[cc[e]];
    const double d0 = mp[(F_X + 0) * NC + cc[e]] - X0;
    const double d1 = mp[(F_X + 1) * NC + cc[e]] - X1;
    const double d2 = mp[(F_X + 2) * NC + cc[e]] - X2;
    double q[6];
    for (int i = 0; i < 6; ++i) q[i] = mp[(F_Q + i) * NC + cc[e]];
    const double md0 = mc * d0, md1 = mc * d1, md2 = mc * d2;
    Q[0] += q[0] + md0 * d0;
    Q[1] += q[1] + md0 * d1;
    Q[2] += q[2] + md0 * d2;
    Q[3] += q[3] + md1 * d1;
    Q[4] += q[4] + md1 * d2;
    Q[5] += q[5] + md2 * d2;
    // 3 sym(q d)_abc = q_ab d_c + q_ac d_b + q_bc d_a
    O[0] += mp[(F_O + 0) * NC + cc[e]] + 3.0 * q[0] * d0 + md0 * d0 * d0;                    // xxx
    O[1] += mp[(F_O + 1) * NC + cc[e]] + q[0] * d1 + 2.0 * q[1] * d0 + md0 * d0 * d1;        // xxy
    O[2] += mp[(F_O + 2) * NC + cc[e]] + q[0] * d2 + 2.0 * q[2] * d0 + md0 * d0 * d2;        // xxz
    O[3] += mp[(F_O + 3) * NC + cc[e]] + 2.0 * q[1] * d1 + q[3] * d0 + md0 * d1 * d1;        // xyy
    O[4] += mp[(F_O + 4) * NC + cc[e]] + q[1] * d2 + q[2] * d1 + q[4] * d0 + md0 * d1 * d2;  // xyz
    O[5] += mp[(F_O + 5) * NC + cc[e]] + 2.0 * q[2] * d2 + q[5] * d0 + md0 * d2 * d2;        // xzz
    O[6] += mp[(F_O + 6) * NC + cc[e]] + 3.0 * q[3] * d1 + md1 * d1 * d1;                    // yyy
    O[7] += mp[(F_O + 7) * NC + cc[e]] + q[3] * d2 + 2.0 * q[4] * d1 + md1 * d1 * d2;        // yyz
    O[8] += mp[(F_O + 8) * NC + cc[e]] + 2.0 * q[4] * d2 + q[5] * d1 + md1 * d2 * d2;        // yzz
    O[9] += mp[(F_O + 9) * NC + cc[e]] + 3.0 * q[5] * d2 + md2 * d2 * d2;                    // zzz
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
    mp32[pc] = (float)m;
    mp32[(F_X + 0) * NC + pc] = (float)((X0 - c0) * ih);
    mp32[(F_X + 1) * NC + pc] = (float)((X1 - c1) * ih);
    mp32[(F_X + 2) * NC + pc] = (float)((X2 - c2) * ih);
    for (int i = 0; i < 6; ++i) mp32[(F_Q + i) * NC + pc] = (float)(Q[i] * ih2);
    for (int i = 0; i < 10; ++i) mp32[(F_O + i) * NC + pc] = (float)(O[i] * ih3);
  }
}

// ---------------------------------------------------------------- M2L (general)
// Same-level M2L for every cell of a node over its parity stencil, sources from
// the 26 neighbouring subgrids.  Block = 256 threads = 4 parity classes; two
// blocks per node.
//  LEAF_TARGET = false: interior target nodes, all sources, results stored (=).
//  LEAF_TARGET = true : leaf target nodes, only sources in refined neighbour
//                       nodes (leaf-leaf pairs are in the convolution), added (+=).
template <bool LEAF_TARGET>
__global__ void __launch_bounds__(256) k_m2l(DevTree t, const int* __restrict__ nodes, Stencils st,
                                              const double* __restrict__ mp, double* __restrict__ loc) {
  const int node = nodes[blockIdx.x >> 1];
  int p, a, b, c;
  parity_cell((blockIdx.x & 1) * 4, threadIdx.x, p, a, b, c);
  const int lvl = t.level[node];
  const int64_t NC = t.NC;
  const int64_t tgt = (int64_t)node * 512 + a + 8 * b + 64 * c;
  const double XA0 = mp[(F_X + 0) * NC + tgt], XA1 = mp[(F_X + 1) * NC + tgt], XA2 = mp[(F_X + 2) * NC + tgt];
  double Oh[10], tOh[3];
  if (!LEAF_TARGET) {
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
    const int slot = ((sa >> 3) + 1) + 3 * ((sb >> 3) + 1) + 9 * ((sc >> 3) + 1);
    const int snode = __ldg(nb + slot);
    if (snode < 0) continue;
    if (LEAF_TARGET && __ldg(t.children + 8 * snode) < 0) continue;
    const int64_t src = (int64_t)snode * 512 + (sa & 7) + 8 * (sb & 7) + 64 * (sc & 7);
    const double R0 = XA0 - __ldg(mp + (F_X + 0) * NC + src);
    const double R1 = XA1 - __ldg(mp + (F_X + 1) * NC + src);
    const double R2 = XA2 - __ldg(mp + (F_X + 2) * NC + src);
    const double m = __ldg(mp + src);
    double Q[6], O[10];
    for (int i = 0; i < 6; ++i) Q[i] = __ldg(mp + (F_Q + i) * NC + src);
    for (int i = 0; i < 10; ++i) O[i] = __ldg(mp + (F_O + i) * NC + src);
    const double rinv = rsqrt_f64(fma(R0, R0, fma(R1, R1, R2 * R2)));
    m2l_pair<!LEAF_TARGET, !LEAF_TARGET>(R0, R1, R2, m, Q, O, Oh, tOh, rinv, acc);
  }
  if (!LEAF_TARGET) {
    acc_finish(acc);
    loc[G_L0 * NC + tgt] = acc.L0;
    for (int i = 0; i < 3; ++i) loc[(G_L1 + i) * NC + tgt] = acc.L1[i];
    for (int i = 0; i < 6; ++i) loc[(G_L2 + i) * NC + tgt] = acc.L2[i];
    for (int i = 0; i < 10; ++i) loc[(G_L3 + i) * NC + tgt] = acc.L3[i];
    for (int i = 0; i < 3; ++i) loc[(G_DG + i) * NC + tgt] = acc.dg[i];
  } else {
    loc[G_L0 * NC + tgt] += acc.L0;
    for (int i = 0; i < 3; ++i) loc[(G_L1 + i) * NC + tgt] += acc.L1[i];
    for (int i = 0; i < 3; ++i) loc[(G_DG + i) * NC + tgt] += acc.dg[i];
  }
}

// ---------------------------------------------------------------- leaf convolution
// Between two leaf cells of one level both expansions are monopoles at cell
// centres, so R = -d h for the stencil offset d and the M2L reduces to the exact
// point-mass field, identical in form to P2P:  L0 += -m / r,  L1 += -m D1 = m R / r^3.
// With kappa0(d) = -1/|d| and kappa1(d) = -d/|d|^3 (unit cell width):
//   L0 = (1/h) sum m kappa0,  L1 = (1/h^2) sum m kappa1
// over the far parity stencil (M2L) and the near offsets (P2P), with the masses of
// same-level leaf cells staged in shared memory (halo of radius R).
// Only L0, L1 (and dg = 0) of leaf cells are ever used; they are stored (=).
__global__ void __launch_bounds__(512) k_leaf_conv(DevTree t, const int* __restrict__ nodes, Stencils st,
                                                   const double* __restrict__ mp, double* __restrict__ loc) {
  extern __shared__ double halo[];
  const int node = nodes[blockIdx.x];
  const int R = st.radius, H = 8 + 2 * R, H2 = H * H, W = 2 * R + 1;
  const int* nb = t.nbr + 27 * node;
  for (int i = threadIdx.x; i < H2 * H; i += blockDim.x) {
    const int hx = i % H - R, hy = (i / H) % H - R, hz = i / H2 - R;
    const int slot = ((hx >> 3) + 1) + 3 * ((hy >> 3) + 1) + 9 * ((hz >> 3) + 1);
    const int sn = nb[slot];
    double m = 0.0;
    if (sn >= 0 && t.children[8 * sn] < 0) m = mp[(int64_t)sn * 512 + (hx & 7) + 8 * (hy & 7) + 64 * (hz & 7)];
    halo[i] = m;
  }
  __syncthreads();
  int p, a, b, c;
  parity_cell(0, threadIdx.x, p, a, b, c);
  const int lvl = t.level[node];
  const int base = (a + R) + H * (b + R) + H2 * (c + R);
  const int kbase = R + W * R + W * W * R;
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  const int* tab = lvl == 0 ? st.root : st.parity + p * st.n_st;
  const int ntab = lvl == 0 ? st.n_root : st.n_st;
  for (int pass = 0; pass < 2; ++pass) {
    const int* tb = pass == 0 ? tab : st.near_;
    const int nt = pass == 0 ? ntab : st.n_near;
    for (int s = 0; s < nt; ++s) {
      int dx, dy, dz;
      unpack(__ldg(tb + s), dx, dy, dz);
      const double m = halo[base + dx + H * dy + H2 * dz];
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
  loc[G_L0 * NC + tgt] = s0 * ih;
  loc[(G_L1 + 0) * NC + tgt] = s1 * (ih * ih);
  loc[(G_L1 + 1) * NC + tgt] = s2 * (ih * ih);
  loc[(G_L1 + 2) * NC + tgt] = s3 * (ih * ih);
  loc[(G_DG + 0) * NC + tgt] = 0.0;
  loc[(G_DG + 1) * NC + tgt] = 0.0;
  loc[(G_DG + 2) * NC + tgt] = 0.0;
}

// ---------------------------------------------------------------- cross-level pairs
// Explicit pairs between a leaf cell and cells of a finer refined region (both
// directions), one thread per target cell, general M2L (a leaf-leaf P2P pair is
// the same expression with zero higher moments).  Results added (+=).
template <bool FULL>
__global__ void __launch_bounds__(128) k_cross(DevTree t, CrossList xl, const double* __restrict__ mp,
                                               double* __restrict__ loc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= xl.n_targets) return;
  const int64_t NC = t.NC;
  const int64_t tgt = xl.targets[i];
  const double XA0 = mp[(F_X + 0) * NC + tgt], XA1 = mp[(F_X + 1) * NC + tgt], XA2 = mp[(F_X + 2) * NC + tgt];
  double Oh[10], tOh[3];
  if (FULL) {
    const double inv_m = 1.0 / mp[tgt];
    for (int k = 0; k < 10; ++k) Oh[k] = mp[(F_O + k) * NC + tgt] * inv_m;
    tOh[0] = Oh[0] + Oh[3] + Oh[5];
    tOh[1] = Oh[1] + Oh[6] + Oh[8];
    tOh[2] = Oh[2] + Oh[7] + Oh[9];
  }
  Acc<double> acc;
  acc_zero(acc);
  for (int64_t e = xl.start[i]; e < xl.start[i + 1]; ++e) {
    const int64_t src = xl.sources[e];
    const double R0 = XA0 - mp[(F_X + 0) * NC + src];
    const double R1 = XA1 - mp[(F_X + 1) * NC + src];
    const double R2 = XA2 - mp[(F_X + 2) * NC + src];
    double Q[6], O[10];
    for (int k = 0; k < 6; ++k) Q[k] = mp[(F_Q + k) * NC + src];
    for (int k = 0; k < 10; ++k) O[k] = mp[(F_O + k) * NC + src];
    const double rinv = rsqrt_f64(fma(R0, R0, fma(R1, R1, R2 * R2)));
    m2l_pair<FULL, FULL>(R0, R1, R2, mp[src], Q, O, Oh, tOh, rinv, acc);
  }
  loc[G_L0 * NC + tgt] += acc.L0;
  for (int k = 0; k < 3; ++k) loc[(G_L1 + k) * NC + tgt] += acc.L1[k];
  for (int k = 0; k < 3; ++k) loc[(G_DG + k) * NC + tgt] += acc.dg[k];
  if (FULL) {
    acc_finish(acc);
    for (int k = 0; k < 6; ++k) loc[(G_L2 + k) * NC + tgt] += acc.L2[k];
    for (int k = 0; k < 10; ++k) loc[(G_L3 + k) * NC + tgt] += acc.L3[k];
  }
}

// ---------------------------------------------------------------- L2L + L2P
// Child expansion += parent expansion shifted by delta = X_child - X_parent
// (exact for the cubic Taylor polynomial), dg carried down unshifted.  At leaf
// nodes the result is evaluated at the cell itself (L2P):
//   phi = L0,  g = -L1 + dg.
__global__ void __launch_bounds__(256) k_l2l(DevTree t, int node_begin, const double* __restrict__ mp,
                                             double* __restrict__ loc, double* __restrict__ phi,
                                             double* __restrict__ g, int64_t NL) {
  const int node = node_begin + (blockIdx.x >> 1);
  const int l = ((blockIdx.x & 1) << 8) + threadIdx.x;
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
cudaError_t configure_kernels() {
  return cudaFuncSetAttribute(k_leaf_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_init_leaf(const DevTree& t, const int* leaf_nodes, int n, double* mp, float* mp32,
                             cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_init_leaf<<<n, 256, 0, s>>>(t, leaf_nodes, mp, mp32);
  return cudaGetLastError();
}

cudaError_t launch_p2m(const DevTree& t, const int* leaf_nodes, int n, const double* rho, double* mp, float* mp32,
                       cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_p2m<<<n, 256, 0, s>>>(t, leaf_nodes, rho, mp, mp32);
  return cudaGetLastError();
}

cudaError_t launch_m2m(const DevTree& t, int b, int e, double* mp, float* mp32, cudaStream_t s) {
  if (e <= b) return cudaSuccess;
  k_m2m<<<2 * (e - b), 256, 0, s>>>(t, b, mp, mp32);
  return cudaGetLastError();
}

cudaError_t launch_m2l_interior(const DevTree& t, const int* nodes, int n, const Stencils& st, const double* mp,
                                double* loc, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_m2l<false><<<2 * n, 256, 0, s>>>(t, nodes, st, mp, loc);
  return cudaGetLastError();
}

cudaError_t launch_m2l_boundary(const DevTree& t, const int* nodes, int n, const Stencils& st, const double* mp,
                                double* loc, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_m2l<true><<<2 * n, 256, 0, s>>>(t, nodes, st, mp, loc);
  return cudaGetLastError();
}

cudaError_t launch_leaf_conv(const DevTree& t, const int* nodes, int n, const Stencils& st, const double* mp,
                             double* loc, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int H = 8 + 2 * st.radius;
  const size_t smem = sizeof(double) * H * H * H;
  k_leaf_conv<<<n, 512, smem, s>>>(t, nodes, st, mp, loc);
  return cudaGetLastError();
}

cudaError_t launch_cross(const DevTree& t, const CrossList& full, const CrossList& leaf, const double* mp,
                         double* loc, cudaStream_t s) {
  if (full.n_targets > 0) {
    k_cross<true><<<(full.n_targets + 127) / 128, 128, 0, s>>>(t, full, mp, loc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (leaf.n_targets > 0) {
    k_cross<false><<<(leaf.n_targets + 127) / 128, 128, 0, s>>>(t, leaf, mp, loc);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

cudaError_t launch_l2l(const DevTree& t, int b, int e, const double* mp, double* loc, double* phi, double* g,
                       int64_t NL, cudaStream_t s) {
  if (e <= b) return cudaSuccess;
  k_l2l<<<2 * (e - b), 256, 0, s>>>(t, b, mp, loc, phi, g, NL);
  return cudaGetLastError();
}

}  // namespace octo
