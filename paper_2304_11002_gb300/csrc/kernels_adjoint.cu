// Adjoint (vector-Jacobian product) of the float64 solve: given dS/dphi and dS/dg
// at the leaf cells, dS/drho through every phase, including the dependence of the
// expansion centres (centres of mass) and moments on the masses.
//
// Order (reverse of the forward): seeds at leaf cells (L2P^T) -> L2L^T from the
// finest level up -> M2L^T / P2P^T of every interaction -> M2M^T from the root down
// -> P2M^T.  Every kernel gathers into the cells it owns (no atomics), so the
// result is deterministic.  Adjoint state: mpb [20][NC] (multipole adjoints, packed
// like the multipoles) and locb [23][NC] (local-expansion adjoints).
#include "kernels.h"
#include "pair_vjp.cuh"
#include "sym.cuh"

namespace octo {

namespace {



__device__ __forceinline__ void parity_cell_a(int cls0, int tid, int& p, int& a, int& b, int& c) {
  const int w = tid >> 5, lane = tid & 31;
  p = cls0 + (w >> 1);
  const int q = ((w & 1) << 5) + lane;
  a = 2 * (q & 3) + (p & 1);
  b = 2 * ((q >> 2) & 3) + ((p >> 1) & 1);
  c = 2 * (q >> 4) + (p >> 2);
}

__device__ __forceinline__ void unpack_a(int e, int& dx, int& dy, int& dz) {
  dx = (int)(int8_t)(e & 0xff);
  dy = (int)(int8_t)((e >> 8) & 0xff);
  dz = (int)(int8_t)((e >> 16) & 0xff);
}

struct AdjState {
  const double* mp;
  const double* loc;
  double* mpb;
  double* locb;
  int* err;  // device-side index checks: bit set = a check failed and the access was skipped
};

// Index checks of the adjoint kernels: a failing check records its bit in *err and
// skips the access (the thread returns, or the pair is skipped).
#define ADJ_RETURN_UNLESS(cond, bit) \
  if (!(cond)) {                     \
    atomicOr(err, bit);              \
    return;                          \
  }
#define ADJ_SKIP_UNLESS(cond, bit) \
  if (!(cond)) {                   \
    atomicOr(as.err, bit);         \
    continue;                      \
  }

__device__ __forceinline__ void load_lb(const double* locb, int64_t NC, int64_t cell, bool full, double* Lb) {
  Lb[0] = locb[cell];
#pragma unroll
  for (int i = 1; i < 4; ++i) Lb[i] = locb[i * NC + cell];
#pragma unroll
  for (int i = 4; i < 20; ++i) Lb[i] = full ? locb[i * NC + cell] : 0.0;
#pragma unroll
  for (int i = 20; i < 23; ++i) Lb[i] = locb[i * NC + cell];
}

// ------------------------------------------------------------ seeds (L2P^T)
__global__ void k_adj_seed(DevTree t, const int* __restrict__ nodes, const double* __restrict__ phib,
                           const double* __restrict__ gb, int64_t NL, double* __restrict__ locb, int* err) {
  const int node = nodes[blockIdx.x];
  ADJ_RETURN_UNLESS(node >= 0 && node < t.n_nodes, 1);
  const int64_t NC = t.NC;
  const int64_t lid = t.leaf_id[node];
  ADJ_RETURN_UNLESS(lid >= 0 && (lid + 1) * 512 <= NL, 1);
  for (int l = threadIdx.x; l < 512; l += blockDim.x) {
    const int64_t cell = (int64_t)node * 512 + l, k = lid * 512 + l;
    locb[cell] = phib[k];
    for (int a = 0; a < 3; ++a) {
      locb[(G_L1 + a) * NC + cell] = -gb[a * NL + k];
      locb[(G_DG + a) * NC + cell] = gb[a * NL + k];
    }
  }
}

// ------------------------------------------------------------ L2L^T
// Parent cell P gathers the adjoints of its 8 children c (child = own + S(d) P,
// d = X_c - X_P): Pb += S(d)^T cb, dgb_P += dgb_c, and dS/dd goes to X_c (+) and
// X_P (-).
__global__ void __launch_bounds__(256) k_adj_l2l(DevTree t, int node_begin, AdjState st) {
  const int node = node_begin + (blockIdx.x >> 1);
  int* err = st.err;
  ADJ_RETURN_UNLESS(node >= 0 && node < t.n_nodes, 2);
  if (t.children[8 * node] < 0) return;
  const int l = ((blockIdx.x & 1) << 8) + threadIdx.x;
  const int a = l & 7, b = (l >> 3) & 7, c = l >> 6;
  const int64_t NC = t.NC;
  const int64_t P = (int64_t)node * 512 + l;
  const int ch = t.children[8 * node + (a >> 2) + 2 * (b >> 2) + 4 * (c >> 2)];
  ADJ_RETURN_UNLESS(ch >= 0 && ch < t.n_nodes, 2);
  const bool cleaf = t.children[8 * ch] < 0;
  double L1[3], L2[6], L3[10];
  for (int i = 0; i < 3; ++i) L1[i] = st.loc[(G_L1 + i) * NC + P];
  for (int i = 0; i < 6; ++i) L2[i] = st.loc[(G_L2 + i) * NC + P];
  for (int i = 0; i < 10; ++i) L3[i] = st.loc[(G_L3 + i) * NC + P];
  const double XP0 = st.mp[(F_X + 0) * NC + P], XP1 = st.mp[(F_X + 1) * NC + P], XP2 = st.mp[(F_X + 2) * NC + P];
  double b0 = 0, b1[3] = {0, 0, 0}, b2[6] = {0, 0, 0, 0, 0, 0}, b3[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  double bdg[3] = {0, 0, 0}, xP[3] = {0, 0, 0};
  for (int e = 0; e < 8; ++e) {
    const int64_t C = (int64_t)ch * 512 + (2 * (a & 3) + (e & 1)) + 8 * (2 * (b & 3) + ((e >> 1) & 1)) +
                      64 * (2 * (c & 3) + (e >> 2));
    const double d0 = st.mp[(F_X + 0) * NC + C] - XP0;
    const double d1 = st.mp[(F_X + 1) * NC + C] - XP1;
    const double d2 = st.mp[(F_X + 2) * NC + C] - XP2;
    double Lb[23];
    load_lb(st.locb, NC, C, !cleaf, Lb);
    const double c0 = Lb[0];
    const double* c1 = Lb + 1;
    const double* c2 = Lb + 4;
    const double* c3 = Lb + 10;
    // forward intermediates
    const double T0 = L3[0] * d0 + L3[1] * d1 + L3[2] * d2, T1 = L3[1] * d0 + L3[3] * d1 + L3[4] * d2;
    const double T2 = L3[2] * d0 + L3[4] * d1 + L3[5] * d2, T3 = L3[3] * d0 + L3[6] * d1 + L3[7] * d2;
    const double T4 = L3[4] * d0 + L3[7] * d1 + L3[8] * d2, T5 = L3[5] * d0 + L3[8] * d1 + L3[9] * d2;
    const double U0 = T0 * d0 + T1 * d1 + T2 * d2, U1 = T1 * d0 + T3 * d1 + T4 * d2, U2 = T2 * d0 + T4 * d1 + T5 * d2;
    const double S0 = L2[0] * d0 + L2[1] * d1 + L2[2] * d2, S1 = L2[1] * d0 + L2[3] * d1 + L2[4] * d2;
    const double S2 = L2[2] * d0 + L2[4] * d1 + L2[5] * d2;
    // adjoints of S, U, T
    const double Sb0 = 0.5 * c0 * d0 + c1[0], Sb1 = 0.5 * c0 * d1 + c1[1], Sb2 = 0.5 * c0 * d2 + c1[2];
    const double Ub0 = c0 * d0 * (1.0 / 6.0) + 0.5 * c1[0], Ub1 = c0 * d1 * (1.0 / 6.0) + 0.5 * c1[1];
    const double Ub2 = c0 * d2 * (1.0 / 6.0) + 0.5 * c1[2];
    const double Tb0 = c2[0] + Ub0 * d0, Tb1 = c2[1] + Ub0 * d1 + Ub1 * d0, Tb2 = c2[2] + Ub0 * d2 + Ub2 * d0;
    const double Tb3 = c2[3] + Ub1 * d1, Tb4 = c2[4] + Ub1 * d2 + Ub2 * d1, Tb5 = c2[5] + Ub2 * d2;
    // parent adjoints
    b0 += c0;
    b1[0] += c0 * d0 + c1[0];
    b1[1] += c0 * d1 + c1[1];
    b1[2] += c0 * d2 + c1[2];
    b2[0] += c2[0] + Sb0 * d0;
    b2[1] += c2[1] + Sb0 * d1 + Sb1 * d0;
    b2[2] += c2[2] + Sb0 * d2 + Sb2 * d0;
    b2[3] += c2[3] + Sb1 * d1;
    b2[4] += c2[4] + Sb1 * d2 + Sb2 * d1;
    b2[5] += c2[5] + Sb2 * d2;
    b3[0] += c3[0] + Tb0 * d0;
    b3[1] += c3[1] + Tb0 * d1 + Tb1 * d0;
    b3[2] += c3[2] + Tb0 * d2 + Tb2 * d0;
    b3[3] += c3[3] + Tb1 * d1 + Tb3 * d0;
    b3[4] += c3[4] + Tb1 * d2 + Tb2 * d1 + Tb4 * d0;
    b3[5] += c3[5] + Tb2 * d2 + Tb5 * d0;
    b3[6] += c3[6] + Tb3 * d1;
    b3[7] += c3[7] + Tb3 * d2 + Tb4 * d1;
    b3[8] += c3[8] + Tb4 * d2 + Tb5 * d1;
    b3[9] += c3[9] + Tb5 * d2;
    for (int i = 0; i < 3; ++i) bdg[i] += Lb[20 + i];
    // dS/dd
    const double Tf[3][3] = {{T0, T1, T2}, {T1, T3, T4}, {T2, T4, T5}};
    const double L2f[3][3] = {{L2[0], L2[1], L2[2]}, {L2[1], L2[3], L2[4]}, {L2[2], L2[4], L2[5]}};
    const double Sv[3] = {S0, S1, S2}, Uv[3] = {U0, U1, U2}, Sbv[3] = {Sb0, Sb1, Sb2}, Ubv[3] = {Ub0, Ub1, Ub2};
    const double Tbv[6] = {Tb0, Tb1, Tb2, Tb3, Tb4, Tb5};
    double dd[3];
    for (int f = 0; f < 3; ++f) {
      double s = c0 * (L1[f] + 0.5 * Sv[f] + Uv[f] * (1.0 / 6.0));
      for (int i = 0; i < 3; ++i) s += Sbv[i] * L2f[i][f] + Ubv[i] * Tf[i][f];
      for (int q = 0; q < 6; ++q) s += Tbv[q] * L3[sym::up(4 + q, f) - 10];
      dd[f] = s;
    }
    for (int f = 0; f < 3; ++f) {
      st.mpb[(F_X + f) * NC + C] += dd[f];
      xP[f] -= dd[f];
    }
  }
  st.locb[P] = b0;
  for (int i = 0; i < 3; ++i) st.locb[(G_L1 + i) * NC + P] = b1[i];
  for (int i = 0; i < 6; ++i) st.locb[(G_L2 + i) * NC + P] = b2[i];
  for (int i = 0; i < 10; ++i) st.locb[(G_L3 + i) * NC + P] = b3[i];
  for (int i = 0; i < 3; ++i) st.locb[(G_DG + i) * NC + P] = bdg[i];
  for (int f = 0; f < 3; ++f) st.mpb[(F_X + f) * NC + P] += xP[f];
}

// ------------------------------------------------------------ leaf convolution^T
// Leaf-leaf pairs (far stencil and near offsets): L0_Y += m_X kappa0(X - Y) / h,
// L1_Y += m_X kappa1(X - Y) / h^2, so with Y = X + d (kappa0 even, kappa1 odd)
//   dS/dm_X = sum_d Lb0_Y kappa0(d) / h - Lb1_Y . kappa1(d) / h^2.
__global__ void __launch_bounds__(256) k_adj_conv(DevTree t, const int* __restrict__ nodes, Stencils st,
                                                  AdjState as) {
  const int node = nodes[blockIdx.x >> 1];
  int* err = as.err;
  ADJ_RETURN_UNLESS(node >= 0 && node < t.n_nodes, 4);
  int p, a, b, c;
  parity_cell_a((blockIdx.x & 1) * 4, threadIdx.x, p, a, b, c);
  const int lvl = t.level[node];
  const int64_t NC = t.NC;
  const int R = st.radius, W = 2 * R + 1;
  const int kbase = R + W * R + W * W * R;
  const int* nb = t.nbr + 27 * node;
  double s0 = 0, s1 = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const int* tab = pass == 1 ? st.near_ : (lvl == 0 ? st.root : st.parity + p * st.n_st);
    const int nt = pass == 1 ? st.n_near : (lvl == 0 ? st.n_root : st.n_st);
    for (int s = 0; s < nt; ++s) {
      int dx, dy, dz;
      unpack_a(__ldg(tab + s), dx, dy, dz);
      const int sa = a + dx, sb = b + dy, sc = c + dz;
      const int sn = __ldg(nb + ((sa >> 3) + 1) + 3 * ((sb >> 3) + 1) + 9 * ((sc >> 3) + 1));
      ADJ_SKIP_UNLESS(sa >= -8 && sa < 16 && sb >= -8 && sb < 16 && sc >= -8 && sc < 16 && sn < t.n_nodes, 4);
      if (sn < 0 || __ldg(t.children + 8 * sn) >= 0) continue;
      const int64_t Y = (int64_t)sn * 512 + (sa & 7) + 8 * (sb & 7) + 64 * (sc & 7);
      const int kidx = kbase + dx + W * dy + W * W * dz;
      ADJ_SKIP_UNLESS(kidx >= 0 && kidx < W * W * W, 4);
      const double2* kp = reinterpret_cast<const double2*>(st.kappa + kbase + dx + W * dy + W * W * dz);
      const double2 ka = __ldg(kp), kb = __ldg(kp + 1);
      s0 = fma(as.locb[Y], ka.x, s0);
      s1 = fma(as.locb[(G_L1 + 0) * NC + Y], ka.y, s1);
      s1 = fma(as.locb[(G_L1 + 1) * NC + Y], kb.x, s1);
      s1 = fma(as.locb[(G_L1 + 2) * NC + Y], kb.y, s1);
    }
  }
  const double ih = 1.0 / t.h[lvl];
  const int64_t X = (int64_t)node * 512 + a + 8 * b + 64 * c;
  as.mpb[X] += s0 * ih - s1 * (ih * ih);
}

// ------------------------------------------------------------ general same-level pairs^T
// Visits the stencil partners Y of cell (a, b, c) of `node` that form a general
// pair with it (not both leaves) and calls f(Y, yleaf).
template <typename F>
__device__ __forceinline__ void general_partners(const DevTree& t, const Stencils& st, int node, int lvl, int p,
                                                 int a, int b, int c, bool xleaf, int* err, F&& f) {
  const int* tab = lvl == 0 ? st.root : st.parity + p * st.n_st;
  const int ntab = lvl == 0 ? st.n_root : st.n_st;
  const int* nb = t.nbr + 27 * node;
  for (int s = 0; s < ntab; ++s) {
    int dx, dy, dz;
    unpack_a(__ldg(tab + s), dx, dy, dz);
    const int sa = a + dx, sb = b + dy, sc = c + dz;
    if (!(sa >= -8 && sa < 16 && sb >= -8 && sb < 16 && sc >= -8 && sc < 16)) {
      atomicOr(err, 8);
      continue;
    }
    const int sn = __ldg(nb + ((sa >> 3) + 1) + 3 * ((sb >> 3) + 1) + 9 * ((sc >> 3) + 1));
    if (sn >= t.n_nodes) {
      atomicOr(err, 8);
      continue;
    }
    if (sn < 0) continue;
    const bool yleaf = __ldg(t.children + 8 * sn) < 0;
    if (xleaf && yleaf) continue;  // leaf-leaf pairs: k_adj_conv
    f((int64_t)sn * 512 + (sa & 7) + 8 * (sb & 7) + 64 * (sc & 7), yleaf);
  }
}

// Cell X of an interior node: every stencil partner Y; cell X of a leaf node: the
// partners in refined neighbour nodes.  Two kernels, one per role of X, keep the
// live state of each small: (a) X as target of (X <- Y) gives the gradients for X's
// centre and octupole (through Oh = O / m), interior X only; (b) X as source of
// (Y <- X) gives those for X's centre, mass and moments (leaf cells keep only the
// mass gradient).  Each kernel adds into the adjoints of the cells it owns, (a)
// before (b).
__global__ void __launch_bounds__(128) k_adj_general_target(DevTree t, const int* __restrict__ nodes, Stencils st,
                                                            AdjState as) {
  const int node = nodes[blockIdx.x >> 2];
  int* err = as.err;
  ADJ_RETURN_UNLESS(node >= 0 && node < t.n_nodes, 8);
  if (t.children[8 * node] < 0) return;  // leaf cells carry no octupole: nothing to do as target
  int p, a, b, c;
  parity_cell_a((blockIdx.x & 3) * 2, threadIdx.x, p, a, b, c);
  const int lvl = t.level[node];
  const int64_t NC = t.NC;
  const int64_t X = (int64_t)node * 512 + a + 8 * b + 64 * c;
  const double* mp = as.mp;
  const double mX = mp[X];
  const double XX0 = mp[(F_X + 0) * NC + X], XX1 = mp[(F_X + 1) * NC + X], XX2 = mp[(F_X + 2) * NC + X];
  double gX[3] = {0, 0, 0}, gm = 0;
  const double inv_m = 1.0 / mX;
  double OhX[10], LbX[23], gOh[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 10; ++i) OhX[i] = mp[(F_O + i) * NC + X] * inv_m;
  load_lb(as.locb, NC, X, true, LbX);
  general_partners(t, st, node, lvl, p, a, b, c, false, err, [&](int64_t Y, bool) {
    double QY[6], OY[10];
    const double mY = mp[Y];
    const double R0 = XX0 - mp[(F_X + 0) * NC + Y], R1 = XX1 - mp[(F_X + 1) * NC + Y], R2 = XX2 - mp[(F_X + 2) * NC + Y];
    for (int i = 0; i < 6; ++i) QY[i] = mp[(F_Q + i) * NC + Y];
    for (int i = 0; i < 10; ++i) OY[i] = mp[(F_O + i) * NC + Y];
    PairVJP g;
    m2l_pair_vjp<true, true, false, true>(R0, R1, R2, mY, QY, OY, OhX, LbX, g);
    for (int f = 0; f < 3; ++f) gX[f] += g.R[f];
    for (int i = 0; i < 10; ++i) gOh[i] += g.Oh[i];
  });
  // Oh = O * (1 / m)
  for (int i = 0; i < 10; ++i) {
    as.mpb[(F_O + i) * NC + X] += gOh[i] * inv_m;
    gm -= gOh[i] * OhX[i] * inv_m;
  }
  for (int f = 0; f < 3; ++f) as.mpb[(F_X + f) * NC + X] += gX[f];
  as.mpb[X] += gm;
}

__global__ void __launch_bounds__(128) k_adj_general_source(DevTree t, const int* __restrict__ nodes, Stencils st,
                                                            AdjState as) {
  const int node = nodes[blockIdx.x >> 2];
  int* err = as.err;
  ADJ_RETURN_UNLESS(node >= 0 && node < t.n_nodes, 8);
  int p, a, b, c;
  parity_cell_a((blockIdx.x & 3) * 2, threadIdx.x, p, a, b, c);
  const int lvl = t.level[node];
  const bool xleaf = t.children[8 * node] < 0;
  const int64_t NC = t.NC;
  const int64_t X = (int64_t)node * 512 + a + 8 * b + 64 * c;
  const double* mp = as.mp;
  const double mX = mp[X];
  const double XX0 = mp[(F_X + 0) * NC + X], XX1 = mp[(F_X + 1) * NC + X], XX2 = mp[(F_X + 2) * NC + X];
  double gX[3] = {0, 0, 0}, gm = 0;
  // Y <- X, R_YX = -R
  double QX[6], OX[10], gQ[6] = {0, 0, 0, 0, 0, 0}, gO[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 6; ++i) QX[i] = mp[(F_Q + i) * NC + X];
  for (int i = 0; i < 10; ++i) OX[i] = mp[(F_O + i) * NC + X];
  general_partners(t, st, node, lvl, p, a, b, c, xleaf, err, [&](int64_t Y, bool yleaf) {
    const double R0 = XX0 - mp[(F_X + 0) * NC + Y], R1 = XX1 - mp[(F_X + 1) * NC + Y], R2 = XX2 - mp[(F_X + 2) * NC + Y];
    double LbY[23];
    PairVJP g;
    if (yleaf) {
      load_lb(as.locb, NC, Y, false, LbY);
      m2l_pair_vjp<false, false, true, false>(-R0, -R1, -R2, mX, QX, OX, nullptr, LbY, g);
    } else {
      double OhY[10];
      const double inv_mY = 1.0 / mp[Y];
      for (int i = 0; i < 10; ++i) OhY[i] = mp[(F_O + i) * NC + Y] * inv_mY;
      load_lb(as.locb, NC, Y, true, LbY);
      m2l_pair_vjp<true, true, true, false>(-R0, -R1, -R2, mX, QX, OX, OhY, LbY, g);
    }
    for (int f = 0; f < 3; ++f) gX[f] -= g.R[f];
    gm += g.m;
    for (int i = 0; i < 6; ++i) gQ[i] += g.Q[i];
    for (int i = 0; i < 10; ++i) gO[i] += g.O[i];
  });
  if (!xleaf) {
    for (int f = 0; f < 3; ++f) as.mpb[(F_X + f) * NC + X] += gX[f];
    for (int i = 0; i < 6; ++i) as.mpb[(F_Q + i) * NC + X] += gQ[i];
    for (int i = 0; i < 10; ++i) as.mpb[(F_O + i) * NC + X] += gO[i];
  }
  as.mpb[X] += gm;
}

// ------------------------------------------------------------ cross-level pairs^T
// The cross-level lists hold both directions of every pair, so the partners of a
// cell as target are also its partners as source.  Same two passes as the general
// pairs; (a) only where X carries L2/L3 and an octupole (FULL).
template <bool FULL>
__global__ void __launch_bounds__(128) k_adj_cross(DevTree t, CrossList xl, AdjState as) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= xl.n_targets) return;
  const int64_t NC = t.NC;
  const double* mp = as.mp;
  const int64_t X = xl.targets[i];
  int* err = as.err;
  ADJ_RETURN_UNLESS(X >= 0 && X < NC, 16);
  const double mX = mp[X];
  const double XX0 = mp[(F_X + 0) * NC + X], XX1 = mp[(F_X + 1) * NC + X], XX2 = mp[(F_X + 2) * NC + X];
  const int64_t e0 = xl.start[i], e1 = xl.start[i + 1];
  double gX[3] = {0, 0, 0}, gm = 0;
  if constexpr (FULL) {  // (a) X <- Y
    const double inv_m = 1.0 / mX;
    double OhX[10], LbX[23], gOh[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 10; ++k) OhX[k] = mp[(F_O + k) * NC + X] * inv_m;
    load_lb(as.locb, NC, X, true, LbX);
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t Y = xl.sources[e];
      ADJ_SKIP_UNLESS(Y >= 0 && Y < NC, 16);
      double QY[6], OY[10];
      const double mY = mp[Y];
      const double R0 = XX0 - mp[(F_X + 0) * NC + Y], R1 = XX1 - mp[(F_X + 1) * NC + Y], R2 = XX2 - mp[(F_X + 2) * NC + Y];
      for (int k = 0; k < 6; ++k) QY[k] = mp[(F_Q + k) * NC + Y];
      for (int k = 0; k < 10; ++k) OY[k] = mp[(F_O + k) * NC + Y];
      PairVJP g;
      m2l_pair_vjp<true, true, false, true>(R0, R1, R2, mY, QY, OY, OhX, LbX, g);
      for (int f = 0; f < 3; ++f) gX[f] += g.R[f];
      for (int k = 0; k < 10; ++k) gOh[k] += g.Oh[k];
    }
    for (int k = 0; k < 10; ++k) {
      as.mpb[(F_O + k) * NC + X] += gOh[k] * inv_m;
      gm -= gOh[k] * OhX[k] * inv_m;
    }
  }
  {  // (b) Y <- X
    double QX[6], OX[10], gQ[6] = {0, 0, 0, 0, 0, 0}, gO[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 6; ++k) QX[k] = mp[(F_Q + k) * NC + X];
    for (int k = 0; k < 10; ++k) OX[k] = mp[(F_O + k) * NC + X];
    for (int64_t e = e0; e < e1; ++e) {
      const int64_t Y = xl.sources[e];
      ADJ_SKIP_UNLESS(Y >= 0 && Y < NC, 16);
      const bool yleaf = t.children[8 * (Y / 512)] < 0;
      const double R0 = XX0 - mp[(F_X + 0) * NC + Y], R1 = XX1 - mp[(F_X + 1) * NC + Y], R2 = XX2 - mp[(F_X + 2) * NC + Y];
      double LbY[23];
      PairVJP g;
      if (yleaf) {
        load_lb(as.locb, NC, Y, false, LbY);
        m2l_pair_vjp<false, false, true, false>(-R0, -R1, -R2, mX, QX, OX, nullptr, LbY, g);
      } else {
        double OhY[10];
        const double inv_mY = 1.0 / mp[Y];
        for (int k = 0; k < 10; ++k) OhY[k] = mp[(F_O + k) * NC + Y] * inv_mY;
        load_lb(as.locb, NC, Y, true, LbY);
        m2l_pair_vjp<true, true, true, false>(-R0, -R1, -R2, mX, QX, OX, OhY, LbY, g);
      }
      for (int f = 0; f < 3; ++f) gX[f] -= g.R[f];
      gm += g.m;
      for (int k = 0; k < 6; ++k) gQ[k] += g.Q[k];
      for (int k = 0; k < 10; ++k) gO[k] += g.O[k];
    }
    if (FULL) {
      for (int f = 0; f < 3; ++f) as.mpb[(F_X + f) * NC + X] += gX[f];
      for (int k = 0; k < 6; ++k) as.mpb[(F_Q + k) * NC + X] += gQ[k];
      for (int k = 0; k < 10; ++k) as.mpb[(F_O + k) * NC + X] += gO[k];
    }
  }
  as.mpb[X] += gm;
}

// ------------------------------------------------------------ M2M^T
// Parent P (complete adjoint) pushes to its 8 children.  Forward, per child c with
// d = X_c - X_P:  Q_P += Q_c + m_c d^e,  O_P += O_c + sum_f e_f Q_c[e - e_f] d_f + m_c d^e
// (e: exponents of the packed component), X_P = sum m_c X_c / m_P, m_P = sum m_c.
__global__ void __launch_bounds__(256) k_adj_m2m(DevTree t, int node_begin, AdjState as) {
  const int node = node_begin + (blockIdx.x >> 1);
  int* err = as.err;
  ADJ_RETURN_UNLESS(node >= 0 && node < t.n_nodes, 32);
  if (t.children[8 * node] < 0) return;
  const int l = ((blockIdx.x & 1) << 8) + threadIdx.x;
  const int a = l & 7, b = (l >> 3) & 7, c = l >> 6;
  const int64_t NC = t.NC;
  const double* mp = as.mp;
  const int64_t P = (int64_t)node * 512 + l;
  const int ch = t.children[8 * node + (a >> 2) + 2 * (b >> 2) + 4 * (c >> 2)];
  ADJ_RETURN_UNLESS(ch >= 0 && ch < t.n_nodes, 32);
  const double mP = mp[P];
  const double XP[3] = {mp[(F_X + 0) * NC + P], mp[(F_X + 1) * NC + P], mp[(F_X + 2) * NC + P]};
  double Pm = as.mpb[P], PX[3], PQ[6], PO[10];
  for (int f = 0; f < 3; ++f) PX[f] = as.mpb[(F_X + f) * NC + P];
  for (int i = 0; i < 6; ++i) PQ[i] = as.mpb[(F_Q + i) * NC + P];
  for (int i = 0; i < 10; ++i) PO[i] = as.mpb[(F_O + i) * NC + P];
  int64_t C[8];
  double dbar[8][3];
  double XPtot[3] = {PX[0], PX[1], PX[2]};
  for (int e = 0; e < 8; ++e) {
    C[e] = (int64_t)ch * 512 + (2 * (a & 3) + (e & 1)) + 8 * (2 * (b & 3) + ((e >> 1) & 1)) +
           64 * (2 * (c & 3) + (e >> 2));
    const int64_t Ce = C[e];
    const double mc = mp[Ce];
    double d[3];
    for (int f = 0; f < 3; ++f) d[f] = mp[(F_X + f) * NC + Ce] - XP[f];
    double qc[6];
    for (int i = 0; i < 6; ++i) qc[i] = mp[(F_Q + i) * NC + Ce];
    double pw[3][4];
    for (int f = 0; f < 3; ++f) pw[f][0] = 1.0, pw[f][1] = d[f], pw[f][2] = d[f] * d[f], pw[f][3] = pw[f][2] * d[f];
    double cm = 0, cd[3] = {0, 0, 0}, cq[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int q = 0; q < 6; ++q) {  // rank 2
      const int e0 = sym::ex(4 + q, 0), e1 = sym::ex(4 + q, 1), e2 = sym::ex(4 + q, 2);
      const double dq = pw[0][e0] * pw[1][e1] * pw[2][e2];
      cm += PQ[q] * dq;
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        const int ef = sym::ex(4 + q, f);
        if (ef > 0) {
          const int dn = sym::down(4 + q, f);  // rank-1 component e - e_f
          const int e0d = sym::ex(dn, 0), e1d = sym::ex(dn, 1), e2d = sym::ex(dn, 2);
          cd[f] += PQ[q] * mc * ef * pw[0][e0d] * pw[1][e1d] * pw[2][e2d];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) {  // rank 3
      const int e0 = sym::ex(10 + q, 0), e1 = sym::ex(10 + q, 1), e2 = sym::ex(10 + q, 2);
      const double dq = pw[0][e0] * pw[1][e1] * pw[2][e2];
      cm += PO[q] * dq;
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        const int ef = sym::ex(10 + q, f);
        if (ef > 0) {
          const int dn = sym::down(10 + q, f);  // rank-2 component e - e_f
          const int e0d = sym::ex(dn, 0), e1d = sym::ex(dn, 1), e2d = sym::ex(dn, 2);
          // d/d d_f of (e_f Q[e-e_f] d_f) and of m d^e
          cd[f] += PO[q] * ef * (qc[dn - 4] + mc * pw[0][e0d] * pw[1][e1d] * pw[2][e2d]);
          cq[dn - 4] += PO[q] * ef * d[f];
        }
      }
    }
    for (int f = 0; f < 3; ++f) {
      dbar[e][f] = cd[f];
      XPtot[f] -= cd[f];
    }
    double* mb = as.mpb;
    mb[Ce] += cm + Pm;
    for (int i = 0; i < 6; ++i) mb[(F_Q + i) * NC + Ce] += PQ[i] + cq[i];
    for (int i = 0; i < 10; ++i) mb[(F_O + i) * NC + Ce] += PO[i];
  }
  for (int e = 0; e < 8; ++e) {
    const int64_t Ce = C[e];
    const double mc = mp[Ce];
    double dm = 0;
    for (int f = 0; f < 3; ++f) {
      const double xc = mp[(F_X + f) * NC + Ce];
      as.mpb[(F_X + f) * NC + Ce] += dbar[e][f] + XPtot[f] * mc / mP;
      dm += XPtot[f] * (xc - XP[f]) / mP;
    }
    as.mpb[Ce] += dm;
  }
}

// ------------------------------------------------------------ P2M^T
__global__ void k_adj_p2m(DevTree t, const int* __restrict__ nodes, const double* __restrict__ mpb,
                          double* __restrict__ rhob, int64_t NL, int* err) {
  const int node = nodes[blockIdx.x];
  ADJ_RETURN_UNLESS(node >= 0 && node < t.n_nodes, 64);
  const double h3 = t.h3[t.level[node]];
  const int64_t lid = t.leaf_id[node];
  ADJ_RETURN_UNLESS(lid >= 0 && (lid + 1) * 512 <= NL, 64);
  for (int l = threadIdx.x; l < 512; l += blockDim.x) rhob[lid * 512 + l] = mpb[(int64_t)node * 512 + l] * h3;
}

}  // namespace

// Largest per-thread local memory (register spills and stack frame) of the adjoint
// kernels, so that the caller can size the per-thread stack limit before launching.
cudaError_t adjoint_local_bytes(size_t* out) {
  size_t m = 0;
  cudaFuncAttributes fa;
  const void* fns[] = {(const void*)k_adj_seed,         (const void*)k_adj_l2l,         (const void*)k_adj_conv,
                       (const void*)k_adj_general_target, (const void*)k_adj_general_source, (const void*)k_adj_cross<true>, (const void*)k_adj_cross<false>,
                       (const void*)k_adj_m2m,          (const void*)k_adj_p2m};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    if (fa.localSizeBytes > m) m = fa.localSizeBytes;
  }
  *out = m;
  return cudaSuccess;
}

cudaError_t launch_backward(const DevTree& t, const BackwardArgs& ba, cudaStream_t s) {
  AdjState as{ba.mp, ba.loc, ba.mpb, ba.locb, ba.err};
  cudaError_t e = cudaMemsetAsync(ba.mpb, 0, sizeof(double) * N_MP * t.NC, s);
  if (e != cudaSuccess) return e;
  if (ba.n_leaf_nodes) k_adj_seed<<<ba.n_leaf_nodes, 256, 0, s>>>(t, ba.leaf_nodes, ba.phib, ba.gb, ba.NL, ba.locb, ba.err);
  for (int l = ba.max_level - 1; l >= 0; --l) {
    const int n = ba.level_start[l + 1] - ba.level_start[l];
    if (n > 0) k_adj_l2l<<<2 * n, 256, 0, s>>>(t, ba.level_start[l], as);
  }
  if (ba.n_leaf_nodes) k_adj_conv<<<2 * ba.n_leaf_nodes, 256, 0, s>>>(t, ba.leaf_nodes, ba.st, as);
  if (ba.n_general) {
    k_adj_general_target<<<4 * ba.n_general, 128, 0, s>>>(t, ba.general_nodes, ba.st, as);
    k_adj_general_source<<<4 * ba.n_general, 128, 0, s>>>(t, ba.general_nodes, ba.st, as);
  }
  if (ba.xf.n_targets) k_adj_cross<true><<<(ba.xf.n_targets + 127) / 128, 128, 0, s>>>(t, ba.xf, as);
  if (ba.xl.n_targets) k_adj_cross<false><<<(ba.xl.n_targets + 127) / 128, 128, 0, s>>>(t, ba.xl, as);
  e = launch_cross_cells_adjoint(t, ba.xc, ba.locb, ba.mpb, ba.xc_grid, s);
  if (e != cudaSuccess) return e;
  for (int l = 0; l < ba.max_level; ++l) {
    const int n = ba.level_start[l + 1] - ba.level_start[l];
    if (n > 0) k_adj_m2m<<<2 * n, 256, 0, s>>>(t, ba.level_start[l], as);
  }
  if (ba.n_leaf_nodes) k_adj_p2m<<<ba.n_leaf_nodes, 256, 0, s>>>(t, ba.leaf_nodes, ba.mpb, ba.rhob, ba.NL, ba.err);
  return cudaGetLastError();
}

}  // namespace octo
