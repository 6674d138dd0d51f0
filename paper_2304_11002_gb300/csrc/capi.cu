// C ABI of the solver (include/octo_fmm.h): handle, device workspace, phase
// ordering on a stream and the CUDA-graph replay of the whole solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/octo_fmm.h"
#include "handle.h"
#include "kernels.h"
#include "pair_vjp.cuh"
#include "plan.h"

using namespace octo;

namespace {

std::mutex g_err_mu;
std::string g_create_error;

}  // namespace

void octo::set_global_error(const std::string& msg) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_create_error = msg;
}

namespace {

// Test hook for allocation failures: with OCTO_FMM_FAIL_ALLOC_AT=N in the
// environment, the N-th device allocation (counting from 1) of an octo_fmm_create
// call fails as if the device were out of memory.  Only create's allocations count;
// the hook is read once at the start of every create call.
thread_local int t_alloc_count = 0, t_alloc_fail_at = 0;

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (t_alloc_fail_at > 0 && ++t_alloc_count == t_alloc_fail_at) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

template <typename T>
cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src) {
  *dst = nullptr;
  if (src.empty()) return cudaSuccess;
  cudaError_t e = dev_malloc((void**)dst, sizeof(T) * src.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

cudaError_t upload_cross(const Plan& P, const std::vector<int64_t>& targets, const std::vector<int64_t>& start,
                         const std::vector<int64_t>& mid, const std::vector<int64_t>& sources, CrossSet& cs) {
  std::vector<int64_t> ft, fs(1, 0), fm, fsrc, lt, ls(1, 0), lm, lsrc;
  for (size_t i = 0; i < targets.size(); ++i) {
    const int64_t tg = targets[i];
    const bool full = P.children[8 * (tg / kCells)] >= 0;
    auto& T = full ? ft : lt;
    auto& S = full ? fs : ls;
    auto& M = full ? fm : lm;
    auto& SRC = full ? fsrc : lsrc;
    T.push_back(tg);
    M.push_back((int64_t)SRC.size() + (mid[i] - start[i]));
    (full ? cs.f_p2p : cs.l_p2p) += start[i + 1] - mid[i];
    SRC.insert(SRC.end(), sources.begin() + start[i], sources.begin() + start[i + 1]);
    S.push_back((int64_t)SRC.size());
  }
  cs.n_f = (int)ft.size();
  cs.n_l = (int)lt.size();
  cs.f_pairs = (int64_t)fsrc.size();
  cs.l_pairs = (int64_t)lsrc.size();
  cudaError_t e = cudaSuccess;
  for (auto [d, v] : {std::pair{&cs.d_ft, &ft}, {&cs.d_fs, &fs}, {&cs.d_fm, &fm}, {&cs.d_fsrc, &fsrc},
                      {&cs.d_lt, &lt}, {&cs.d_ls, &ls}, {&cs.d_lm, &lm}, {&cs.d_lsrc, &lsrc}})
    if (e == cudaSuccess) e = upload(d, *v);
  cs.f = CrossList{cs.d_ft, cs.d_fs, cs.d_fsrc, cs.n_f, cs.d_fm};
  cs.l = CrossList{cs.d_lt, cs.d_ls, cs.d_lsrc, cs.n_l, cs.d_lm};
  return e;
}

}  // namespace


namespace {

int fail(octo_fmm* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(octo_fmm* h, cudaError_t e, const char* what) {
  return fail(h, OCTO_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void free_all(octo_fmm* h) {
  void* ptrs[] = {h->d_level,    h->d_parent,  h->d_octant, h->d_children, h->d_nbr,    h->d_leaf_id,
                  h->d_ijk,      h->d_interior, h->d_leaf,  h->d_boundary, h->d_st_parity, h->d_st_root,
                  h->d_st_near,  h->d_kappa,   h->d_xc_t,   h->d_xc_off,   h->d_xc_ent,  h->d_xc_tab,  h->d_xc_counter,
                  h->d_mp,       h->d_loc,      h->d_io,        h->d_mp32,     h->d_near,     h->d_xcf,
                  h->d_cell_ent, h->d_cell_ent_off, h->d_bnd_perm,
                  h->d_bnd_index, h->d_mpb,    h->d_locb,
                  h->d_general,  h->d_queue,   h->d_counter, h->d_err,
                  h->d_leaf_far, h->d_leaf_root, h->d_leaf_near,
                  h->d_leaf_blocks, h->d_scf,  h->d_scf_nodes, h->d_st_pair, h->d_st_pair_root,
                  h->d_cell_pair, h->d_cell_pair_off};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int64_t* p : {h->xg.d_ft, h->xg.d_fs, h->xg.d_fm, h->xg.d_fsrc, h->xg.d_lt, h->xg.d_ls, h->xg.d_lm,
                     h->xg.d_lsrc})
    if (p) cudaFree(p);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (auto& ev : h->ev)
    if (ev) cudaEventDestroy(ev);
}

// Kinds in solve order; [S_M2L, S_CROSS_LEAF] is the interaction phase.
enum StageKind { S_P2M, S_M2M, S_M2L, S_CONV, S_NEAR, S_PERSIST, S_CROSS_CELLS, S_CROSS_FULL, S_CROSS_LEAF, S_L2L };

// Interaction strategies (option key 3).
enum { MODE_AUTO = 0, MODE_PER_KIND = 1, MODE_PERSISTENT = 2 };

// Floating-point operations of the per-pair expression as written (a fused
// multiply-add counts as two), obtained by running the same template with a
// counting scalar type.
int64_t g_counted_ops = 0;
#define HD __host__ __device__
struct Counted {
  double v;
  HD Counted() : v(0) {}
  HD Counted(double x) : v(x) {}
  HD static void tick() {
#ifndef __CUDA_ARCH__
    ++g_counted_ops;
#endif
  }
  HD friend Counted operator+(Counted a, Counted b) { tick(); return Counted(a.v + b.v); }
  HD friend Counted operator-(Counted a, Counted b) { tick(); return Counted(a.v - b.v); }
  HD friend Counted operator*(Counted a, Counted b) { tick(); return Counted(a.v * b.v); }
  HD friend Counted operator/(Counted a, Counted b) { tick(); return Counted(a.v / b.v); }
  HD friend Counted sqrt(Counted a) {
    tick();
#ifndef __CUDA_ARCH__
    return Counted(std::sqrt(a.v));
#else
    return Counted(::sqrt(a.v));
#endif
  }
  HD Counted operator-() const { return Counted(-v); }
  HD Counted& operator+=(Counted b) { tick(); v += b.v; return *this; }
  HD Counted& operator-=(Counted b) { tick(); v -= b.v; return *this; }
};
#undef HD

// Per pair: R = X_A - X_B (3), r^2 (5), the float64 reciprocal square root
// refinement (8) and the expansion arithmetic.
template <bool FULL, bool TOCT>
int64_t m2l_pair_flops() {
  Counted Q[6], O[10], Oh[10], tOh[3];
  Acc<Counted> a;
  acc_zero(a);
  g_counted_ops = 0;
  m2l_pair<FULL, TOCT, Counted>(Counted(1.0), Counted(2.0), Counted(3.0), Counted(1.0), Q, O, Oh, tOh,
                                Counted(0.5), a);
  return g_counted_ops + 3 + 5 + 8;
}
constexpr int64_t kConvFlopsPerPair = 8;  // four fused multiply-adds

// One reverse-mode pair (pair_vjp.cuh) as written, with the host's 1/sqrt for
// the reciprocal square root (the device refines a float32 seed instead: 8 more).
template <bool FULL, bool TOCT, bool SRC, bool OH>
int64_t vjp_flops() {
  Counted Q[6], O[10], Oh[10], Lb[23];
  PairVJPT<Counted> g;
  g_counted_ops = 0;
  m2l_pair_vjp<FULL, TOCT, SRC, OH, Counted>(Counted(1.0), Counted(2.0), Counted(3.0), Counted(1.0), Q, O, Oh, Lb,
                                             g);
  return g_counted_ops - 2 + 8;
}
// near offsets run as (d, -d) pairs: one add, one subtract and four fused
// multiply-adds per two pairs
constexpr int64_t kNearFlopsPer2Pairs = 2 + 4 * 2;
// Tree passes, float64 in both modes, counted from the expressions of k_m2m / k_l2l
// as written (FMA = 2): M2M per parent cell = 8 children x (mass and centre sums 7,
// d 3, m d 3, M2 18, M3 64) + 3 divisions; L2L per cell = d 3, (L3 d) 30, (L3 d d)
// 15, (L2 d) 15, L0 21, L1 12, dg 3, plus L2 / L3 updates 22 at refined cells or
// L2P (g, near field) 7 at leaf cells.
constexpr int64_t kM2MFlopsPerCell = 8 * (7 + 3 + 3 + 18 + 64) + 3;
// parent cells whose children are point masses (leaf child node): M2 6 fused
// multiply-adds, M3 10 multiplies and 10 fused multiply-adds per child
constexpr int64_t kM2MFlopsPointChildren = 8 * (7 + 3 + 3 + 12 + 30) + 3;
constexpr int64_t kL2LFlopsInterior = 99 + 22, kL2LFlopsLeaf = 99 + 7;
// exact point-mass pair: R (3), r^2 (5), reciprocal square root (8), m/r, m/r^3 (3), phi and g (7)
constexpr int64_t kP2PFlopsPerPair = 26;

// Builds the fixed stage list (its length does not depend on the data, so the
// whole sequence can be captured once into a CUDA graph).
void make_stages(octo_fmm* h) {
  const Plan& P = h->plan;
  auto add = [&](int kind, int a, int b, std::string name, int64_t pairs, int64_t cells) {
    // algorithmic flops and bytes of the stage (bytes: each value read or written once)
    // Far-field flops run in float32 in mixed mode; near-field (P2P) flops are always float64.
    int64_t far = 0, near = 0, bytes = 0;
    const int64_t f_int = m2l_pair_flops<true, true>(), f_leaf = m2l_pair_flops<false, false>();
    switch (kind) {
      case S_P2M: bytes = cells * 16; break;                      // rho in, m out
      case S_M2M: {  // 8 children in, parent out (point-mass children: only m and X read)
        int64_t point = 0;  // parent cells whose children are point masses
        for (int k = a; k < b; ++k)
          if (P.children[8 * k] >= 0)
            for (int o = 0; o < 8; ++o) point += P.children[8 * P.children[8 * k + o]] < 0 ? kCells / 8 : 0;
        bytes = (cells - point) * (8 * 20 + 20) * 8 + point * (8 * 4 + 20) * 8;
        near = (cells - point) * kM2MFlopsPerCell + point * kM2MFlopsPointChildren;
        break;
      }
      case S_M2L: far = pairs * f_int; break;
      case S_CONV:  // mixed precision: the near field is the separate S_NEAR stage
        far = P.kernel_pairs[1] * kConvFlopsPerPair + P.kernel_pairs[3] * f_leaf;
        if (h->precision != OCTO_MIXED) near = P.kernel_pairs[2] * kNearFlopsPer2Pairs / 2;
        break;
      case S_NEAR: near = P.kernel_pairs[2] * kNearFlopsPer2Pairs / 2; break;
      case S_PERSIST:  // including the tabulated cross-level pairs (cross items)
        far = P.kernel_pairs[0] * f_int + P.kernel_pairs[1] * kConvFlopsPerPair + P.kernel_pairs[3] * f_leaf;
        near = P.kernel_pairs[2] * kNearFlopsPer2Pairs / 2 + (h->xc.n_slices > 0 ? P.xc_pairs * kConvFlopsPerPair : 0);
        break;
      case S_CROSS_CELLS: near = pairs * kConvFlopsPerPair; break;  // float64 in both modes
      case S_CROSS_FULL:
        far = (pairs - h->xg.f_p2p) * f_int;
        near = h->xg.f_p2p * kP2PFlopsPerPair;
        break;
      case S_CROSS_LEAF:
        far = (pairs - h->xg.l_p2p) * f_leaf;
        near = h->xg.l_p2p * kP2PFlopsPerPair;
        break;
      case S_L2L: {  // own L/X in + L out + parent share
        bytes = cells * 52 * 8;
        int64_t leaf_cells = 0;
        for (int k = a; k < b; ++k) leaf_cells += P.children[8 * k] < 0 ? kCells : 0;
        near = leaf_cells * kL2LFlopsLeaf + (cells - leaf_cells) * kL2LFlopsInterior;
        break;
      }
    }
    const int64_t flops = far + near;
    const int64_t flops64 = h->precision == OCTO_MIXED ? near : flops;
    h->stages.push_back({kind, a, b, std::move(name), pairs, cells, flops, flops64, bytes});
  };
  h->stages.clear();
  if (!P.leaf_nodes.empty()) add(S_P2M, 0, 0, "p2m", 0, (int64_t)P.leaf_nodes.size() * kCells);
  for (int l = P.max_level - 1; l >= 0; --l)
    if (P.level_start[l + 1] > P.level_start[l]) {
      int64_t ni = 0;
      for (int k = P.level_start[l]; k < P.level_start[l + 1]; ++k) ni += P.children[8 * k] >= 0;
      add(S_M2M, P.level_start[l], P.level_start[l + 1], "m2m_l" + std::to_string(l), 0, ni * kCells);
    }
  const bool mixed = h->precision == OCTO_MIXED;
  if (h->mode == MODE_PERSISTENT) {
    add(S_PERSIST, 0, 0, mixed ? "interact_persistent_mixed" : "interact_persistent",
        P.kernel_pairs[0] + P.kernel_pairs[1] + P.kernel_pairs[2] + P.kernel_pairs[3] +
            (h->xc.n_slices > 0 ? P.xc_pairs : 0),
        (int64_t)P.n_nodes * kCells);
  } else {
    if (!P.interior_nodes.empty())
      add(S_M2L, 0, 0, mixed ? "m2l_interior_f32" : "m2l_interior", P.kernel_pairs[0],
          (int64_t)P.interior_nodes.size() * kCells);
    if (!P.leaf_nodes.empty()) {
      if (mixed) {
        add(S_CONV, 0, 0, "leaf_far_f32", P.kernel_pairs[1] + P.kernel_pairs[3], (int64_t)P.leaf_nodes.size() * kCells);
        add(S_NEAR, 0, 0, "leaf_near_f64", P.kernel_pairs[2], (int64_t)P.leaf_nodes.size() * kCells);
      } else {
        add(S_CONV, 0, 0, "leaf", P.kernel_pairs[1] + P.kernel_pairs[2] + P.kernel_pairs[3],
            (int64_t)P.leaf_nodes.size() * kCells);
      }
    }
  }
  if (h->xc.n_slices > 0) {
    int64_t nt = 0;
    for (int64_t t : P.xc_targets) nt += t >= 0;
    if (h->mode == MODE_PERSISTENT)
      add(S_CROSS_CELLS, 0, 0, "cross_cells_apply", 0, nt);
    else
      add(S_CROSS_CELLS, 0, 0, "cross_cells", P.xc_pairs, nt);
  }
  if (h->xg.n_f > 0) add(S_CROSS_FULL, 0, 0, "cross_interior", h->xg.f_pairs, h->xg.n_f);
  if (h->xg.n_l > 0) add(S_CROSS_LEAF, 0, 0, "cross_leaf", h->xg.l_pairs, h->xg.n_l);
  for (int l = 0; l <= P.max_level; ++l)
    if (P.level_start[l + 1] > P.level_start[l])
      add(S_L2L, P.level_start[l], P.level_start[l + 1], "l2l_l" + std::to_string(l), 0,
          (int64_t)(P.level_start[l + 1] - P.level_start[l]) * kCells);
}

// Rebuilds the stage list for the current strategy, with one timing event per
// stage boundary, and drops the captured graph.
cudaError_t rebuild_stages(octo_fmm* h) {
  make_stages(h);
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  while (h->ev.size() < h->stages.size() + 1) {
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
    h->ev.push_back(ev);
  }
  return cudaSuccess;
}

InteractArgs interact_args(const octo_fmm* h) {
  const Plan& P = h->plan;
  InteractArgs a;
  a.mp = h->d_mp;
  a.mp32 = h->d_mp32;
  a.loc = h->d_loc;
  a.st = h->st;
  a.mixed = h->precision == OCTO_MIXED;
  a.interior = h->d_interior;
  a.n_interior = (int)P.interior_nodes.size();
  a.leaf = h->d_leaf;
  a.n_leaf = (int)P.leaf_nodes.size();
  a.nearf = h->d_near;
  a.NL = h->n_leaf_cells();
  a.queue = h->d_queue;
  a.n_items = h->n_items;
  a.counter = h->d_counter;
  a.n32 = h->paced ? h->n32 : -1;
  a.grid = h->n_sm * h->persist_per_sm[h->min_blocks];
  a.min_blocks = h->min_blocks;
  a.xc = h->xc;
  a.xcf = h->d_xcf;
  a.corr64 = h->corr64;
  return a;
}

cudaError_t enq_stage(octo_fmm* h, const octo_fmm::Stage& st, const double* rho, double* phi, double* g,
                      cudaStream_t s) {
  const Plan& P = h->plan;
  switch (st.kind) {
    case S_P2M:
      return launch_p2m(h->dt, h->d_leaf, (int)P.leaf_nodes.size(), rho, h->d_mp, h->d_mp32, h->d_err, s);
    case S_M2M: return launch_m2m(h->dt, st.a, st.b, h->d_mp, h->d_mp32, s);
    case S_M2L: return launch_interior_items(h->dt, interact_args(h), s);
    case S_CONV: return launch_leaf_items(h->dt, interact_args(h), s);
    case S_NEAR: return launch_near_items(h->dt, interact_args(h), s);
    case S_PERSIST: return launch_persistent(h->dt, interact_args(h), s);
    case S_CROSS_CELLS:  // persistent mode: the sums came from the queue's cross items
      if (h->mode == MODE_PERSISTENT) return launch_cross_apply(h->dt, h->xc, h->d_xcf, h->d_loc, s);
      return launch_cross_cells(h->dt, h->xc, h->d_mp, h->d_loc, h->xc_grid, s);
    case S_CROSS_FULL:
      return launch_cross_list(h->dt, h->xg.f, true, h->d_mp, h->d_loc, h->precision == OCTO_MIXED, s, h->corr64);
    case S_CROSS_LEAF:
      return launch_cross_list(h->dt, h->xg.l, false, h->d_mp, h->d_loc, h->precision == OCTO_MIXED, s, h->corr64);
    case S_L2L: return launch_l2l(h->dt, st.a, st.b, h->d_mp, h->d_loc, phi, g, h->n_leaf_cells(), h->d_near, s);
  }
  return cudaErrorInvalidValue;
}

// Phases: stages [0, i_interact) are the upward pass, [i_interact, i_downward) the
// interactions and the rest the downward pass.
cudaError_t enq_range(octo_fmm* h, int kind_lo, int kind_hi, const double* rho, double* phi, double* g,
                      cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < h->stages.size() && e == cudaSuccess; ++i) {
    const auto& st = h->stages[i];
    if (st.kind < kind_lo || st.kind > kind_hi) continue;
    if (h->profile) e = cudaEventRecordWithFlags(h->ev[i], s, cudaEventRecordExternal);
    if (e == cudaSuccess) e = enq_stage(h, st, rho, phi, g, s);
  }
  return e;
}

cudaError_t enq_upward(octo_fmm* h, const double* rho, cudaStream_t s) {
  return enq_range(h, S_P2M, S_M2M, rho, nullptr, nullptr, s);
}
cudaError_t enq_interact(octo_fmm* h, cudaStream_t s) {
  return enq_range(h, S_M2L, S_CROSS_LEAF, nullptr, nullptr, nullptr, s);
}
cudaError_t enq_downward(octo_fmm* h, double* phi, double* g, cudaStream_t s) {
  return enq_range(h, S_L2L, S_L2L, nullptr, phi, g, s);
}

cudaError_t enq_solve(octo_fmm* h, const double* rho, double* phi, double* g, cudaStream_t s) {
  cudaError_t e = enq_range(h, S_P2M, S_L2L, rho, phi, g, s);
  if (e == cudaSuccess && h->profile) e = cudaEventRecordWithFlags(h->ev[h->stages.size()], s, cudaEventRecordExternal);
  return e;
}

int count_launches(const octo_fmm* h) { return (int)h->stages.size(); }

// Monopole kernel table over [-R, R]^3 for unit cell width (see k_leaf_conv):
// kappa0 = -1/|d|, kappa1 = -d/|d|^3, zero at d = 0.
std::vector<Kappa> make_kappa(int R) {
  const int W = 2 * R + 1;
  std::vector<Kappa> k((size_t)W * W * W);
  for (int z = -R; z <= R; ++z)
    for (int y = -R; y <= R; ++y)
      for (int x = -R; x <= R; ++x) {
        Kappa v = {{0, 0, 0, 0}};
        double r2 = (double)(x * x + y * y + z * z);
        if (r2 > 0) {
          double r = std::sqrt(r2);
          double ir3 = 1.0 / (r2 * r);
          v.v[0] = -1.0 / r;
          v.v[1] = -(double)x * ir3;
          v.v[2] = -(double)y * ir3;
          v.v[3] = -(double)z * ir3;
        }
        k[(size_t)(x + R) + W * (y + R) + (size_t)W * W * (z + R)] = v;
      }
  return k;
}

}  // namespace

namespace {

// Estimates before measurement, in SM cycles: an M2L pair with correction ~240
// float32 instructions at 128 per cycle; a leaf node's far field ~1200 entries x 512
// cells at ~24 instructions per pair (halo staging and boundary pairs included); its
// near field 170 x 512 pairs of 3 float64 operations at 2 per cycle, at about 60 %
// of that rate when it shares the SM; a tabulated cross-level pair 4 DFMA, likewise.
ItemCosts default_costs(const Plan& P) {
  return {240.0 / 128.0, 512.0 * P.n_st * 24.0 / 128.0, 512.0 * (double)P.st_near.size() * 3.0 / 2.0 / 0.6,
          4.0 / 2.0 / 0.6};
}

// The persistent work queue (item = (node << 4) | (kind << 2) | part).  Interior
// items (kind 0, one per half node, or per quarter with split 2) of the root first
// (the largest), then of the other levels; leaf items (kind 1, whole node) with refined neighbours before the
// others; cross items (kind 3, kCrossSlicesPerItem slices of the tabulated
// cross-level pairs, widest first).  Float64: all interior items, then all leaf
// items, then the cross items.  Mixed precision: the float32-bound items (interior,
// leaf far field) and the float64-bound items (cross, then near items, kind 2) are
// merged so that every prefix of the queue holds the same fraction of the work of
// both, so that the two pipes of every SM stay busy side by side.
// Paced mode (n32 != nullptr, mixed precision): the float32-bound items in their
// order, then the float64-bound ones, instead of the merged order; *n32 receives the
// number of float32-bound items.
std::vector<int32_t> build_queue(const Plan& P, bool mixed, const ItemCosts& c, int split = 1,
                                 int* n32 = nullptr) {
  std::vector<int32_t> q32, q64, q;
  std::vector<double> w32, w64;
  auto item = [](int node, int kind, int part) { return (node << 4) | (kind << 2) | part; };
  const int parts = mixed ? 2 * split : 2;
  for (int pass = 0; pass < 2; ++pass)
    for (int k : P.interior_nodes)
      if ((P.level[k] == 0) == (pass == 0))
        for (int part = 0; part < parts; ++part) {
          q32.push_back(item(k, 0, part));
          w32.push_back(512.0 / parts * (P.level[k] == 0 ? (double)P.st_root.size() : (double)P.n_st) *
                        c.interior_pair);
        }
  const int n_slices = P.xc_slice_off.empty() ? 0 : (int)P.xc_slice_off.size() - 1;
  if (mixed)  // float64-bound: the cross items head the float64 list
    for (int ci = 0; ci * kCrossSlicesPerItem < n_slices; ++ci) {
      const int s1 = std::min((ci + 1) * kCrossSlicesPerItem, n_slices);
      q64.push_back(item(ci, 3, 0));
      w64.push_back((double)(P.xc_slice_off[s1] - P.xc_slice_off[ci * kCrossSlicesPerItem]) * c.cross_pair);
    }
  std::vector<char> bnd(P.n_nodes, 0);
  for (int k : P.boundary_nodes) bnd[k] = 1;
  for (int pass = 0; pass < 2; ++pass)
    for (int k : P.leaf_nodes)
      if ((bnd[k] != 0) == (pass == 0)) {
        q32.push_back(item(k, 1, 0));
        w32.push_back(c.leaf_far);
        if (mixed) {
          q64.push_back(item(k, 2, 0));
          w64.push_back(c.leaf_near);
        }
      }
  if (!mixed) {  // float64: the cross items last
    for (int ci = 0; ci * kCrossSlicesPerItem < n_slices; ++ci) q32.push_back(item(ci, 3, 0));
    return q32;
  }
  if (n32) {
    *n32 = (int)q32.size();
    q32.insert(q32.end(), q64.begin(), q64.end());
    return q32;
  }
  double t32 = 0, t64 = 0, c32 = 0, c64 = 0;
  for (double v : w32) t32 += v;
  for (double v : w64) t64 += v;
  size_t i = 0, j = 0;
  while (i < q32.size() || j < q64.size()) {
    // take the list whose consumed fraction of its total work is smaller
    const bool take32 = j == q64.size() || (i < q32.size() && c32 * t64 <= c64 * t32);
    if (take32) {
      c32 += w32[i];
      q.push_back(q32[i++]);
    } else {
      c64 += w64[j];
      q.push_back(q64[j++]);
    }
  }
  return q;
}

// (Re)builds the persistent queue for the handle's item costs and interior split
// and copies it to the device, synchronising stream s.
cudaError_t load_queue(octo_fmm* h, cudaStream_t s) {
  const bool paced = h->paced && h->precision == OCTO_MIXED;
  const std::vector<int32_t> q = build_queue(h->plan, h->precision == OCTO_MIXED, h->costs, h->st.interior_split,
                                             paced ? &h->n32 : nullptr);
  if ((int)q.size() > h->queue_cap) return cudaErrorInvalidValue;
  h->n_items = (int)q.size();
  if (q.empty()) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(h->d_queue, q.data(), sizeof(int32_t) * q.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

// Mean time (ms) of one launch of the per-kind stage of `kind` (0 if the stage list
// has none), over five launches on stream ts after a warm-up.
constexpr int kTuneReps = 5;
cudaError_t time_stage(octo_fmm* h, int kind, cudaStream_t ts, cudaEvent_t t0, cudaEvent_t t1, float* ms) {
  *ms = 0.0f;
  for (const auto& st : h->stages) {
    if (st.kind != kind) continue;
    cudaError_t e = enq_stage(h, st, nullptr, nullptr, nullptr, ts);
    if (e == cudaSuccess) e = cudaEventRecord(t0, ts);
    for (int r = 0; r < kTuneReps && e == cudaSuccess; ++r) e = enq_stage(h, st, nullptr, nullptr, nullptr, ts);
    if (e == cudaSuccess) e = cudaEventRecord(t1, ts);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, t0, t1);
    *ms /= (float)kTuneReps;
    return e;
  }
  return cudaSuccess;
}

// Mean time (ms) of the whole interaction phase as the stage list stands, over five
// runs after a warm-up.
cudaError_t time_interact(octo_fmm* h, cudaStream_t ts, cudaEvent_t t0, cudaEvent_t t1, float* ms) {
  *ms = 0.0f;
  cudaError_t e = enq_interact(h, ts);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(t0, ts);
  for (int r = 0; r < kTuneReps && e == cudaSuccess; ++r) e = enq_interact(h, ts);
  if (e == cudaSuccess) e = cudaEventRecord(t1, ts);
  if (e == cudaSuccess) e = cudaEventSynchronize(t1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, t0, t1);
  *ms /= (float)kTuneReps;
  return e;
}

// Project autotuner of the batched interaction phase, run once per handle on the
// private stream (ordered after the caller's pending work) after one upward pass
// with this rho, on the handle's own tree:
//  1. mixed precision: times the item kinds alone (per-kind launches) and rebuilds
//     the persistent queue with the measured item costs;
//  2. schedule: per-kind launches, or the persistent queue under the 1-, 2- and (mixed
//     precision) 3-blocks-per-SM register budgets; keeps the fastest;
//  3. mixed precision, unless options 6 / 7 fixed it: the shape of the interior
//     items under that schedule, one parameter at a time: the stencil entries per
//     float32 partial sum (32, 64), then half-node or quarter-node items.
// The schedule never changes the arithmetic (bit-identical results); the shape
// changes the float32 summation order only (results within the mixed tolerance).
int autotune(octo_fmm* h, const double* rho, cudaStream_t s) {
  cudaStream_t ts = h->cap_stream;
  cudaEvent_t ready = nullptr, t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) e = cudaEventRecord(ready, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ts, ready, 0);
  const bool prof = h->profile;
  h->profile = false;
  if (e == cudaSuccess) e = enq_upward(h, rho, ts);
  struct Cand {
    int mode, minb;
  } cands[4] = {{MODE_PER_KIND, 1}, {MODE_PERSISTENT, 1}, {MODE_PERSISTENT, 2}, {MODE_PERSISTENT, 3}};
  const bool mixed = h->precision == OCTO_MIXED;
  const int n_cands = mixed ? 4 : 3;  // budget 3: mixed precision only
  int best = 0;
  if (e == cudaSuccess && mixed && h->n_items > 0) {
    // 1. measured item costs -> persistent queue
    const Plan& P = h->plan;
    h->mode = MODE_PER_KIND;
    e = rebuild_stages(h);
    float t_int = 0, t_far = 0, t_near = 0, t_cross = 0;
    if (e == cudaSuccess) e = time_stage(h, S_M2L, ts, t0, t1, &t_int);
    if (e == cudaSuccess) e = time_stage(h, S_CONV, ts, t0, t1, &t_far);
    if (e == cudaSuccess) e = time_stage(h, S_NEAR, ts, t0, t1, &t_near);
    if (e == cudaSuccess && h->xc.n_slices > 0) e = time_stage(h, S_CROSS_CELLS, ts, t0, t1, &t_cross);
    if (e == cudaSuccess && t_int > 0 && t_far > 0 && t_near > 0 && P.kernel_pairs[0] > 0 && P.n_leaf > 0) {
      // (the cross pairs' cost in the same unit; the default ratio when there are none)
      const double cross_pair = t_cross > 0 && P.xc_pairs > 0
                                    ? t_cross / (double)P.xc_pairs
                                    : t_near / (double)P.n_leaf / default_costs(P).leaf_near * default_costs(P).cross_pair;
      h->costs = {t_int / (double)P.kernel_pairs[0], t_far / (double)P.n_leaf, t_near / (double)P.n_leaf, cross_pair};
      e = load_queue(h, ts);
    }
  }
  // 2. schedule
  for (int c = 0; c < n_cands && e == cudaSuccess; ++c) {
    h->mode = cands[c].mode;
    h->min_blocks = cands[c].minb;
    e = rebuild_stages(h);
    if (e == cudaSuccess) e = time_interact(h, ts, t0, t1, &h->tune_ms[c]);
    if (h->tune_ms[c] < h->tune_ms[best]) best = c;
  }
  if (e == cudaSuccess) {
    h->mode = cands[best].mode;
    h->min_blocks = cands[best].minb;
    e = rebuild_stages(h);
  }
  // 3. interior shape (mixed precision)
  float t_best = h->tune_ms[best];
  if (e == cudaSuccess && mixed && !h->corr64 && h->requested_shape == 0 && !h->plan.interior_nodes.empty()) {
    h->st.acc_block = 64;
    e = time_interact(h, ts, t0, t1, &h->tune_shape_ms[0]);
    if (e == cudaSuccess && h->tune_shape_ms[0] < t_best)
      t_best = h->tune_shape_ms[0];
    else
      h->st.acc_block = 32;
    if (e == cudaSuccess) {
      h->st.interior_split = 2;
      e = load_queue(h, ts);
      if (e == cudaSuccess) e = time_interact(h, ts, t0, t1, &h->tune_shape_ms[1]);
      if (e == cudaSuccess && h->tune_shape_ms[1] < t_best) {
        t_best = h->tune_shape_ms[1];
      } else if (e == cudaSuccess) {
        h->st.interior_split = 1;
        e = load_queue(h, ts);
      }
    }
    if (e == cudaSuccess) e = rebuild_stages(h);
  }
  // 4. mixed precision under the persistent queue, unless option 8 fixed it: the
  //    paced queue (at most one float64 item per SM at a time) against the merged one
  if (e == cudaSuccess && mixed && h->mode == MODE_PERSISTENT && h->requested_paced == 0) {
    h->paced = true;
    e = load_queue(h, ts);
    if (e == cudaSuccess) e = time_interact(h, ts, t0, t1, &h->tune_shape_ms[2]);
    if (e == cudaSuccess && !(h->tune_shape_ms[2] < t_best)) {
      h->paced = false;
      e = load_queue(h, ts);
    }
    if (e == cudaSuccess) e = rebuild_stages(h);
  }
  h->profile = prof;
  if (ready) cudaEventDestroy(ready);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune");
  return OCTO_OK;
}

// Reports the device error word read back as `err` (OCTO_ENONPOS for a density
// that was not finite and positive, OCTO_ETIMEOUT for a bounded wait that ran out,
// else OCTO_ECUDA for a failed index check of the adjoint) and clears it, so that
// each error is reported once.
int report_device_errors(octo_fmm* h, int err, cudaStream_t s) {
  if (!err) return OCTO_OK;
  cudaError_t e = cudaMemsetAsync(h->d_err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "clear the device error word");
  if (err & kErrDensity)
    return fail(h, OCTO_ENONPOS, "the density of a leaf cell was not finite and positive (NaN, <= 0 or inf)");
  if (err & kErrTimeout)
    return fail(h, OCTO_ETIMEOUT, "a kernel's bounded wait for its own asynchronous copies ran out; results incomplete");
  return fail(h, OCTO_ECUDA, "a device-side index check failed (bits " + std::to_string(err) + ")");
}

}  // namespace

extern "C" {

int octo_fmm_plan_counts(const octo_tree_desc* tree, double theta, int64_t counts[4]) {
  if (!counts) return OCTO_EINVAL;
  Plan P;
  int rc = build_plan(tree, theta, P);
  if (rc != OCTO_OK) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_create_error = P.error;
    return rc;
  }
  for (int i = 0; i < 4; ++i) counts[i] = P.counts[i];
  return OCTO_OK;
}

int octo_fmm_create(const octo_tree_desc* tree, double theta, int order, int precision, octo_fmm_t* out) {
  auto create_fail = [](int code, const std::string& msg) {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_create_error = msg;
    return code;
  };
  if (!out) return create_fail(OCTO_EINVAL, "out is null");
  *out = nullptr;
  {
    const char* v = std::getenv("OCTO_FMM_FAIL_ALLOC_AT");
    t_alloc_count = 0;
    t_alloc_fail_at = v ? std::atoi(v) : 0;
  }
  struct DisarmHook {
    ~DisarmHook() { t_alloc_fail_at = 0; }
  } disarm_hook;
  if (order != 3) return create_fail(OCTO_EINVAL, "only order 3 is supported");
  if (precision != OCTO_FP64 && precision != OCTO_MIXED) return create_fail(OCTO_EINVAL, "unknown precision");
  octo_fmm* h = new (std::nothrow) octo_fmm();
  if (!h) return create_fail(OCTO_ENOMEM, "host allocation failed");
  int rc = build_plan(tree, theta, h->plan);
  if (rc != OCTO_OK) {
    std::string m = h->plan.error;
    delete h;
    return create_fail(rc, m);
  }
  h->precision = precision;
  cudaGetDevice(&h->device);
  Plan& P = h->plan;
  cudaError_t e = cudaSuccess;
  auto up = [&](auto** d, const auto& v) {
    if (e == cudaSuccess) e = upload(d, v);
  };
  up(&h->d_level, P.level);
  up(&h->d_parent, P.parent);
  up(&h->d_octant, P.octant);
  up(&h->d_children, P.children);
  up(&h->d_nbr, P.nbr);
  up(&h->d_leaf_id, P.leaf_id);
  up(&h->d_ijk, P.ijk);
  up(&h->d_interior, P.interior_nodes);
  up(&h->d_leaf, P.leaf_nodes);
  up(&h->d_boundary, P.boundary_nodes);
  up(&h->d_st_parity, P.st_parity);
  up(&h->d_st_root, P.st_root);
  up(&h->d_st_near, P.st_near);
  std::vector<int32_t> st_pair, st_pair_root;
  const int n_pair = build_pair_tables(P.st_parity.data(), P.n_st, true, st_pair);
  const int n_pair_root = build_pair_tables(P.st_root.data(), (int)P.st_root.size(), false, st_pair_root);
  if (precision == OCTO_MIXED) {
    std::vector<int32_t> cell_pair, cell_pair_off;
    build_cell_pair_lists(P.cell_ent, P.cell_ent_off, cell_pair, cell_pair_off);
    up(&h->d_st_pair, st_pair);
    up(&h->d_st_pair_root, st_pair_root);
    up(&h->d_cell_pair, cell_pair);
    up(&h->d_cell_pair_off, cell_pair_off);
  }
  int R = 7;
  for (int32_t v : P.st_parity)
    for (int k = 0; k < 3; ++k) R = std::max(R, std::abs((int)(int8_t)((v >> (8 * k)) & 0xff)));
  std::vector<Kappa> kap = make_kappa(R);
  up(&h->d_kappa, kap);
  if (e == cudaSuccess) e = upload_cross(P, P.xg_targets, P.xg_start, P.xg_mid, P.xg_sources, h->xg);
  up(&h->d_xc_t, P.xc_targets);
  up(&h->d_xc_off, P.xc_slice_off);
  up(&h->d_xc_ent, P.xc_entries);
  up(&h->d_xc_tab, P.xc_table);
  if (e == cudaSuccess) e = dev_malloc(&h->d_xc_counter, sizeof(int));
  up(&h->d_cell_ent, P.cell_ent);
  up(&h->d_cell_ent_off, P.cell_ent_off);
  up(&h->d_bnd_perm, P.bnd_perm);
  up(&h->d_bnd_index, P.bnd_index);
  const int64_t NC = (int64_t)P.n_nodes * kCells;
  if (e == cudaSuccess) e = dev_malloc(&h->d_mp, sizeof(double) * N_MP * NC);
  if (e == cudaSuccess) e = dev_malloc(&h->d_loc, sizeof(double) * N_LOC * NC);
  if (e == cudaSuccess && precision == OCTO_MIXED) e = dev_malloc(&h->d_mp32, sizeof(float) * N_MP * NC);
  if (e == cudaSuccess && precision == OCTO_MIXED) e = dev_malloc(&h->d_near, sizeof(double) * 4 * h->n_leaf_cells());
  if (e == cudaSuccess && P.xc_slice_off.size() > 1)
    e = dev_malloc(&h->d_xcf, sizeof(double) * 4 * 32 * (P.xc_slice_off.size() - 1));
  if (e == cudaSuccess) e = dev_malloc(&h->d_io, sizeof(double) * 5 * h->n_leaf_cells());
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    std::string m = std::string("device setup failed: ") + cudaGetErrorString(e);
    bool oom = e == cudaErrorMemoryAllocation;
    free_all(h);
    delete h;
    return create_fail(oom ? OCTO_ENOMEM : OCTO_ECUDA, m);
  }
  DevTree& t = h->dt;
  t.NC = NC;
  t.n_nodes = P.n_nodes;
  t.level = h->d_level;
  t.parent = h->d_parent;
  t.octant = h->d_octant;
  t.children = h->d_children;
  t.nbr = h->d_nbr;
  t.leaf_id = h->d_leaf_id;
  t.ijk = h->d_ijk;
  for (int d = 0; d < 3; ++d) t.origin[d] = P.origin[d];
  for (int l = 0; l < 16; ++l) {
    double hl = cell_width(P, l);
    t.h[l] = hl;
    t.h3[l] = hl * hl * hl;
  }
  int RN = 0, far_blocks = 0, root_blocks = 0;
  for (int32_t v : P.st_near)
    for (int k = 0; k < 3; ++k) RN = std::max(RN, std::abs((int)(int8_t)((v >> (8 * k)) & 0xff)));
  {  // leaf-item tables (halo offsets and kernel rows per parity class and entry)
    const int ns = P.n_st, nr = (int)P.st_root.size(), nn = (int)P.st_near.size();
    std::vector<int2> lf((size_t)8 * ns), lr((size_t)8 * nr), ln((size_t)8 * nn);
    build_leaf_tables(P.st_parity.data(), ns, P.st_root.data(), nr, P.st_near.data(), nn, R, RN,
                      precision == OCTO_MIXED, lf.data(), lr.data(), ln.data());
    e = upload(&h->d_leaf_far, lf);
    if (e == cudaSuccess) e = upload(&h->d_leaf_root, lr);
    if (e == cudaSuccess) e = upload(&h->d_leaf_near, ln);
    if (precision == OCTO_MIXED) {
      // z-column blocks (see kLeafBlock): parity stencils, then level 0
      std::vector<uint32_t> words;
      far_blocks = build_leaf_column_blocks(P.st_parity.data(), ns, true, R, kap.data(), words);
      root_blocks = build_leaf_column_blocks(P.st_root.data(), nr, false, R, kap.data(), words);
      std::vector<uint4> blk(words.size() / 4);
      std::memcpy(blk.data(), words.data(), sizeof(uint32_t) * words.size());
      if (e == cudaSuccess) e = upload(&h->d_leaf_blocks, blk);
    }
    if (e != cudaSuccess) {
      std::string m = std::string("device setup failed: ") + cudaGetErrorString(e);
      free_all(h);
      delete h;
      return create_fail(e == cudaErrorMemoryAllocation ? OCTO_ENOMEM : OCTO_ECUDA, m);
    }
  }
  h->st = Stencils{h->d_st_parity, P.n_st,       h->d_st_root,   (int)P.st_root.size(), h->d_st_pair, n_pair,
                   h->d_st_pair_root, n_pair_root, h->d_st_near,
                   (int)P.st_near.size(), h->d_kappa, h->d_leaf_blocks, far_blocks, root_blocks, R, RN,
                   h->d_cell_ent, h->d_cell_ent_off, h->d_cell_pair, h->d_cell_pair_off, h->d_bnd_perm,
                   h->d_bnd_index, h->d_leaf_far, h->d_leaf_root, h->d_leaf_near, h->d_err};
  h->xc = CrossCells{h->d_xc_t, h->d_xc_off, h->d_xc_ent, h->d_xc_tab, (int)(P.xc_slice_off.size() - 1),
                     (int)(P.xc_table.size() / 4), h->d_xc_counter};
  e = launch_init_leaf(t, h->d_leaf, (int)P.leaf_nodes.size(), h->d_mp, h->d_mp32, h->cap_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->cap_stream);
  if (e != cudaSuccess) {
    std::string m = std::string("init failed: ") + cudaGetErrorString(e);
    free_all(h);
    delete h;
    return create_fail(OCTO_ECUDA, m);
  }
  // persistent work queue (see build_queue); mixed precision: estimated item costs
  // until the autotuner has measured them
  {
    h->costs = default_costs(P);
    h->queue_cap = (int)build_queue(P, precision == OCTO_MIXED, h->costs, precision == OCTO_MIXED ? 2 : 1).size();
    e = h->queue_cap > 0 ? dev_malloc(&h->d_queue, sizeof(int32_t) * h->queue_cap) : cudaSuccess;
    if (e == cudaSuccess) e = load_queue(h, h->cap_stream);
    if (e == cudaSuccess) e = dev_malloc(&h->d_counter, sizeof(int) * (2 + kPaceFlags));
    if (e == cudaSuccess) e = dev_malloc(&h->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(int));
    h->st.err = h->d_err;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = configure_interact_kernels();
    for (int mb = 1; mb <= (precision == OCTO_MIXED ? 3 : 2) && e == cudaSuccess; ++mb)
      e = persistent_blocks_per_sm(precision == OCTO_MIXED, mb, h->st, h->xc, &h->persist_per_sm[mb]);
    int xc_per_sm = 0;
    if (e == cudaSuccess && h->xc.n_slices > 0) e = cross_cells_blocks_per_sm(h->xc, &xc_per_sm);
    h->xc_grid = h->n_sm * std::max(xc_per_sm, 1);
    if (e != cudaSuccess) {
      std::string m = std::string("work queue setup failed: ") + cudaGetErrorString(e);
      free_all(h);
      delete h;
      return create_fail(e == cudaErrorMemoryAllocation ? OCTO_ENOMEM : OCTO_ECUDA, m);
    }
  }
  h->mode = MODE_PER_KIND;  // until the autotuner (or option 3) decides
  e = rebuild_stages(h);
  if (e != cudaSuccess) {
    free_all(h);
    delete h;
    return create_fail(OCTO_ECUDA, "event creation failed");
  }
  *out = h;
  return OCTO_OK;
}

int octo_fmm_upward(octo_fmm_t h, const double* rho, void* stream) {
  if (!h || !rho) return h ? fail(h, OCTO_EINVAL, "rho is null") : OCTO_EINVAL;
  h->forward_done = false;
  h->phase = 0;
  cudaError_t e = enq_upward(h, rho, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "upward");
  h->phase = 1;
  return OCTO_OK;
}

int octo_fmm_interact(octo_fmm_t h, void* stream) {
  if (!h) return OCTO_EINVAL;
  h->forward_done = false;
  const bool after_upward = h->phase == 1;
  h->phase = 0;
  cudaError_t e = enq_interact(h, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "interact");
  if (after_upward) h->phase = 2;
  return OCTO_OK;
}

int octo_fmm_downward(octo_fmm_t h, double* phi, double* g, void* stream) {
  if (!h || !phi || !g) return h ? fail(h, OCTO_EINVAL, "phi or g is null") : OCTO_EINVAL;
  cudaError_t e = enq_downward(h, phi, g, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "downward");
  // the state is that of one whole solve only if upward and interact preceded this
  if (h->phase == 2) h->forward_done = true;
  h->phase = 0;
  return OCTO_OK;
}

int octo_fmm_forces(octo_fmm_t h, const double* rho, double* phi, double* g, void* stream) {
  if (!h || !rho || !phi || !g) return h ? fail(h, OCTO_EINVAL, "null buffer") : OCTO_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  h->forward_done = false;
  h->phase = 0;
  if (h->requested_mode == MODE_AUTO && h->tune_ms[0] == 0.0f) {
    int rc = autotune(h, rho, s);
    if (rc != OCTO_OK) return rc;
  }
  if (!h->use_graph) {
    cudaError_t e = enq_solve(h, rho, phi, g, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "forces");
    h->forward_done = true;
    return OCTO_OK;
  }
  if (!h->gexec || h->g_rho != rho || h->g_phi != phi || h->g_g != g) {
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "begin capture");
    cudaError_t el = enq_solve(h, rho, phi, g, h->cap_stream);
    e = cudaStreamEndCapture(h->cap_stream, &graph);
    if (el != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(h, el, "capture launches");
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      h->gexec = nullptr;
      return cuda_fail(h, e, "instantiate graph");
    }
    h->g_rho = rho;
    h->g_phi = phi;
    h->g_g = g;
  }
  cudaError_t e = cudaGraphLaunch(h->gexec, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
  h->forward_done = true;
  return OCTO_OK;
}

int octo_fmm_forces_host(octo_fmm_t h, const double* rho_host, double* phi_host, double* g_host, void* stream) {
  if (!h || !rho_host || !phi_host || !g_host) return h ? fail(h, OCTO_EINVAL, "null buffer") : OCTO_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = h->n_leaf_cells();
  double* d_rho = h->d_io;
  double* d_phi = h->d_io + n;
  double* d_g = h->d_io + 2 * n;
  // Straight between the caller's (pageable) buffers and the device: on a Grace host
  // the copy engines read and write pageable memory through the coherent link at the
  // same rate as pinned memory, so a host-side staging copy would only add time.
  // (Splitting the copies over several streams gained nothing: a copy to pageable
  // memory returns only once it is done, so the copies run one after another.)
  cudaError_t e = cudaMemcpyAsync(d_rho, rho_host, sizeof(double) * n, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "copy rho in");
  int rc = octo_fmm_forces(h, d_rho, d_phi, d_g, stream);
  if (rc != OCTO_OK) return rc;
  e = cudaMemcpyAsync(phi_host, d_phi, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g_host, d_g, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s);
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(h, e, "copy results out");
  return report_device_errors(h, err, s);
}

int octo_fmm_backward(octo_fmm_t h, const double* dphi, const double* dg, double* drho, void* stream) {
  if (!h || !dphi || !dg || !drho) return h ? fail(h, OCTO_EINVAL, "null buffer") : OCTO_EINVAL;
  if (!h->forward_done) return fail(h, OCTO_ESTATE, "backward needs a forward solve on this handle");
  const Plan& P = h->plan;
  const int64_t NC = (int64_t)P.n_nodes * kCells;
  cudaError_t e = cudaSuccess;
  if (!h->d_mpb) {  // adjoint workspace, allocated on first use
    std::vector<int32_t> general(P.interior_nodes);
    general.insert(general.end(), P.boundary_nodes.begin(), P.boundary_nodes.end());
    h->n_general = (int)general.size();
    e = upload(&h->d_general, general);
    // the adjoint kernels keep large per-thread frames: make sure the stack limit covers them
    size_t need = 0, cur = 0;
    if (e == cudaSuccess) e = adjoint_local_bytes(&need);
    if (e == cudaSuccess) e = cudaDeviceGetLimit(&cur, cudaLimitStackSize);
    if (e == cudaSuccess && cur < need) e = cudaDeviceSetLimit(cudaLimitStackSize, need);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_mpb, sizeof(double) * N_MP * NC);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_locb, sizeof(double) * N_LOC * NC);
    if (e != cudaSuccess) {
      cudaFree(h->d_mpb);
      cudaFree(h->d_locb);
      h->d_mpb = h->d_locb = nullptr;
      return e == cudaErrorMemoryAllocation ? fail(h, OCTO_ENOMEM, "adjoint workspace") : cuda_fail(h, e, "backward setup");
    }
  }
  BackwardArgs ba;
  ba.mp = h->d_mp;
  ba.loc = h->d_loc;
  ba.mpb = h->d_mpb;
  ba.locb = h->d_locb;
  ba.phib = dphi;
  ba.gb = dg;
  ba.rhob = drho;
  ba.NL = h->n_leaf_cells();
  ba.leaf_nodes = h->d_leaf;
  ba.n_leaf_nodes = (int)P.leaf_nodes.size();
  ba.general_nodes = h->d_general;
  ba.n_general = h->n_general;
  ba.level_start = P.level_start.data();
  ba.max_level = P.max_level;
  ba.st = h->st;
  ba.xf = h->xg.f;  // the same cross-level lists as the forward (both directions of every pair)
  ba.xl = h->xg.l;
  ba.xc = h->xc;
  ba.xc_grid = h->xc_grid;
  ba.err = h->d_err;
  e = launch_backward(h->dt, ba, (cudaStream_t)stream);
  return e == cudaSuccess ? OCTO_OK : cuda_fail(h, e, "backward");
}

int octo_fmm_stats(octo_fmm_t h, int64_t counts[4]) {
  if (!h || !counts) return OCTO_EINVAL;
  for (int i = 0; i < 4; ++i) counts[i] = h->plan.counts[i];
  int err = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "stats");
  return report_device_errors(h, err, nullptr);
}

int octo_fmm_read_state(octo_fmm_t h, int which, double* out) {
  if (!h || !out || (which != 0 && which != 1)) return h ? fail(h, OCTO_EINVAL, "bad arguments") : OCTO_EINVAL;
  const Plan& P = h->plan;
  const int nf = which == 0 ? N_MP : N_LOC;
  const int64_t NC = (int64_t)P.n_nodes * kCells;
  std::vector<double> buf((size_t)nf * NC);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(buf.data(), which == 0 ? h->d_mp : h->d_loc, sizeof(double) * nf * NC, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "read state");
  for (int f = 0; f < nf; ++f)
    for (int i = 0; i < P.n_nodes; ++i) {
      int k = P.dnode_of_desc[i];
      bool leaf = P.children[8 * k] < 0;
      for (int c = 0; c < kCells; ++c) {
        double v = buf[(size_t)f * NC + (size_t)k * kCells + c];
        if (which == 1 && leaf && f >= G_L2 && f < G_DG) v = NAN;
        out[(size_t)f * NC + (size_t)i * kCells + c] = v;
      }
    }
  return OCTO_OK;
}

int octo_fmm_set_option(octo_fmm_t h, int key, int64_t value) {
  if (!h) return OCTO_EINVAL;
  if (key == 1 && (value == 0 || value == 1)) {
    h->use_graph = value != 0;
    return OCTO_OK;
  }
  if (key == 0 && value >= 0) return OCTO_OK;
  if (key == 5 && (value == 0 || value == 1) && h->precision == OCTO_MIXED) {
    // the float64-correction variant runs as per-kind launches of half-node items
    h->corr64 = value != 0;
    cudaError_t e = cudaSuccess;
    if (h->corr64) {
      h->requested_mode = h->mode = MODE_PER_KIND;
      h->st.interior_split = 1;
      e = load_queue(h, h->cap_stream);
    }
    if (e == cudaSuccess) e = rebuild_stages(h);
    return e == cudaSuccess ? OCTO_OK : cuda_fail(h, e, "set correction precision");
  }
  if (key == 6 && (value == 32 || value == 64)) {
    h->st.acc_block = (int)value;
    h->requested_shape = 1;
    cudaError_t e = rebuild_stages(h);
    return e == cudaSuccess ? OCTO_OK : cuda_fail(h, e, "set chunk length");
  }
  if (key == 8 && (value == 0 || value == 1) && h->precision == OCTO_MIXED) {
    h->paced = value != 0;
    h->requested_paced = 1;
    cudaError_t e = load_queue(h, h->cap_stream);
    if (e == cudaSuccess) e = rebuild_stages(h);
    return e == cudaSuccess ? OCTO_OK : cuda_fail(h, e, "set paced queue");
  }
  if (key == 7 && (value == 1 || (value == 2 && h->precision == OCTO_MIXED && !h->corr64))) {
    h->st.interior_split = (int)value;
    h->requested_shape = 1;
    cudaError_t e = load_queue(h, h->cap_stream);
    if (e == cudaSuccess) e = rebuild_stages(h);
    return e == cudaSuccess ? OCTO_OK : cuda_fail(h, e, "set interior split");
  }
  if (key == 3 && value >= MODE_AUTO && value <= MODE_PERSISTENT) {
    if (h->corr64 && value != MODE_PER_KIND)
      return fail(h, OCTO_EINVAL, "the float64-correction variant runs as per-kind launches only");
    h->requested_mode = (int)value;
    if (value != MODE_AUTO) h->mode = (int)value;
    cudaError_t e = rebuild_stages(h);
    return e == cudaSuccess ? OCTO_OK : cuda_fail(h, e, "set strategy");
  }
  if (key == 4 && (value == 1 || value == 2 || (value == 3 && h->precision == OCTO_MIXED))) {
    h->min_blocks = (int)value;
    cudaError_t e = rebuild_stages(h);
    return e == cudaSuccess ? OCTO_OK : cuda_fail(h, e, "set blocks");
  }
  if (key == 2 && (value == 0 || value == 1)) {
    h->profile = value != 0;
    if (h->gexec) {  // re-capture with or without the timing events
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    return OCTO_OK;
  }
  return fail(h, OCTO_EINVAL, "unknown option");
}

int octo_fmm_stage_count(octo_fmm_t h) { return h ? (int)h->stages.size() : 0; }

int octo_fmm_stage_info(octo_fmm_t h, int i, const char** name, int64_t* pairs, int64_t* cells, int64_t* flops,
                        int64_t* flops64, int64_t* bytes) {
  if (!h || i < 0 || i >= (int)h->stages.size()) return OCTO_EINVAL;
  if (name) *name = h->stages[i].name.c_str();
  if (pairs) *pairs = h->stages[i].pairs;
  if (cells) *cells = h->stages[i].cells;
  if (flops) *flops = h->stages[i].flops;
  if (flops64) *flops64 = h->stages[i].flops64;
  if (bytes) *bytes = h->stages[i].bytes;
  return OCTO_OK;
}

int octo_fmm_stage_times(octo_fmm_t h, float* ms, int cap) {
  if (!h || !ms) return OCTO_EINVAL;
  if (!h->profile) return fail(h, OCTO_ESTATE, "stage profiling is off (option 2)");
  const int n = (int)h->stages.size();
  if (cap < n) return fail(h, OCTO_EINVAL, "buffer too small");
  for (int i = 0; i < n; ++i) {
    cudaError_t e = cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]);
    if (e != cudaSuccess) return cuda_fail(h, e, "stage times");
  }
  return n;
}

int octo_fmm_launches_per_solve(octo_fmm_t h) { return h ? count_launches(h) : 0; }

int octo_fmm_get_option(octo_fmm_t h, int key, int64_t* value) {
  if (!h || !value) return OCTO_EINVAL;
  switch (key) {
    case 1: *value = h->use_graph ? 1 : 0; return OCTO_OK;
    case 2: *value = h->profile ? 1 : 0; return OCTO_OK;
    case 3: *value = h->mode; return OCTO_OK;
    case 4: *value = h->min_blocks; return OCTO_OK;
    case 5: *value = h->corr64 ? 1 : 0; return OCTO_OK;
    case 6: *value = h->st.acc_block; return OCTO_OK;
    case 7: *value = h->st.interior_split; return OCTO_OK;
    case 8: *value = h->paced ? 1 : 0; return OCTO_OK;
    case 14:
    case 15:
    case 16: *value = (int64_t)(1000.0f * h->tune_shape_ms[key - 14]); return OCTO_OK;
    case 10:
    case 11:
    case 12:
    case 13: *value = (int64_t)(1000.0f * h->tune_ms[key - 10]); return OCTO_OK;
    case 24: {
      // algorithmic float64 flops of one octo_fmm_backward over its pair kinds: every
      // same-level M2L pair twice (as target: centre and octupole adjoints; as
      // source: centre, mass and moments), leaf-leaf and tabulated cross-level pairs
      // (4 fused multiply-adds each), the general cross-level lists likewise; the
      // tree passes (L2L, M2M, P2M, L2P transposes) are not counted
      const Plan& P = h->plan;
      const int64_t a = vjp_flops<true, true, false, true>(), bf = vjp_flops<true, true, true, false>(),
                    bl = vjp_flops<false, false, true, false>();
      int64_t f = P.kernel_pairs[0] * (a + bf) + P.kernel_pairs[3] * bl;
      f += (P.kernel_pairs[1] + P.kernel_pairs[2] + P.xc_pairs) * kConvFlopsPerPair;
      f += (h->xg.f_pairs - h->xg.f_p2p) * (a + bf) + (h->xg.l_pairs - h->xg.l_p2p) * bl;
      f += (h->xg.f_p2p + h->xg.l_p2p) * 2 * kP2PFlopsPerPair;
      *value = f;
      return OCTO_OK;
    }
    case 20: *value = h->n_leaf_cells(); return OCTO_OK;
    case 21: *value = h->device; return OCTO_OK;
    case 22: *value = h->plan.n_nodes; return OCTO_OK;
    case 23: *value = h->precision; return OCTO_OK;
  }
  return fail(h, OCTO_EINVAL, "unknown option");
}

const char* octo_fmm_last_error(octo_fmm_t h) {
  if (h) return h->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_create_error.c_str();
}

void octo_fmm_destroy(octo_fmm_t h) {
  if (!h) return;
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
}

}  // extern "C"
