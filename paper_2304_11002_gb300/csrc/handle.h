// The solver handle behind the C ABI's opaque octo_fmm_t: the plan, the device
// workspace and the state of the batched solve.  Shared by the translation units
// that implement entry points (capi.cu, scf.cu); nothing outside the library sees it.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/octo_fmm.h"
#include "kernels.h"
#include "plan.h"

namespace octo {

// Cross-level pair lists on the device, split by target: refined target cells
// (full local expansion) and leaf target cells.  CSR per target, far partners
// before near ones.
struct CrossSet {
  int64_t *d_ft = nullptr, *d_fs = nullptr, *d_fm = nullptr, *d_fsrc = nullptr;
  int64_t *d_lt = nullptr, *d_ls = nullptr, *d_lm = nullptr, *d_lsrc = nullptr;
  int n_f = 0, n_l = 0;
  int64_t f_pairs = 0, l_pairs = 0, f_p2p = 0, l_p2p = 0;  // entries, of which near
  CrossList f{}, l{};
};

// Work of the persistent queue's items, in any common unit: per M2L pair of an
// interior item, per leaf node for the far-field item and for the near item.
struct ItemCosts {
  double interior_pair, leaf_far, leaf_near, cross_pair;
};

}  // namespace octo

using namespace octo;  // internal header: the handle is defined in terms of the library's types

struct octo_fmm {
  Plan plan;
  int precision = OCTO_FP64;
  int device = 0;
  std::string err;

  // tree and lists
  int *d_level = nullptr, *d_parent = nullptr, *d_octant = nullptr, *d_children = nullptr, *d_nbr = nullptr,
      *d_leaf_id = nullptr, *d_ijk = nullptr;
  int *d_interior = nullptr, *d_leaf = nullptr, *d_boundary = nullptr;
  int *d_st_parity = nullptr, *d_st_root = nullptr, *d_st_near = nullptr;
  int *d_st_pair = nullptr, *d_st_pair_root = nullptr;  // x-pair stencils of the mixed interior items
  int *d_cell_pair = nullptr, *d_cell_pair_off = nullptr;  // x-pair lists of the mixed boundary pairs
  Kappa* d_kappa = nullptr;
  // cross-level pairs: tabulated point-mass pairs and the general remainder (both
  // directions of every pair, so the adjoint gathers over the same lists)
  int64_t *d_xc_t = nullptr, *d_xc_off = nullptr, *d_xc_ent = nullptr;
  double* d_xc_tab = nullptr;
  int* d_xc_counter = nullptr;
  CrossCells xc{};
  int xc_grid = 0;
  CrossSet xg;
  // batched interaction phase: strategy (MODE_*), persistent work queue and counter
  int mode = 0, requested_mode = 0;
  bool corr64 = false;  // mixed precision: correction terms in float64 (option 5)
  int requested_paced = 0;  // 1: option 8 fixed the paced queue
  int requested_shape = 0;  // 0: the autotuner picks the interior shape; 1: set by options 6 / 7
  float tune_shape_ms[3] = {0, 0, 0};  // autotune: chunk 64, quarter-node split, paced queue
  int min_blocks = 1, n_sm = 0;
  int persist_per_sm[4] = {0, 0, 0, 0};  // resident blocks per SM of the persistent variants (index = budget)
  int* d_queue = nullptr;  // sized for the largest queue (interior split 2)
  int n_items = 0, queue_cap = 0;
  bool paced = false;  // mixed precision: two queues, at most one float64 item per SM (option 8)
  int n32 = 0;         // paced queue: number of float32-bound items (they come first)
  ItemCosts costs{};  // item costs the queue is ordered by (estimates, then the autotuner's)
  int* d_counter = nullptr;
  int* d_err = nullptr;  // device-side check word of the adjoint kernels
  float tune_ms[4] = {0, 0, 0, 0};  // measured interaction time per strategy candidate (autotune)
  double *d_mpb = nullptr, *d_locb = nullptr;  // adjoint workspace
  int* d_general = nullptr;
  int n_general = 0;
  int *d_cell_ent = nullptr, *d_cell_ent_off = nullptr, *d_bnd_index = nullptr;
  int2 *d_leaf_far = nullptr, *d_leaf_root = nullptr, *d_leaf_near = nullptr;
  unsigned short* d_bnd_perm = nullptr;

  // state
  double *d_mp = nullptr, *d_loc = nullptr;
  float* d_mp32 = nullptr;    // float32 multipoles (mixed precision only)
  double* d_near = nullptr;   // [4][leaf cells] near-field sums (mixed precision only)
  double* d_xcf = nullptr;    // [4][32 x cross slices] sums of the persistent kernel's cross items
  uint4* d_leaf_blocks = nullptr;  // mixed only: the leaf far tables in 32-entry blocks (items.cuh)
  DevTree dt;
  Stencils st;
  // Forward state for the adjoint: set once a whole solve has been enqueued (forces,
  // or upward, interact and downward in that order); an upward or interact call
  // starts a new solve and clears it until the solve is complete.
  bool forward_done = false;
  int phase = 0;  // 1 after upward, 2 after upward + interact
  bool use_graph = true;

  // host-buffer path (rho, phi, g), also the SCF iteration's phi and g
  double* d_io = nullptr;
  // SCF initial models (scf.cu): reduction partials and constants, leaf-to-node map
  double* d_scf = nullptr;
  int* d_scf_nodes = nullptr;

  // the solve as a fixed list of stages, one kernel launch each
  struct Stage {
    int kind;   // see enum StageKind
    int a, b;   // level range or list selector
    std::string name;
    int64_t pairs;  // interactions processed (0 for tree passes)
    int64_t cells;  // cells processed
    int64_t flops;  // algorithmic floating-point operations
    int64_t flops64;  // of which in float64
    int64_t bytes;  // algorithmic HBM bytes of the tree passes
  };
  std::vector<Stage> stages;
  bool profile = false;
  std::vector<cudaEvent_t> ev;

  // graph
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const double* g_rho = nullptr;
  double *g_phi = nullptr, *g_g = nullptr;

  int64_t n_leaf_cells() const { return (int64_t)plan.n_leaf * kCells; }
};
