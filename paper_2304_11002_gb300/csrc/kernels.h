// Launchers of the solver's kernels (host side).  Every launcher enqueues on
// `stream` and returns the cudaError_t of the launch.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "device.cuh"
#include "tables.h"

namespace octo {

struct Stencils {
  const int* parity;  // [8][n_st] packed offsets
  int n_st;
  const int* root;    // level-0 far offsets
  int n_root;
  // Mixed path's interior items: the stencils grouped into aligned x-pairs of source
  // cells per parity class (build_pair_tables): packed offset of the even cell, bit
  // 24 / 25 set when the even / odd cell is in the stencil.
  const int* pair;       // [8][n_pair]       parity stencils
  int n_pair;
  const int* pair_root;  // [8][n_pair_root]  level-0 stencil
  int n_pair_root;
  const int* near_;   // non-zero near offsets
  int n_near;
  const Kappa* kappa;    // dense monopole kernel table over [-R, R]^3, unit cell width
  const uint4* leaf_blocks;  // mixed path: the leaf far-field tables as blocks of z-column
                             // chunks (see kLeafBlock in tables.h; 640 bytes each):
                             // [8][far_blocks] for the parity stencils, then
                             // [8][root_blocks] for the level-0 stencil
  int far_blocks, root_blocks;
  int radius;            // R: maximum |offset component|
  int near_radius;       // maximum |offset component| of the near offsets
  const int* cell_ent;   // parity offsets per (cell, neighbour slot), see Plan::cell_ent
  const int* cell_ent_off;
  const int* cell_pair;      // mixed path: the lists of cell_ent grouped into x-pairs of
  const int* cell_pair_off;  // source cells (build_cell_pair_lists), same indexing
  const unsigned short* bnd_perm;  // per boundary leaf node: its 512 cells by decreasing load
  const int* bnd_index;            // per node: row of bnd_perm or -1
  // Leaf items, per parity class p of the target cell and stencil entry s:
  // {offset into the shared-memory mass halo, row of kappa} (see items.cuh).
  const int2* leaf_far;   // [8][n_st]   parity stencil (far halo)
  const int2* leaf_root;  // [8][n_root] level-0 stencil (far halo)
  const int2* leaf_near;  // [8][n_near] near offsets (mixed: near float64 halo; float64: far halo)
  // Shape of the mixed-precision interior items, chosen by the autotuner:
  int* err = nullptr;       // device error word of the handle (kErrTimeout: a bounded wait ran out)
  int acc_block = 32;       // stencil entries per float32 partial sum before the compensated merge (32, 64)
  int interior_split = 1;   // 1: an item is half a node, one thread per target cell;
                            // 2: an item is a quarter node, two threads per target cell (one
                            //    stencil half each, merged at the end)
};

// Host: the leaf-item tables above for the given stencils and precision mode.
void build_leaf_tables(const int* parity, int n_st, const int* root, int n_root, const int* near_, int n_near, int R,
                       int RN, bool mixed, int2* far_out, int2* root_out, int2* near_out);

struct CrossList {
  const int64_t* targets;
  const int64_t* start;
  const int64_t* sources;
  int n_targets;
  const int64_t* mid;    // per target: first near (P2P) partner; far (M2L) partners precede it
};

// Cross-level pairs of two leaf cells one level apart, tabulated (SELL-32 layout
// and entry encoding as built by the planner: see Plan::xc_* in plan.h).
struct CrossCells {
  const int64_t* targets;    // [32 * n_slices], -1 for padding lanes
  const int64_t* slice_off;  // [n_slices + 1]
  const int64_t* entries;
  const double* table;       // [n_rows][4]
  int n_slices;
  int n_rows;
  int* counter;              // device scratch: next slice to claim (reset by the launcher)
};
// SM ids covered by the per-SM flags of the persistent kernel's paced mode (larger
// ids are not paced); the work counters are 2 + kPaceFlags ints.
constexpr int kPaceFlags = 1024;
// Slices of one cross item of the persistent interaction kernel (kind 3).
constexpr int kCrossSlicesPerItem = 64;

// ------------------------------------------------------------ tree passes (kernels_fp64.cu)
// mp32 (may be null): float32 copy of the multipoles for the mixed-precision path.
cudaError_t launch_init_leaf(const DevTree& t, const int* leaf_nodes, int n_leaf_nodes, double* mp, float* mp32,
                             cudaStream_t s);
// err: device word; kErrDensity is set when a density is not finite and positive.
cudaError_t launch_p2m(const DevTree& t, const int* leaf_nodes, int n_leaf_nodes, const double* rho, double* mp,
                       float* mp32, int* err, cudaStream_t s);
cudaError_t launch_m2m(const DevTree& t, int node_begin, int node_end, double* mp, float* mp32, cudaStream_t s);
// nearf (may be null): [4][n_leaf_cells] near-field L0, L1 of the leaf cells, added at L2P.
cudaError_t launch_l2l(const DevTree& t, int node_begin, int node_end, const double* mp, double* loc, double* phi,
                       double* g, int64_t n_leaf_cells, const double* nearf, cudaStream_t s);

// ------------------------------------------------------------ same-level interactions (kernels_interact.cu)
struct InteractArgs {
  const double* mp;
  const float* mp32;   // mixed precision only
  double* loc;
  Stencils st;
  bool mixed;
  const int* interior; // refined nodes (all levels)
  int n_interior;
  const int* leaf;     // leaf nodes (all levels)
  int n_leaf;
  double* nearf;       // mixed precision: [4][NL] near-field sums of the leaf cells (near items)
  int64_t NL;          // leaf cells
  const int* queue;    // persistent queue: (node << 4) | (kind << 2) | part, see kernels_interact.cu
  int n_items;
  int* counter;        // work counters of the persistent launch (device scratch, 2 + 1024 ints)
  int n32 = -1;        // paced mode: float32-bound items first in the queue (see interact.cuh), else -1
  int grid;            // blocks of the persistent launch (SMs x resident blocks per SM)
  int min_blocks;      // launch-bounds variant of the persistent kernel (1, 2 or 3)
  CrossCells xc;       // tabulated cross-level pairs: cross items of the persistent queue
  double* xcf;         // [4][32 * xc.n_slices] their per-slot sums (persistent mode)
  bool corr64 = false; // mixed precision: the angular-momentum correction in float64
                       // (measurement variant; per-kind launches only)
};
// Once per process and device (opts the leaf-item kernels into large shared memory).
cudaError_t configure_interact_kernels();
// Resident blocks per SM of the persistent kernel variant (also sets its shared
// memory limit); call outside stream capture.
cudaError_t persistent_blocks_per_sm(bool mixed, int min_blocks, const Stencils& st, const CrossCells& xc,
                                     int* per_sm);
cudaError_t launch_interior_items(const DevTree& t, const InteractArgs& a, cudaStream_t s);
cudaError_t launch_leaf_items(const DevTree& t, const InteractArgs& a, cudaStream_t s);
cudaError_t launch_near_items(const DevTree& t, const InteractArgs& a, cudaStream_t s);  // mixed precision only
cudaError_t launch_persistent(const DevTree& t, const InteractArgs& a, cudaStream_t s);

// ------------------------------------------------------------ cross-level pairs (kernels_boundary.cu)
// corr64 (mixed only): the angular-momentum correction of the far pairs in float64.
cudaError_t launch_cross_list(const DevTree& t, const CrossList& xl, bool full, const double* mp, double* loc,
                              bool mixed, cudaStream_t s, bool corr64 = false);
// Tabulated point-mass pairs, float64 in both precision modes.  grid: a multiple of
// the SM count (cross_cells_blocks_per_sm gives the resident blocks per SM).
cudaError_t cross_cells_blocks_per_sm(const CrossCells& xc, int* blocks);
// Adjoint of the tabulated pairs: mpb (mass part) of every list target from the
// local-expansion adjoints locb of its partners.
cudaError_t launch_cross_cells_adjoint(const DevTree& t, const CrossCells& xc, const double* locb, double* mpb,
                                       int grid, cudaStream_t s);
// The per-slot sums the persistent kernel's cross items left in xcf, added to the targets.
cudaError_t launch_cross_apply(const DevTree& t, const CrossCells& xc, const double* xcf, double* loc,
                               cudaStream_t s);
cudaError_t launch_cross_cells(const DevTree& t, const CrossCells& xc, const double* mp, double* loc, int grid,
                               cudaStream_t s);

// ------------------------------------------------------------ adjoint (kernels_adjoint.cu)
struct BackwardArgs {
  const double* mp;   // forward multipoles
  const double* loc;  // forward local expansions (final, interior cells)
  double* mpb;        // [20][NC] multipole adjoints (workspace)
  double* locb;       // [23][NC] local-expansion adjoints (workspace)
  const double* phib;
  const double* gb;
  double* rhob;
  int64_t NL;
  const int* leaf_nodes;
  int n_leaf_nodes;
  const int* general_nodes;  // interior nodes and leaf nodes with a refined neighbour
  int n_general;
  const int* level_start;    // host array [max_level + 2]
  int max_level;
  Stencils st;
  CrossList xf, xl;          // general cross-level pairs (refined targets, leaf targets)
  CrossCells xc;             // tabulated cross-level pairs of leaf cells one level apart
  int xc_grid;
  int* err;                  // device word: bits of failed index checks (see kernels_adjoint.cu)
};
cudaError_t launch_backward(const DevTree& t, const BackwardArgs& ba, cudaStream_t s);
cudaError_t adjoint_local_bytes(size_t* out);

}  // namespace octo
