// Host-side planning of the FMM solve: tree validation, device node order,
// same-level neighbour tables, per-parity interaction stencils, cross-level pair
// lists and interaction counts.  Pure C++ (no CUDA calls), so it also runs on a
// machine without a GPU.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/octo_fmm.h"

namespace octo {

constexpr int kCells = 512;  // 8^3 cells per node
constexpr int kMaxLevel = 14;

// One stencil entry: a same-level cell offset d (|d_i| <= 7) packed as bytes.
inline int32_t pack_offset(int dx, int dy, int dz) {
  return (int32_t)((uint32_t)(uint8_t)(int8_t)dx | ((uint32_t)(uint8_t)(int8_t)dy << 8) |
                   ((uint32_t)(uint8_t)(int8_t)dz << 16));
}

struct Plan {
  // ---- tree in device order (sorted by level, then descriptor order) ----
  int n_nodes = 0, max_level = 0, n_leaf = 0;
  std::vector<int32_t> dnode_of_desc;  // descriptor node -> device node
  std::vector<int32_t> desc_of_dnode;
  std::vector<int32_t> level, ijk;     // [n], [n*3] in device order
  std::vector<int32_t> parent, octant; // parent device node, octant in parent
  std::vector<int32_t> children;       // [n*8] device nodes, -1 for leaves
  std::vector<int32_t> leaf_id;        // leaf order index (rho/phi/g), -1 for interior
  std::vector<int32_t> nbr;            // [n*27] same-level neighbour device node or -1
  std::vector<int32_t> level_start;    // [max_level+2] device-node range per level
  double origin[3] = {0, 0, 0}, extent = 1.0;
  double theta = 0.5;

  // ---- stencils (same-level offsets) ----
  // Level >= 1: 8 parity classes (p = px + 2 py + 4 pz), far offsets whose parent
  // offset is not far.  Level 0: all far offsets inside [-7, 7]^3.  Near: all
  // non-zero offsets that are not far (leaf-level P2P).
  std::vector<int32_t> st_parity;  // [8 * n_st]
  int n_st = 0;
  std::vector<int32_t> st_root;
  std::vector<int32_t> st_near;
  // Per (target cell local index l, neighbour slot o): the parity-stencil offsets
  // of cell l whose source lands in slot o; list l * 27 + o spans
  // cell_ent[cell_ent_off[i] .. cell_ent_off[i+1]).
  std::vector<int32_t> cell_ent;
  std::vector<int32_t> cell_ent_off;
  // Leaf nodes with refined same-level neighbours: per node, the 256 cells of each
  // half (even / odd z) ordered by decreasing number of pairs with those
  // neighbours, so that the lanes of a warp get similar trip counts.
  std::vector<uint16_t> bnd_perm;   // [n_boundary][512] local cells by decreasing boundary load
  std::vector<int32_t> bnd_index;   // per device node: row of bnd_perm, or -1

  // ---- work lists ----
  std::vector<int32_t> interior_nodes;   // refined device nodes (all levels)
  std::vector<int32_t> leaf_nodes;       // leaf device nodes (all levels)
  std::vector<int32_t> boundary_nodes;   // leaf device nodes with a refined same-level neighbour
  // cross-level pairs, CSR by target cell (global cell index = dnode*512 + local)
  std::vector<int64_t> x_targets;        // distinct target cells
  std::vector<int64_t> x_start;          // [n_targets+1]
  std::vector<int64_t> x_mid;            // [n_targets]: first P2P entry (M2L entries come first)
  std::vector<int64_t> x_sources;        // source cell per entry

  // The cross-level pairs split for the forward solve.  Pairs of two leaf cells one
  // level apart are exact point-mass terms between cell centres whose offset, in
  // units of half the finer cell width, has odd integer components v; they go to a
  // tabulated list in SELL-32 layout: targets sorted by decreasing partner count,
  // 32 targets per slice (padding targets are -1), the entries of a slice stored
  // interleaved (entry k of lane j at xc_slice_off[s] + 32 k + j; slice widths are
  // multiples of 4, padded with the zero table row).  Entry = source cell << 20 |
  // sign bits of v << 16 | table row.  Every other pair stays in the general CSR
  // lists xg_* (same layout as x_*).
  std::vector<int64_t> xc_targets;       // [32 * n_slices]
  std::vector<int64_t> xc_slice_off;     // [n_slices + 1]
  std::vector<int64_t> xc_entries;
  // Table rows (4 doubles each): row g * na^3 + (ax * na + ay) * na + az, with
  // a = (|v| - 1) / 2 per axis and g = 0 when the source is the finer cell (v in
  // units of h_t / 4), g = 1 when it is the coarser one (units of h_t / 2); row
  // 2 na^3 is zero.  Row = (s / |v|, s^2 |v_x| / |v|^3, s^2 |v_y| / |v|^3,
  // s^2 |v_z| / |v|^3) with s = 4 or 2 (the target cell width in those units).
  std::vector<double> xc_table;
  int xc_na = 0;
  int64_t xc_pairs = 0;
  std::vector<int64_t> xg_targets, xg_start, xg_mid, xg_sources;

  // ordered interaction counts: same-level M2L, cross-level M2L, same-level P2P, cross-level P2P
  int64_t counts[4] = {0, 0, 0, 0};
  // same-level pairs per kernel: [0] M2L into interior cells, [1] leaf-leaf M2L,
  // [2] leaf-leaf P2P, [3] M2L from refined neighbours into leaf cells
  int64_t kernel_pairs[4] = {0, 0, 0, 0};

  std::string error;
};

// Builds everything above.  Returns OCTO_OK or a negative status (message in plan.error).
int build_plan(const octo_tree_desc* desc, double theta, Plan& plan);

double cell_width(const Plan& p, int level);

// Message returned by octo_fmm_last_error(NULL) (failures without a handle).
void set_global_error(const std::string& msg);

}  // namespace octo
