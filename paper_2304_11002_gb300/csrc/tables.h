// Host-side construction of the stencil tables that the interaction kernels read
// (plain C++: built with the host compiler too, so that the tables can be checked
// on a machine without a GPU).
#pragma once
#include <cstdint>
#include <vector>

namespace octo {

// Monopole kernel entry: kappa0 = -1/|d|, kappa1 = -d/|d|^3 (unit cell width).
struct alignas(16) Kappa {
  double v[4];
};

// The mixed path's leaf far-field tables are z-columns of a parity stencil (runs
// of entries d, d + 2 e_z, d + 4 e_z, ...: consecutive planes of one parity block
// of the halo) cut into chunks of 3, 2 or 1 entries.  A block of the table (one
// bulk asynchronous copy, kLeafTableBlockBytes) holds chunks of one length C only:
// kLeafBlock int32 chunk headers (halo offset of the chunk's first entry | C << 20;
// a header of 0 ends the block), then kLeafBlock float4 kernel rows, chunk c at
// rows C c .. C c + C - 1.  Blocks of C = 3 hold 10 chunks, C = 2 16, C = 1 32;
// a partial block is padded with chunks of halo offset 0 and zero rows.  A block is
// also one float32 partial sum.
constexpr int kLeafBlock = 32;
constexpr int kLeafTableBlockBytes = kLeafBlock * (4 + 16);

// Host: the stencil tab (n packed offsets; per_parity: [8][n], else one table for
// every parity class) grouped into aligned x-pairs of source cells for each parity
// class p: the entries dx, dx' with floor((p_x + dx) / 2) = floor((p_x + dx') / 2)
// and equal dy, dz form one pair, in the order of their first entry.  Returns the
// pairs per class (every class padded to the largest with entries of no cell).
int build_pair_tables(const int* tab, int n, bool per_parity, std::vector<int32_t>& out);

// Host: the per-(cell, neighbour slot) offset lists (ent, off: list i spans
// ent[off[i] .. off[i + 1]), i = l * 27 + o for local cell l) grouped into aligned
// x-pairs of source cells as in build_pair_tables, for the x-parity of cell l.
void build_cell_pair_lists(const std::vector<int32_t>& ent, const std::vector<int32_t>& off,
                           std::vector<int32_t>& pair_ent, std::vector<int32_t>& pair_off);

// Host: the mixed path's leaf far-field table blocks (see kLeafBlock) of the stencil
// tab (n packed offsets; per_parity: [8][n], else one table for every class) for a
// far halo of border R, kernel rows from kap (the dense table over [-R, R]^3),
// appended to out (32-bit words) as [8][blocks] blocks of kLeafTableBlockBytes;
// returns the blocks
// per parity class (every class padded to the most with empty blocks).
int build_leaf_column_blocks(const int* tab, int n, bool per_parity, int R, const Kappa* kap,
                             std::vector<uint32_t>& out);

}  // namespace octo
