// Host program (no GPU): checks the float32 record layout of the mixed far field
// (mp32_index / mp32_pair_base, device.cuh).  Every (cell, field) of a node has its
// own float inside the node's 20 x 512 floats; the two cells of an x-pair hold each
// field in adjacent floats of one 16-byte plane word (lane 0 the even cell), fields
// 2k and 2k + 1 in the same word; and for every stencil offset that keeps the
// sources inside one node, the 32 lanes of a parity-class warp read 32 consecutive
// 16-byte words of each plane.  Prints "ok" or the first failure.
#include <cstdio>
#include <set>

#include "device.cuh"

using namespace octo;

int main() {
  for (int node : {0, 1, 7}) {
    std::set<long long> seen;
    for (int c = 0; c < 8; ++c)
      for (int b = 0; b < 8; ++b)
        for (int a = 0; a < 8; ++a)
          for (int f = 0; f < N_MP; ++f) {
            const long long i = mp32_index(node, a, b, c, f);
            if (i < (long long)node * N_MP * 512 || i >= (long long)(node + 1) * N_MP * 512 || !seen.insert(i).second) {
              std::printf("FAIL bijection node %d cell %d %d %d field %d\n", node, a, b, c, f);
              return 1;
            }
            const long long word = mp32_pair_base(node, a >> 1, b, c) + (long long)(f >> 1) * kMp32Pairs;
            if (i != 4 * word + 2 * (f & 1) + (a & 1)) {
              std::printf("FAIL pair word node %d cell %d %d %d field %d\n", node, a, b, c, f);
              return 1;
            }
          }
  }
  // a parity-class warp: lanes (i, j, k) = (lane & 3, (lane >> 2) & 3, lane >> 4) hold
  // targets (2i + pa, 2j + pb, 2(2zh + k) + pc); an even source start dx0 per entry
  for (int p = 0; p < 8; ++p)
    for (int zh = 0; zh < 2; ++zh)
      for (int dz = -8; dz <= 8; ++dz)
        for (int dy = -8; dy <= 8; ++dy)
          for (int dx = -9; dx <= 8; ++dx) {
            const int pa = p & 1, pb = (p >> 1) & 1, pc = p >> 2;
            if (((pa + dx) & 1) != 0) continue;  // pair entries start on an even source cell
            long long first = 0;
            bool inside = true, consecutive = true;
            for (int lane = 0; lane < 32 && inside; ++lane) {
              const int a = 2 * (lane & 3) + pa + dx, b = 2 * ((lane >> 2) & 3) + pb + dy,
                        c = 2 * (2 * zh + (lane >> 4)) + pc + dz;
              if (a < 0 || a > 7 || b < 0 || b > 7 || c < 0 || c > 7) inside = false;
              if (!inside) break;
              const long long w = mp32_pair_base(0, a >> 1, b, c);
              if (lane == 0) first = w;
              consecutive = consecutive && w == first + lane;
            }
            if (inside && !consecutive) {
              std::printf("FAIL coalescing parity %d zh %d offset %d %d %d\n", p, zh, dx, dy, dz);
              return 1;
            }
          }
  std::printf("ok\n");
  return 0;
}
