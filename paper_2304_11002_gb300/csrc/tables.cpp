// Host-side stencil tables of the interaction kernels (see tables.h).
#include "tables.h"

#include <algorithm>
#include <cstring>
#include <set>
#include <utility>

#include "halo.h"

namespace octo {

namespace {

// The entries tp[0 .. n) for targets of x-parity pa grouped into aligned x-pairs of
// source cells, appended to out in the order of their first entry.
void group_pairs(const int* tp, int n, int pa, std::vector<int32_t>& out) {
  std::vector<std::pair<int32_t, size_t>> key_slot;  // (pair index X, dy, dz) -> slot
  for (int s = 0; s < n; ++s) {
    const int e = tp[s];
    const int dx = (int)(int8_t)(e & 0xff), dy = (int)(int8_t)((e >> 8) & 0xff), dz = (int)(int8_t)((e >> 16) & 0xff);
    const int v = pa + dx, X = v >= 0 ? v / 2 : -((1 - v) / 2), bit = v - 2 * X;  // X = floor(v / 2)
    const int32_t key = (int32_t)(((uint32_t)(X & 0xff)) | ((uint32_t)(dy & 0xff) << 8) | ((uint32_t)(dz & 0xff) << 16));
    size_t slot = out.size();
    for (const auto& ks : key_slot)
      if (ks.first == key) slot = ks.second;
    if (slot == out.size()) {
      key_slot.push_back({key, slot});
      const int dx0 = 2 * X - pa;  // a + dx0 is even for targets of x-parity pa
      out.push_back((int32_t)(((uint32_t)(dx0 & 0xff)) | ((uint32_t)(dy & 0xff) << 8) | ((uint32_t)(dz & 0xff) << 16)));
    }
    out[slot] |= (int32_t)(1u << (24 + bit));
  }
}

}  // namespace

int build_pair_tables(const int* tab, int n, bool per_parity, std::vector<int32_t>& out) {
  std::vector<std::vector<int32_t>> per(8);
  size_t n_pair = 0;
  for (int p = 0; p < 8; ++p) {
    group_pairs(per_parity ? tab + (size_t)p * n : tab, n, p & 1, per[p]);
    n_pair = std::max(n_pair, per[p].size());
  }
  out.assign(8 * n_pair, 0);
  for (int p = 0; p < 8; ++p)
    for (size_t s = 0; s < n_pair; ++s)  // padding: the first pair's offset with no cell
      out[p * n_pair + s] = s < per[p].size() ? per[p][s] : (per[p][0] & 0xffffff);
  return (int)n_pair;
}

void build_cell_pair_lists(const std::vector<int32_t>& ent, const std::vector<int32_t>& off,
                           std::vector<int32_t>& pair_ent, std::vector<int32_t>& pair_off) {
  pair_ent.clear();
  pair_off.assign(1, 0);
  for (size_t i = 0; i + 1 < off.size(); ++i) {
    const int l = (int)(i / 27);
    group_pairs(ent.data() + off[i], off[i + 1] - off[i], (l & 7) & 1, pair_ent);
    pair_off.push_back((int32_t)pair_ent.size());
  }
}

int build_leaf_column_blocks(const int* tab, int n, bool per_parity, int R, const Kappa* kap,
                             std::vector<uint32_t>& out) {
  const items::HaloGeom gf = items::far_geom(R, true);
  const int W = 2 * R + 1, kbase = R + W * R + W * W * R;
  struct Chunk {
    int off, dx, dy, dz;  // halo offset and stencil offset of the first entry
  };
  constexpr int kPerBlock[4] = {0, 32, 16, 10};  // chunks per block of chunk length C
  std::vector<std::vector<std::pair<int, std::vector<Chunk>>>> blocks(8);  // [p] -> (C, chunks)
  size_t nb = 0;
  for (int p = 0; p < 8; ++p) {
    const int pa = p & 1, pb = (p >> 1) & 1, pc = p >> 2;
    const int* tp = per_parity ? tab + (size_t)p * n : tab;
    std::set<int32_t> in(tp, tp + n);
    auto key = [](int dx, int dy, int dz) {
      return (int32_t)(((uint32_t)(dx & 0xff)) | ((uint32_t)(dy & 0xff) << 8) | ((uint32_t)(dz & 0xff) << 16));
    };
    std::vector<Chunk> by_len[4];
    for (int s = 0; s < n; ++s) {  // columns in the order of their first entry
      const int e = tp[s];
      const int dx = (int)(int8_t)(e & 0xff), dy = (int)(int8_t)((e >> 8) & 0xff), dz = (int)(int8_t)((e >> 16) & 0xff);
      if (in.count(key(dx, dy, dz - 2))) continue;  // not the first entry of its column
      int len = 0;
      while (in.count(key(dx, dy, dz + 2 * len))) ++len;
      // chunks of 3, then 2 + 2 for a remainder of 4 and 2 for a remainder of 2
      for (int w = 0; w < len;) {
        const int left = len - w, c = left == 1 ? 1 : left == 2 || left == 4 ? 2 : 3;
        by_len[c].push_back({items::halo_index(gf, pa + R + dx, pb + R + dy, pc + R + dz + 2 * w), dx, dy, dz + 2 * w});
        w += c;
      }
    }
    for (int c = 3; c >= 1; --c)
      for (size_t k = 0; k < by_len[c].size(); k += kPerBlock[c])
        blocks[p].push_back({c, std::vector<Chunk>(by_len[c].begin() + k,
                                                   by_len[c].begin() + std::min(by_len[c].size(), k + kPerBlock[c]))});
    nb = std::max(nb, blocks[p].size());
  }
  constexpr int kWords = kLeafTableBlockBytes / 4;
  const size_t b0 = out.size();
  out.resize(b0 + (size_t)8 * nb * kWords, 0u);
  for (int p = 0; p < 8; ++p)
    for (size_t bk = 0; bk < blocks[p].size(); ++bk) {
      unsigned char* base = reinterpret_cast<unsigned char*>(&out[b0 + ((size_t)p * nb + bk) * kWords]);
      const int C = blocks[p][bk].first;
      const std::vector<Chunk>& ch = blocks[p][bk].second;
      for (int ci = 0; ci < kPerBlock[C]; ++ci) {  // padding chunks: offset 0, zero rows
        const int32_t h = (ci < (int)ch.size() ? ch[ci].off : 0) | (C << 20);
        std::memcpy(base + 4 * ci, &h, 4);
        if (ci >= (int)ch.size()) continue;
        for (int w = 0; w < C; ++w) {
          const Kappa& v = kap[kbase + ch[ci].dx + W * ch[ci].dy + W * W * (ch[ci].dz + 2 * w)];
          const float k4[4] = {(float)v.v[0], (float)v.v[1], (float)v.v[2], (float)v.v[3]};
          std::memcpy(base + 4 * kLeafBlock + 16 * (C * ci + w), k4, 16);
        }
      }
    }
  return (int)nb;
}

}  // namespace octo
