// Host checks of the interaction kernels' stencil tables (csrc/tables.cpp) and of
// the leaf halo geometry (csrc/halo.h), built with the host compiler by
// tests/test_tables_host.py.  The stencils are generated here from the opening
// criterion (paper Section IV-C: well separated at the child level, near at the
// parent level), independently of the library's planner.  Prints one line per
// check and exits non-zero on the first failure.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <set>
#include <vector>

#include "halo.h"
#include "tables.h"

using namespace octo;

namespace {

int failures = 0;

void check(bool ok, const char* what, double theta) {
  if (!ok) {
    std::printf("FAIL %s (theta %.2f)\n", what, theta);
    ++failures;
  }
}

int32_t pack(int dx, int dy, int dz) {
  return (int32_t)(((uint32_t)(dx & 0xff)) | ((uint32_t)(dy & 0xff) << 8) | ((uint32_t)(dz & 0xff) << 16));
}

void unpack(int32_t e, int& dx, int& dy, int& dz) {
  dx = (int8_t)(e & 0xff), dy = (int8_t)((e >> 8) & 0xff), dz = (int8_t)((e >> 16) & 0xff);
}

int floor_div(int v, int k) { return v >= 0 ? v / k : -((-v + k - 1) / k); }

// theta |d| >= sqrt(3) in units of the cell width (equal cells of width 1)
bool well_separated(double theta, int dx, int dy, int dz) {
  return theta * theta * (double)(dx * dx + dy * dy + dz * dz) >= 3.0;
}

// Parity stencils: offsets d far at the child level whose parents are near.
std::vector<std::vector<int32_t>> parity_stencils(double theta) {
  std::vector<std::vector<int32_t>> st(8);
  for (int p = 0; p < 8; ++p) {
    const int pp[3] = {p & 1, (p >> 1) & 1, p >> 2};
    for (int dz = -9; dz <= 9; ++dz)
      for (int dy = -9; dy <= 9; ++dy)
        for (int dx = -9; dx <= 9; ++dx) {
          if (!well_separated(theta, dx, dy, dz)) continue;
          const int d[3] = {dx, dy, dz};
          int D[3];
          for (int a = 0; a < 3; ++a) D[a] = floor_div(pp[a] + d[a], 2);
          if (well_separated(theta, D[0], D[1], D[2])) continue;
          st[p].push_back(pack(dx, dy, dz));
        }
  }
  return st;
}

// The pairs of one class cover its stencil exactly once, start on an even source
// cell for targets of x-parity pa, and carry at least one cell unless padding.
bool pairs_cover(const int32_t* pairs, int n_pair, const std::vector<int32_t>& want, int pa, bool allow_pad) {
  std::multiset<int32_t> got;
  bool pad_seen = false;
  for (int s = 0; s < n_pair; ++s) {
    const int32_t e = pairs[s];
    int dx, dy, dz;
    unpack(e, dx, dy, dz);
    const int mask = (e >> 24) & 3;
    if ((e >> 26) != 0 || ((pa + dx) & 1) != 0) return false;
    if (mask == 0) {
      if (!allow_pad) return false;
      pad_seen = true;
      continue;
    }
    if (pad_seen) return false;  // padding only at the end
    if (mask & 1) got.insert(pack(dx, dy, dz));
    if (mask & 2) got.insert(pack(dx + 1, dy, dz));
  }
  return got == std::multiset<int32_t>(want.begin(), want.end());
}

}  // namespace

int main() {
  // ---- halo geometry: bijective, in bounds, and the lane patterns conflict-free
  for (int r = 3; r <= 8; ++r)
    for (int mixed = 0; mixed < 2; ++mixed) {
      const items::HaloGeom g = items::far_geom(r, mixed != 0);
      const int H = 8 + 2 * r;
      std::set<int> seen;
      bool ok = true;
      for (int z = 0; z < H; ++z)
        for (int y = 0; y < H; ++y)
          for (int x = 0; x < H; ++x) {
            const int i = items::halo_index(g, x, y, z);
            ok = ok && i >= 0 && i < 8 * g.PQ && seen.insert(i).second;
          }
      check(ok, "halo index is a bijection into 8 parity blocks", r);
      std::set<int> banks;
      if (mixed) {  // 32 float32 loads: lane (i, j, kh) at i + PY j + PZ 2 kh
        for (int lane = 0; lane < 32; ++lane)
          banks.insert(((lane & 3) + g.PY * ((lane >> 2) & 3) + g.PZ * 2 * (lane >> 4)) % 32);
        check(banks.size() == 32, "mixed far halo: 32 distinct banks", r);
      } else {  // each half-warp's 16 float64 loads: lane (i, j, k) at i + PY j + PZ k
        for (int half = 0; half < 2; ++half) {
          banks.clear();
          for (int l = 0; l < 16; ++l) {
            const int lane = 16 * half + l;
            banks.insert(((lane & 3) + g.PY * ((lane >> 2) & 3) + g.PZ * (lane >> 4)) % 16);
          }
          check(banks.size() == 16, "float64 far halo: 16 distinct bank pairs per half-warp", r);
        }
      }
    }

  for (double theta : {0.5, 0.45, 1.0}) {
    const auto st = parity_stencils(theta);
    const int n = (int)st[0].size();
    std::vector<int32_t> flat;
    for (int p = 0; p < 8; ++p) {
      check((int)st[p].size() == n, "parity stencils of equal size", theta);
      flat.insert(flat.end(), st[p].begin(), st[p].end());
    }
    std::vector<int32_t> root;
    for (int dz = -7; dz <= 7; ++dz)
      for (int dy = -7; dy <= 7; ++dy)
        for (int dx = -7; dx <= 7; ++dx)
          if (well_separated(theta, dx, dy, dz)) root.push_back(pack(dx, dy, dz));

    // ---- x-pair tables
    std::vector<int32_t> pairs, root_pairs;
    const int np = build_pair_tables(flat.data(), n, true, pairs);
    const int npr = build_pair_tables(root.data(), (int)root.size(), false, root_pairs);
    check((int)pairs.size() == 8 * np && (int)root_pairs.size() == 8 * npr, "pair table sizes", theta);
    for (int p = 0; p < 8; ++p) {
      check(pairs_cover(pairs.data() + p * np, np, st[p], p & 1, true), "parity pairs cover the stencil once", theta);
      check(pairs_cover(root_pairs.data() + p * npr, npr, root, p & 1, true), "level-0 pairs cover its stencil once",
            theta);
    }
    check(2 * np >= n && np < n, "pairs halve the stencil", theta);

    // ---- per-cell lists by neighbour slot, and their x-pairs
    std::vector<int32_t> ent, off(1, 0);
    for (int l = 0; l < 512; ++l) {
      const int c[3] = {l & 7, (l >> 3) & 7, l >> 6};
      const int p = (c[0] & 1) + 2 * (c[1] & 1) + 4 * (c[2] & 1);
      for (int o = 0; o < 27; ++o) {
        for (int32_t e : st[p]) {
          int d[3];
          unpack(e, d[0], d[1], d[2]);
          const int so = (floor_div(c[0] + d[0], 8) + 1) + 3 * (floor_div(c[1] + d[1], 8) + 1) +
                         9 * (floor_div(c[2] + d[2], 8) + 1);
          if (so == o) ent.push_back(e);
        }
        off.push_back((int32_t)ent.size());
      }
    }
    std::vector<int32_t> pent, poff;
    build_cell_pair_lists(ent, off, pent, poff);
    bool lists_ok = poff.size() == off.size();
    for (size_t i = 0; lists_ok && i + 1 < off.size(); ++i) {
      const int l = (int)(i / 27), o = (int)(i % 27);
      const int a = l & 7, b = (l >> 3) & 7, c = l >> 6;
      std::vector<int32_t> want(ent.begin() + off[i], ent.begin() + off[i + 1]);
      lists_ok = pairs_cover(pent.data() + poff[i], poff[i + 1] - poff[i], want, a & 1, false);
      for (int k = poff[i]; lists_ok && k < poff[i + 1]; ++k) {  // both cells in slot o
        int dx, dy, dz;
        unpack(pent[k], dx, dy, dz);
        for (int h = 0; h < 2; ++h)
          if ((pent[k] >> (24 + h)) & 1)
            lists_ok = lists_ok && (floor_div(a + dx + h, 8) + 1) + 3 * (floor_div(b + dy, 8) + 1) +
                                           9 * (floor_div(c + dz, 8) + 1) == o;
      }
    }
    check(lists_ok, "per-cell pair lists cover each list once, both cells in its slot", theta);

    // ---- leaf far-field chunk blocks: decode (halo offset, kernel row) per entry
    int R = 7;
    for (int32_t e : flat) {
      int d[3];
      unpack(e, d[0], d[1], d[2]);
      for (int a = 0; a < 3; ++a) R = std::max(R, std::abs(d[a]));
    }
    const int W = 2 * R + 1, kbase = R + W * R + W * W * R;
    std::vector<Kappa> kap((size_t)W * W * W);
    for (size_t i = 0; i < kap.size(); ++i)  // tagged rows, never zero: row i -> 4 i + 4
      for (int c = 0; c < 4; ++c) kap[i].v[c] = 4.0 * (double)i + 4.0 + c;
    for (int which = 0; which < 2; ++which) {
      const bool par = which == 0;
      const int nt = par ? n : (int)root.size();
      std::vector<uint32_t> words;
      const int nb = build_leaf_column_blocks(par ? flat.data() : root.data(), nt, par, R, kap.data(), words);
      const int kWords = kLeafTableBlockBytes / 4;
      check((int)words.size() == 8 * nb * kWords, "chunk block sizes", theta);
      const items::HaloGeom g = items::far_geom(R, true);
      bool ok = true;
      for (int p = 0; p < 8 && ok; ++p) {
        const int pa = p & 1, pb = (p >> 1) & 1, pc = p >> 2;
        std::multiset<std::pair<int, int>> want, got;
        for (int32_t e : (par ? st[p] : root)) {
          int dx, dy, dz;
          unpack(e, dx, dy, dz);
          want.insert({items::halo_index(g, pa + R + dx, pb + R + dy, pc + R + dz), kbase + dx + W * dy + W * W * dz});
        }
        for (int b = 0; b < nb && ok; ++b) {
          const unsigned char* base = reinterpret_cast<const unsigned char*>(&words[((size_t)p * nb + b) * kWords]);
          int h0;
          std::memcpy(&h0, base, 4);
          const int C = h0 >> 20, N = C == 3 ? 10 : C == 2 ? 16 : C == 1 ? 32 : 0;
          if (C == 0) continue;  // an empty block ends the class
          for (int ci = 0; ci < N && ok; ++ci) {
            int h;
            std::memcpy(&h, base + 4 * ci, 4);
            ok = (h >> 20) == C;  // one chunk length per block
            for (int u = 0; u < C && ok; ++u) {
              float k4[4];
              std::memcpy(k4, base + 4 * kLeafBlock + 16 * (C * ci + u), 16);
              if (k4[0] == 0.0f) {  // padding: a zero row
                ok = k4[1] == 0.0f && k4[2] == 0.0f && k4[3] == 0.0f;
                continue;
              }
              const int row = (int)std::lround((k4[0] - 4.0f) / 4.0f);
              ok = k4[1] == k4[0] + 1.0f;
              // entry u of a chunk is u planes further along z in the same parity block
              got.insert({(h & 0xfffff) + u * g.PZ, row});
            }
          }
        }
        ok = ok && got == want;
      }
      check(ok, par ? "parity chunk blocks reproduce the stencil's halo offsets and kernel rows"
                    : "level-0 chunk blocks reproduce the stencil's halo offsets and kernel rows",
            theta);
    }
    std::printf("theta %.2f: %d entries, %d pairs, %zu cell-list entries in %zu pairs\n", theta, n, np, ent.size(),
                pent.size());
  }
  std::printf(failures ? "FAILED %d\n" : "ok\n", failures);
  return failures ? 1 : 0;
}
