// The same-level interaction phase as batched launches.
//
//  * per-kind launches: one grid over all interior items of every level, one grid
//    over all leaf items;
//  * persistent queue: one grid of (SMs x blocks per SM) blocks that pull items of
//    every kind (interior, leaf far field, leaf near field, tabulated cross-level
//    slices), of every level, from a single atomic counter, so that float32-heavy
//    and float64-heavy items share the SMs and the tail of one kind overlaps the
//    others.  The counter is reset by a memset issued before every launch; no block
//    ever waits for another.
// The autotuner in capi.cu times both on the actual tree and keeps the faster.
#include <cstring>
#include <set>

#include "interact.cuh"

namespace octo {

namespace {

// The mixed path's paired boundary pairs fit 128 registers (two blocks per SM)
// without spilling.
template <bool MIXED, bool C64 = false>
__global__ void __launch_bounds__(items::kThreads, MIXED && !C64 ? 2 : 1)
    k_leaf_items(DevTree t, const int* __restrict__ nodes, Stencils st, const double* __restrict__ mp,
                 const float* __restrict__ mp32, double* __restrict__ loc) {
  extern __shared__ __align__(16) unsigned char smem[];
  items::leaf_item<MIXED, C64>(t, nodes[blockIdx.x], st, mp, mp32, loc, smem);
}

__global__ void __launch_bounds__(items::kThreads) k_near_items(DevTree t, const int* __restrict__ nodes, Stencils st,
                                                                 const double* __restrict__ mp,
                                                                 double* __restrict__ nearf, int64_t NL) {
  extern __shared__ __align__(16) unsigned char smem[];
  items::near_item(t, nodes[blockIdx.x], st, mp, nearf, NL, smem);
}

}  // namespace

void build_leaf_tables(const int* parity, int n_st, const int* root, int n_root, const int* near_, int n_near, int R,
                       int RN, bool mixed, int2* far_out, int2* root_out, int2* near_out) {
  const items::HaloGeom gf = items::far_geom(R, false), gn = mixed ? items::near_geom(RN) : items::far_geom(R, false);
  const int W = 2 * R + 1, kbase = R + W * R + W * W * R;
  // entry of offset d for targets of parity (pa, pb, pc) in a halo of border g.r
  auto entry = [&](const items::HaloGeom& g, int pa, int pb, int pc, int e) {
    const int dx = (int)(int8_t)(e & 0xff), dy = (int)(int8_t)((e >> 8) & 0xff), dz = (int)(int8_t)((e >> 16) & 0xff);
    return make_int2(items::halo_index(g, pa + g.r + dx, pb + g.r + dy, pc + g.r + dz), kbase + dx + W * dy + W * W * dz);
  };
  for (int p = 0; p < 8; ++p) {
    const int pa = p & 1, pb = (p >> 1) & 1, pc = p >> 2;
    for (int s = 0; s < n_st; ++s) far_out[p * n_st + s] = entry(gf, pa, pb, pc, parity[p * n_st + s]);
    for (int s = 0; s < n_root; ++s) root_out[p * n_root + s] = entry(gf, pa, pb, pc, root[s]);
    for (int s = 0; s < n_near; ++s) near_out[p * n_near + s] = entry(gn, pa, pb, pc, near_[s]);
  }
}

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
                             std::vector<uint4>& out) {
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
  constexpr int kWords = kLeafTableBlockBytes / 16;
  const size_t b0 = out.size();
  out.resize(b0 + (size_t)8 * nb * kWords, make_uint4(0, 0, 0, 0));
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

cudaError_t configure_interact_kernels() {
  cudaError_t e = cudaSuccess;
  const int big = 200 * 1024;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_leaf_items<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_leaf_items<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_leaf_items<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  return e;
}

cudaError_t launch_interior_items(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
  if (a.n_interior == 0) return cudaSuccess;
  if (a.mixed && a.corr64) {
    k_interior_items<true, true, 32, 1><<<2 * a.n_interior, items::kThreads, items::interior_smem_bytes(), s>>>(
        t, a.interior, a.st, a.mp, a.mp32, a.loc);
    return cudaGetLastError();
  }
  if (a.mixed) return a.st.acc_block == 64 ? interior_items_b64(t, a, s) : MixedShapes<32>::interior(t, a, s);
  k_interior_items<false, false, 32, 1><<<2 * a.n_interior, items::kThreads, 0, s>>>(t, a.interior, a.st, a.mp,
                                                                                     a.mp32, a.loc);
  return cudaGetLastError();
}

cudaError_t launch_leaf_items(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
  if (a.n_leaf == 0) return cudaSuccess;
  const size_t smem = items::leaf_smem_bytes(a.st, a.mixed);
  if (a.mixed && a.corr64)
    k_leaf_items<true, true><<<a.n_leaf, items::kThreads, smem, s>>>(t, a.leaf, a.st, a.mp, a.mp32, a.loc);
  else if (a.mixed)
    k_leaf_items<true><<<a.n_leaf, items::kThreads, smem, s>>>(t, a.leaf, a.st, a.mp, a.mp32, a.loc);
  else
    k_leaf_items<false><<<a.n_leaf, items::kThreads, smem, s>>>(t, a.leaf, a.st, a.mp, a.mp32, a.loc);
  return cudaGetLastError();
}

cudaError_t launch_near_items(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
  if (a.n_leaf == 0) return cudaSuccess;
  k_near_items<<<a.n_leaf, items::kThreads, items::near_smem_bytes(a.st), s>>>(t, a.leaf, a.st, a.mp, a.nearf, a.NL);
  return cudaGetLastError();
}

// Register budgets: 1 or 2 resident blocks per SM, and 3 in mixed precision (whose
// items all fit 85 registers; the float64 interior item needs twice that).  Mixed
// precision: the fewest resident blocks over every interior shape of the budget
// (sets every variant's shared-memory limit).
cudaError_t persistent_blocks_per_sm(bool mixed, int min_blocks, const Stencils& st, const CrossCells& xc,
                                     int* per_sm) {
  if (mixed) {
    if (min_blocks < 1 || min_blocks > 3) return cudaErrorInvalidValue;
    int a = 0, b = 0;
    cudaError_t e = MixedShapes<32>::occupancy(min_blocks, st, xc, &a);
    if (e == cudaSuccess) e = persistent_occupancy_b64(min_blocks, st, xc, &b);
    *per_sm = std::min(a, b);
    return e;
  }
  if (min_blocks == 3) return cudaErrorInvalidValue;
  return min_blocks == 2 ? persistent_occupancy<false, 2, 32, 1>(st, xc, per_sm)
                         : persistent_occupancy<false, 1, 32, 1>(st, xc, per_sm);
}

cudaError_t launch_persistent(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
  if (a.n_items == 0) return cudaSuccess;
  if (a.grid < 1 || a.corr64) return cudaErrorInvalidConfiguration;  // float64 correction: per-kind launches only
  if (a.mixed) return a.st.acc_block == 64 ? persistent_b64(t, a, s) : MixedShapes<32>::persistent(t, a, s);
  if (a.min_blocks == 3) return cudaErrorInvalidValue;
  return a.min_blocks == 2 ? persistent_launch<false, 2, 32, 1>(t, a, s) : persistent_launch<false, 1, 32, 1>(t, a, s);
}

}  // namespace octo
