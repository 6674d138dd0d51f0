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
