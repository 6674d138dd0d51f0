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
#include <algorithm>

#include "cross.cuh"
#include "items.cuh"

namespace octo {

namespace {

template <bool MIXED>
__global__ void __launch_bounds__(items::kThreads, MIXED ? 3 : 1) k_interior_items(DevTree t, const int* __restrict__ nodes,
                                                                     Stencils st, const double* __restrict__ mp,
                                                                     const float* __restrict__ mp32,
                                                                     double* __restrict__ loc) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int node = nodes[blockIdx.x >> 1];
  if (MIXED)
    items::interior_f32(t, node, blockIdx.x & 1, st, mp32, loc, smem);
  else
    items::interior_f64(t, node, blockIdx.x & 1, st, mp, loc);
}

template <bool MIXED>
__global__ void __launch_bounds__(items::kThreads, MIXED ? 3 : 1) k_leaf_items(DevTree t, const int* __restrict__ nodes, Stencils st,
                                                                 const double* __restrict__ mp,
                                                                 const float* __restrict__ mp32,
                                                                 double* __restrict__ loc) {
  extern __shared__ __align__(16) unsigned char smem[];
  items::leaf_item<MIXED>(t, nodes[blockIdx.x], st, mp, mp32, loc, smem);
}

__global__ void __launch_bounds__(items::kThreads) k_near_items(DevTree t, const int* __restrict__ nodes, Stencils st,
                                                                 const double* __restrict__ mp,
                                                                 double* __restrict__ nearf, int64_t NL) {
  extern __shared__ __align__(16) unsigned char smem[];
  items::near_item(t, nodes[blockIdx.x], st, mp, nearf, NL, smem);
}

// item = (node << 3) | (kind << 1) | half; kind 0 = interior (one half of the node),
// 1 = leaf (the whole node), 2 = near field of a leaf node (mixed precision only),
// 3 = kCrossSlicesPerItem slices of the tabulated cross-level pairs starting at
// slice node * kCrossSlicesPerItem (sums per slot into xcf; k_cross_apply adds them
// to the targets after the launch, so that no item writes what another one reads)
template <bool MIXED, int MINB>
__global__ void __launch_bounds__(items::kThreads, MINB)
    k_persistent(DevTree t, const int* __restrict__ queue, int n_items, int* __restrict__ counter, Stencils st,
                 const double* __restrict__ mp, const float* __restrict__ mp32, double* __restrict__ loc,
                 double* __restrict__ nearf, int64_t NL, CrossCells xc, double* __restrict__ xcf) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int next;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    __syncthreads();
    const int k = next;
    if (k >= n_items) return;
    const int it = queue[k];
    const int node = it >> 3, half = it & 1, kind = (it >> 1) & 3;
    if (kind == 3) {
      double2* tab2 = reinterpret_cast<double2*>(smem);
      cross::stage_table(xc, tab2);
      __syncthreads();
      const int lane = threadIdx.x & 31;
      const int s1 = min((node + 1) * kCrossSlicesPerItem, xc.n_slices);
      const int64_t n_slots = (int64_t)xc.n_slices * 32;
      for (int sl = node * kCrossSlicesPerItem + (threadIdx.x >> 5); sl < s1; sl += items::kThreads / 32) {
        double S[4];
        cross::slice_sums(xc, tab2, mp, sl, lane, S);
        const int64_t slot = (int64_t)sl * 32 + lane;
        for (int k = 0; k < 4; ++k) xcf[k * n_slots + slot] = S[k];
      }
    } else if (kind == 2) {
      if (MIXED) items::near_item(t, node, st, mp, nearf, NL, smem);
    } else if (kind == 1) {
      items::leaf_item<MIXED>(t, node, st, mp, mp32, loc, smem);
    } else {
      if (MIXED)
        items::interior_f32(t, node, half, st, mp32, loc, smem);
      else
        items::interior_f64(t, node, half, st, mp, loc);
    }
  }
}

// Dynamic shared memory of the persistent kernel: the largest of its item kinds
// (float64 interior items use none; cross items hold the cross kernel table).
size_t persistent_smem_bytes(const Stencils& st, const CrossCells& xc, bool mixed) {
  const size_t leaf = items::leaf_smem_bytes(st, mixed), cross = sizeof(double) * 4 * (size_t)xc.n_rows;
  return std::max(cross, mixed ? std::max({leaf, items::near_smem_bytes(st), items::interior_smem_bytes()}) : leaf);
}

// Resident blocks per SM of a persistent variant (sets its shared-memory limit);
// called once per handle, outside any stream capture.
template <bool MIXED, int MINB>
cudaError_t persistent_occupancy(const Stencils& st, const CrossCells& xc, int* per_sm) {
  const size_t smem = persistent_smem_bytes(st, xc, MIXED);
  cudaError_t e = cudaFuncSetAttribute(k_persistent<MIXED, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_persistent<MIXED, MINB>, items::kThreads, smem);
  if (e == cudaSuccess && *per_sm < 1) e = cudaErrorInvalidConfiguration;
  return e;
}

template <bool MIXED, int MINB>
cudaError_t persistent_launch(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
  const size_t smem = persistent_smem_bytes(a.st, a.xc, MIXED);
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_persistent<MIXED, MINB><<<a.grid, items::kThreads, smem, s>>>(t, a.queue, a.n_items, a.counter, a.st, a.mp,
                                                                  a.mp32, a.loc, a.nearf, a.NL, a.xc, a.xcf);
  return cudaGetLastError();
}

}  // namespace

void build_leaf_tables(const int* parity, int n_st, const int* root, int n_root, const int* near_, int n_near, int R,
                       int RN, bool mixed, int2* far_out, int2* root_out, int2* near_out) {
  const items::HaloGeom gf = items::far_geom(R), gn = mixed ? items::near_geom(RN) : items::far_geom(R);
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
  return e;
}

cudaError_t launch_interior_items(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
  if (a.n_interior == 0) return cudaSuccess;
  if (a.mixed)
    k_interior_items<true><<<2 * a.n_interior, items::kThreads, items::interior_smem_bytes(), s>>>(
        t, a.interior, a.st, a.mp, a.mp32, a.loc);
  else
    k_interior_items<false><<<2 * a.n_interior, items::kThreads, 0, s>>>(t, a.interior, a.st, a.mp, a.mp32, a.loc);
  return cudaGetLastError();
}

cudaError_t launch_leaf_items(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
  if (a.n_leaf == 0) return cudaSuccess;
  const size_t smem = items::leaf_smem_bytes(a.st, a.mixed);
  if (a.mixed)
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
// items all fit 85 registers; the float64 interior item needs twice that).
cudaError_t persistent_blocks_per_sm(bool mixed, int min_blocks, const Stencils& st, const CrossCells& xc,
                                     int* per_sm) {
  if (mixed) {
    if (min_blocks == 3) return persistent_occupancy<true, 3>(st, xc, per_sm);
    return min_blocks == 2 ? persistent_occupancy<true, 2>(st, xc, per_sm)
                           : persistent_occupancy<true, 1>(st, xc, per_sm);
  }
  if (min_blocks == 3) return cudaErrorInvalidValue;
  return min_blocks == 2 ? persistent_occupancy<false, 2>(st, xc, per_sm) : persistent_occupancy<false, 1>(st, xc, per_sm);
}

cudaError_t launch_persistent(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
  if (a.n_items == 0) return cudaSuccess;
  if (a.grid < 1) return cudaErrorInvalidConfiguration;
  if (a.mixed) {
    if (a.min_blocks == 3) return persistent_launch<true, 3>(t, a, s);
    return a.min_blocks == 2 ? persistent_launch<true, 2>(t, a, s) : persistent_launch<true, 1>(t, a, s);
  }
  if (a.min_blocks == 3) return cudaErrorInvalidValue;
  return a.min_blocks == 2 ? persistent_launch<false, 2>(t, a, s) : persistent_launch<false, 1>(t, a, s);
}

}  // namespace octo
