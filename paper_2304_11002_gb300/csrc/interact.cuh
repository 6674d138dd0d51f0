// Kernels of the interaction phase as templates over the precision and, in mixed
// precision, the shape of the interior items (BLK: stencil entries per float32
// partial sum; SPLIT: half-node or quarter-node items).  Every shape is its own
// kernel: chosen at run time inside one kernel, the shapes made the 80-register
// variants spill.  Each translation unit instantiates the shapes it launches:
// kernels_interact.cu the float64 kernels and BLK = 32, kernels_interact_b64.cu
// BLK = 64 (compiled in parallel).
#pragma once
#include <algorithm>

#include "cross.cuh"
#include "items.cuh"

namespace octo {
namespace {

// C64 (mixed precision only): the float64-correction variant of the items.  The
// paired float32 items hold two source records (40 registers) and fit 128
// registers, two blocks per SM, without spilling.
template <bool MIXED, bool C64, int BLK, int SPLIT>
__global__ void __launch_bounds__(items::kThreads, MIXED && !C64 ? 2 : 1)
    k_interior_items(DevTree t, const int* __restrict__ nodes, Stencils st, const double* __restrict__ mp,
                     const float* __restrict__ mp32, double* __restrict__ loc) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int parts = MIXED ? 2 * SPLIT : 2;  // items per node
  const int node = nodes[blockIdx.x / parts];
  if constexpr (MIXED)
    if constexpr (C64)
      items::interior_f32<true, BLK, SPLIT>(t, node, blockIdx.x % parts, st, mp32, loc, smem, mp);
    else
      items::interior_f32x2<BLK, SPLIT>(t, node, blockIdx.x % parts, st, mp32, loc, smem);
  else
    items::interior_f64(t, node, blockIdx.x & 1, st, mp, loc);
}

// item = (node << 4) | (kind << 2) | part; kind 0 = interior (part: one half of the
// node, or in mixed precision with SPLIT 2 one quarter), 1 = leaf (the whole node),
// 2 = near field of a leaf node (mixed precision only), 3 = kCrossSlicesPerItem
// slices of the tabulated cross-level pairs starting at slice node *
// kCrossSlicesPerItem (sums per slot into xcf; k_cross_apply adds them to the
// targets after the launch, so that no item writes what another one reads)
//
// Paced mode (n32 >= 0, mixed precision): the queue holds the float32-bound items
// (interior, leaf far field) in [0, n32) and the float64-bound ones (cross, near)
// in [n32, n_items), each claimed from its own counter (counter[0], counter[1]);
// counter[2 + smid] flags an SM on which a block holds a float64 item.  A block
// takes a float64 item only if it can set its SM's flag (so at most one of an
// SM's blocks keeps the float64 pipe busy while the others run float32 items),
// and float32 items otherwise; once the float32 items are gone it takes the
// remaining float64 items regardless.  Nothing waits: a block that cannot set the
// flag takes other work.  Otherwise (n32 < 0) one counter over the merged queue.
template <bool MIXED, int MINB, int BLK, int SPLIT>
__global__ void __launch_bounds__(items::kThreads, MINB)
    k_persistent(DevTree t, const int* __restrict__ queue, int n_items, int n32, int* __restrict__ counter,
                 Stencils st, const double* __restrict__ mp, const float* __restrict__ mp32, double* __restrict__ loc,
                 double* __restrict__ nearf, int64_t NL, CrossCells xc, double* __restrict__ xcf) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int next;
  bool holding = false, done32 = false, done64 = false;  // thread 0's state in paced mode
  unsigned smid = 0;
  if (n32 >= 0) asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  int* flag = counter + 2 + (smid < kPaceFlags ? smid : 0);
  const bool pace = n32 >= 0 && smid < kPaceFlags;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      if (n32 < 0) {
        const int k = atomicAdd(counter, 1);
        next = k < n_items ? queue[k] : -1;
      } else {
        const int n64 = n_items - n32;
        if (holding) {
          atomicExch(flag, 0);
          holding = false;
        }
        int item = -1;
        if (pace && !done64 && atomicCAS(flag, 0, 1) == 0) {
          const int k = atomicAdd(counter + 1, 1);
          if (k < n64) {
            item = queue[n32 + k];
            holding = true;
          } else {
            atomicExch(flag, 0);
            done64 = true;
          }
        }
        if (item < 0 && !done32) {
          const int k = atomicAdd(counter, 1);
          if (k < n32)
            item = queue[k];
          else
            done32 = true;
        }
        if (item < 0 && !done64) {  // no float32 item left: the float64 items regardless
          const int k = atomicAdd(counter + 1, 1);
          if (k < n64)
            item = queue[n32 + k];
          else
            done64 = true;
        }
        next = item;
      }
    }
    __syncthreads();
    const int it = next;
    if (it < 0) return;
    const int node = it >> 4, part = it & 3, kind = (it >> 2) & 3;
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
      if constexpr (MIXED)
        items::interior_f32x2<BLK, SPLIT>(t, node, SPLIT == 2 ? part : (part & 1), st, mp32, loc, smem);
      else
        items::interior_f64(t, node, part & 1, st, mp, loc);
    }
  }
}

// Dynamic shared memory of the persistent kernel: the largest of its item kinds
// (float64 interior items use none; cross items hold the cross kernel table).
inline size_t persistent_smem_bytes(const Stencils& st, const CrossCells& xc, bool mixed) {
  const size_t leaf = items::leaf_smem_bytes(st, mixed), cross = sizeof(double) * 4 * (size_t)xc.n_rows;
  return std::max(cross, mixed ? std::max({leaf, items::near_smem_bytes(st), items::interior_smem_bytes()}) : leaf);
}

// Resident blocks per SM of a persistent variant (sets its shared-memory limit);
// called once per handle, outside any stream capture.
template <bool MIXED, int MINB, int BLK, int SPLIT>
cudaError_t persistent_occupancy(const Stencils& st, const CrossCells& xc, int* per_sm) {
  const size_t smem = persistent_smem_bytes(st, xc, MIXED);
  auto* k = k_persistent<MIXED, MINB, BLK, SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, items::kThreads, smem);
  if (e == cudaSuccess && *per_sm < 1) e = cudaErrorInvalidConfiguration;
  return e;
}

template <bool MIXED, int MINB, int BLK, int SPLIT>
cudaError_t persistent_launch(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
  const size_t smem = persistent_smem_bytes(a.st, a.xc, MIXED);
  const int n32 = MIXED ? a.n32 : -1;
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(int) * (n32 >= 0 ? 2 + kPaceFlags : 1), s);
  if (e != cudaSuccess) return e;
  k_persistent<MIXED, MINB, BLK, SPLIT><<<a.grid, items::kThreads, smem, s>>>(
      t, a.queue, a.n_items, n32, a.counter, a.st, a.mp, a.mp32, a.loc, a.nearf, a.NL, a.xc, a.xcf);
  return cudaGetLastError();
}

// The mixed-precision shape set of one BLK: per-kind interior launch, persistent
// launch and occupancy for every (register budget, split).
template <int BLK>
struct MixedShapes {
  static cudaError_t interior(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
    const size_t smem = items::interior_smem_bytes();
    if (a.st.interior_split == 2)
      k_interior_items<true, false, BLK, 2><<<4 * a.n_interior, items::kThreads, smem, s>>>(t, a.interior, a.st, a.mp,
                                                                                           a.mp32, a.loc);
    else
      k_interior_items<true, false, BLK, 1><<<2 * a.n_interior, items::kThreads, smem, s>>>(t, a.interior, a.st, a.mp,
                                                                                           a.mp32, a.loc);
    return cudaGetLastError();
  }
  static cudaError_t persistent(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
    const bool q = a.st.interior_split == 2;
    switch (a.min_blocks) {
      case 1: return q ? persistent_launch<true, 1, BLK, 2>(t, a, s) : persistent_launch<true, 1, BLK, 1>(t, a, s);
      case 2: return q ? persistent_launch<true, 2, BLK, 2>(t, a, s) : persistent_launch<true, 2, BLK, 1>(t, a, s);
      case 3: return q ? persistent_launch<true, 3, BLK, 2>(t, a, s) : persistent_launch<true, 3, BLK, 1>(t, a, s);
    }
    return cudaErrorInvalidValue;
  }
  // Fewest resident blocks per SM over both splits (sets every variant's limit).
  static cudaError_t occupancy(int min_blocks, const Stencils& st, const CrossCells& xc, int* per_sm) {
    int a = 0, b = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (min_blocks) {
      case 1:
        e = persistent_occupancy<true, 1, BLK, 1>(st, xc, &a);
        if (e == cudaSuccess) e = persistent_occupancy<true, 1, BLK, 2>(st, xc, &b);
        break;
      case 2:
        e = persistent_occupancy<true, 2, BLK, 1>(st, xc, &a);
        if (e == cudaSuccess) e = persistent_occupancy<true, 2, BLK, 2>(st, xc, &b);
        break;
      case 3:
        e = persistent_occupancy<true, 3, BLK, 1>(st, xc, &a);
        if (e == cudaSuccess) e = persistent_occupancy<true, 3, BLK, 2>(st, xc, &b);
        break;
    }
    *per_sm = std::min(a, b);
    return e;
  }
};

}  // namespace

// Entry points of the BLK = 64 shape set (kernels_interact_b64.cu).
cudaError_t interior_items_b64(const DevTree& t, const InteractArgs& a, cudaStream_t s);
cudaError_t persistent_b64(const DevTree& t, const InteractArgs& a, cudaStream_t s);
cudaError_t persistent_occupancy_b64(int min_blocks, const Stencils& st, const CrossCells& xc, int* per_sm);

}  // namespace octo
