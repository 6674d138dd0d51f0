// Launchers of the solver's kernels (host side).  Every launcher enqueues on
// `stream` and returns the cudaError_t of the launch.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"

namespace octo {

// Monopole kernel entry: kappa0 = -1/|d|, kappa1 = -d/|d|^3 (unit cell width).
struct alignas(16) Kappa {
  double v[4];
};

struct Stencils {
  const int* parity;  // [8][n_st] packed offsets
  int n_st;
  const int* root;    // level-0 far offsets
  int n_root;
  const int* near_;   // non-zero near offsets
  int n_near;
  const Kappa* kappa;    // dense monopole kernel table over [-R, R]^3, unit cell width
  const float4* kappa32; // the same table rounded to float32
  int radius;            // R: maximum |offset component|
  int near_radius;       // maximum |offset component| of the near offsets
};

struct CrossList {
  const int64_t* targets;
  const int64_t* start;
  const int64_t* sources;
  int n_targets;
};

// Once per process and device, before the first launch (opts into large shared memory).
cudaError_t configure_kernels();

// mp32 (may be null): float32 copy of the multipoles for the mixed-precision path.
cudaError_t launch_init_leaf(const DevTree& t, const int* leaf_nodes, int n_leaf_nodes, double* mp, float* mp32,
                             cudaStream_t s);
cudaError_t launch_p2m(const DevTree& t, const int* leaf_nodes, int n_leaf_nodes, const double* rho, double* mp,
                       float* mp32, cudaStream_t s);
cudaError_t launch_m2m(const DevTree& t, int node_begin, int node_end, double* mp, float* mp32, cudaStream_t s);
cudaError_t launch_m2l_interior(const DevTree& t, const int* nodes, int n_nodes, const Stencils& st,
                                const double* mp, double* loc, cudaStream_t s);
cudaError_t launch_m2l_boundary(const DevTree& t, const int* nodes, int n_nodes, const Stencils& st,
                                const double* mp, double* loc, cudaStream_t s);
cudaError_t launch_leaf_conv(const DevTree& t, const int* nodes, int n_nodes, const Stencils& st, const double* mp,
                             double* loc, cudaStream_t s);
cudaError_t launch_cross(const DevTree& t, const CrossList& full, const CrossList& leaf, const double* mp,
                         double* loc, cudaStream_t s);
// Mixed precision (kernels_mixed.cu): far-field M2L in float32 with compensated sums.
cudaError_t launch_m2l_interior_f32(const DevTree& t, const int* nodes, int n_nodes, const Stencils& st,
                                    const float* mp32, double* loc, cudaStream_t s);
cudaError_t launch_leaf_conv_mixed(const DevTree& t, const int* nodes, int n_nodes, const Stencils& st,
                                   const double* mp, double* loc, cudaStream_t s);
cudaError_t configure_kernels_mixed();

cudaError_t launch_l2l(const DevTree& t, int node_begin, int node_end, const double* mp, double* loc, double* phi,
                       double* g, int64_t n_leaf_cells, cudaStream_t s);

}  // namespace octo
