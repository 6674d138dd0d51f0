// Mixed-precision interaction kernels whose interior items sum 64 stencil entries
// per float32 partial (the autotuner's alternative to 32, kernels_interact.cu);
// a translation unit of their own so that the shape variants compile in parallel.
#include "interact.cuh"

namespace octo {

cudaError_t interior_items_b64(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
  return MixedShapes<64>::interior(t, a, s);
}

cudaError_t persistent_b64(const DevTree& t, const InteractArgs& a, cudaStream_t s) {
  return MixedShapes<64>::persistent(t, a, s);
}

cudaError_t persistent_occupancy_b64(int min_blocks, const Stencils& st, const CrossCells& xc, int* per_sm) {
  return MixedShapes<64>::occupancy(min_blocks, st, xc, per_sm);
}

}  // namespace octo
