// Measured arithmetic peaks of the GPU (octo_fmm_measure_peak, include/octo_fmm.h):
// the denominators of the solver's float64 / float32 roofline fractions, measured on
// the device that runs the solve instead of derived from unit counts and the
// nominal clock.
//
// Each thread runs kChains independent fused multiply-add chains (x <- x a + b), so
// the pipe, not the FMA latency, bounds the rate; the grid is 8 blocks of 256
// threads per SM.  The chains' sum is stored only when it equals a value it never
// reaches, which keeps the work alive without a result buffer.
#include <cuda_runtime.h>

#include <string>

#include "../../include/octo_fmm.h"
#include "plan.h"

namespace octo {

namespace {

constexpr int kChains = 8, kUnroll = 16, kThreadsPeak = 256, kBlocksPerSm = 8;

__device__ double g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(kThreadsPeak) k_fma_chains(T a, T b, int iters) {
  T x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = (T)(threadIdx.x + 1 + i) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == (T)-1.25) g_peak_sink = (double)s;  // never true: the chains converge to b / (1 - a) > 0
}

template <typename T>
cudaError_t time_chains(int iters, int grid, cudaStream_t s, float* ms) {
  const T a = (T)0.999, b = (T)1e-4;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_fma_chains<T><<<grid, kThreadsPeak, 0, s>>>(a, b, iters);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
    k_fma_chains<T><<<grid, kThreadsPeak, 0, s>>>(a, b, iters);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  *ms /= 3.0f;
  return e;
}

}  // namespace

}  // namespace octo

using namespace octo;

extern "C" int octo_fmm_measure_peak(int fp64, double* flops_per_s, void* stream) {
  if (!flops_per_s || (fp64 != 0 && fp64 != 1)) {
    set_global_error("octo_fmm_measure_peak: bad arguments");
    return OCTO_EINVAL;
  }
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_global_error(std::string("octo_fmm_measure_peak: ") + cudaGetErrorString(e));
    return OCTO_ECUDA;
  }
  const int grid = n_sm * kBlocksPerSm;
  // about 20-50 ms per launch at the nominal rates (float64 is 1/64 of float32)
  const int iters = fp64 ? 600 : 38400;
  float ms = 0.0f;
  e = fp64 ? time_chains<double>(iters, grid, (cudaStream_t)stream, &ms)
           : time_chains<float>(iters, grid, (cudaStream_t)stream, &ms);
  if (e != cudaSuccess || !(ms > 0.0f)) {
    set_global_error(std::string("octo_fmm_measure_peak: ") + cudaGetErrorString(e));
    return OCTO_ECUDA;
  }
  const double flops = 2.0 * (double)grid * kThreadsPeak * (double)iters * kUnroll * kChains;
  *flops_per_s = flops / (ms * 1e-3);
  return OCTO_OK;
}
