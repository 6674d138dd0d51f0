// Allocation-free entry point (octo_fmm_subgrids_noalloc, include/octo_fmm.h).
//
// Some callers cannot allocate device memory when they need the solve: engines
// whose memory manager owns every byte of device memory and forbids libraries from
// allocating behind its back, and time-critical loops that must not stall on, or
// fail on, an allocation mid-run.  For them this file offers the solve of a batch of
// independent single-subgrid problems (each one 8^3 cells, the tree being a single
// leaf node) with no allocation at all: the caller passes rho, phi and g, and the
// only intermediate state - the cell masses written by the P2M step and read by the
// interaction step, the workspace that octo_fmm_forces keeps in handle-owned memory -
// lives in one fixed file-scope device array.
//
// With CUDA's lazy module loading (the default), the first use of this file's kernels
// or of the array on a device - the first call on that device - loads the module,
// and that load is when the driver reserves the array and the module's code.  Every
// later call allocates nothing.
//
// For a tree of one leaf node every pair of distinct cells is either well separated
// (M2L between two monopoles at cell centres) or near (P2P); both are the exact
// point-mass interaction, so each subgrid's result is its direct sum.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/octo_fmm.h"
#include "device.cuh"
#include "plan.h"

namespace octo {

namespace {

// Largest batch the scratch array holds: 1024 subgrids (4 MiB of masses).  Every
// GPU that loads the library keeps this array until the process exits.
constexpr int kNoallocMaxSubgrids = 1024;
static __device__ __align__(256) double g_noalloc_mass[kNoallocMaxSubgrids * 512];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {nullptr};  // per device: device address of g_noalloc_mass

// P2M: m = rho h^3 into the scratch masses (every entry used below is written).
__global__ void k_noalloc_p2m(const double* __restrict__ rho, double h3, int n, double* __restrict__ mass) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * 512) mass[i] = rho[i] * h3;
}

// One block per subgrid, one thread per target cell: all other cells of the
// subgrid as exact point masses, phi = -sum m / r, g = -sum m (x_i - x_j) / r^3.
__global__ void __launch_bounds__(512) k_noalloc_cells(const double* __restrict__ mass, double h, int n,
                                                       double* __restrict__ phi, double* __restrict__ g) {
  __shared__ double m[512];
  const int s = blockIdx.x, i = threadIdx.x;
  m[i] = mass[s * 512 + i];
  __syncthreads();
  const int ax = i & 7, ay = (i >> 3) & 7, az = i >> 6;
  double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
  for (int j = 0; j < 512; ++j) {
    if (j == i) continue;
    // R = x_i - x_j = -(d h) with d the integer offset of cell j from cell i
    const double dx = (double)((j & 7) - ax), dy = (double)(((j >> 3) & 7) - ay), dz = (double)((j >> 6) - az);
    const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double ir = rsqrt_f64(r2);
    const double mr = m[j] * ir, mr3 = mr * ir * ir;
    p -= mr;
    gx += mr3 * dx;
    gy += mr3 * dy;
    gz += mr3 * dz;
  }
  const int64_t k = (int64_t)s * 512 + i, NL = (int64_t)n * 512;
  const double ih = 1.0 / h;
  phi[k] = p * ih;
  g[k] = gx * ih * ih;
  g[NL + k] = gy * ih * ih;
  g[2 * NL + k] = gz * ih * ih;
}

// Failure: the message is reported by octo_fmm_last_error(NULL).
int noalloc_fail(int code, const std::string& msg) {
  set_global_error(msg);
  return code;
}

}  // namespace

}  // namespace octo

using namespace octo;

extern "C" int octo_fmm_subgrids_noalloc(int n_subgrids, const double* rho_dev, double h, double* phi_dev,
                                          double* g_dev, void* stream) {
  if (n_subgrids < 0 || n_subgrids > kNoallocMaxSubgrids)
    return noalloc_fail(OCTO_EINVAL, "octo_fmm_subgrids_noalloc: n_subgrids must be in [0, " +
                                         std::to_string(kNoallocMaxSubgrids) + "]");
  if (!rho_dev || !phi_dev || !g_dev) return noalloc_fail(OCTO_EINVAL, "octo_fmm_subgrids_noalloc: null buffer");
  if (!(h > 0.0)) return noalloc_fail(OCTO_EINVAL, "octo_fmm_subgrids_noalloc: cell width must be positive");
  if (n_subgrids == 0) return OCTO_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(OCTO_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return noalloc_fail(OCTO_EINVAL, "octo_fmm_subgrids_noalloc: device index above 63");
  double* mass = nullptr;
  {
    // set-up, once per device with that device current: the device address of the
    // scratch array (its host-side name is only a stand-in and must not be passed)
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_mass);
      if (e != cudaSuccess) {
        set_global_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return OCTO_ECUDA;
      }
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    mass = g_noalloc_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int n = n_subgrids;
  // A launch error is read with cudaGetLastError, which also returns (and clears) an
  // error left by an earlier, unrelated runtime call of this thread: take that one
  // first, so that it is not reported as a failure of these launches.
  (void)cudaGetLastError();
  k_noalloc_p2m<<<(n * 512 + 255) / 256, 256, 0, s>>>(rho_dev, h * h * h, n, mass);
  k_noalloc_cells<<<n, 512, 0, s>>>(mass, h, n, phi_dev, g_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(OCTO_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return OCTO_OK;
}
