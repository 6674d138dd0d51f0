// Self-consistent-field (SCF) initial models (octo_fmm_scf_step, octo_fmm_scf_solve;
// include/octo_fmm.h).  Section IV-C of the paper initialises its binaries by an
// SCF iteration: the hydrostatic equilibrium equation in the rotating frame,
// integrated, is an algebraic relation between the effective potential and the
// enthalpy, H + Phi - Omega^2 w^2 / 2 = C_i inside star i, with H = (n + 1) K
// rho^(1/n) for a polytrope.  One step, given the potential Phi of the current
// density (from the FMM solve):
//   1. rotation axis parallel to z through the centre of mass of the density;
//   2. H = 0 at three given surface cells, A and B of star 1 and C of star 2:
//      Omega^2 = 2 (Phi_A - Phi_B) / (w_A^2 - w_B^2), C_1 = Phi_A - Omega^2 w_A^2 / 2,
//      C_2 = Phi_C - Omega^2 w_C^2 / 2;
//   3. H = C_i - Phi + Omega^2 w^2 / 2, star 1 where x < x_split, else star 2;
//   4. rho_new = rho_max_i (H / H_max_i)^n + rho_floor where H > 0, else rho_floor;
//   5. diagnostics of the state that produced Phi: largest density change over
//      max(rho_max), W = sum m Phi / 2, T = Omega^2 sum m w^2 / 2,
//      Pi = sum K_i rho^(1 + 1/n) h^3 with K_i = H_max_i / ((n + 1) rho_max_i^(1/n)),
//      and the virial error |2 T + W + 3 Pi| / |W|.
// Every reduction is deterministic: per-node partials, then one block in node order.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/octo_fmm.h"
#include "handle.h"

namespace octo {

namespace {

constexpr int kScfThreads = 256;
// per-node partials: 0..2 mass, m x, m y | 3, 4 H max of star 1, 2 | 5 max |drho| |
// 6, 7, 8 W, T, Pi
constexpr int kScfPartials = 9;
// device constants: 0 M, 1 xc, 2 yc, 3 omega2, 4 c1, 5 c2, 6 hmax1, 7 hmax2, then the
// 8 statistics (octo_fmm_scf_step) at 8..15
constexpr int kScfConsts = 16;

struct ScfArgs {
  DevTree t;
  const int* leaf_nodes;  // dnode of every leaf, any order
  int n_leaf_nodes;
  const int* node_of_lid; // dnode of leaf lid (descriptor leaf order)
  double* rho;
  const double* phi;
  double* part;           // [n_leaf_nodes][kScfPartials]
  double* c;              // [kScfConsts]
  octo_scf_params p;
};

__device__ __forceinline__ void cell_centre(const DevTree& t, int node, int l, double x[3]) {
  const double h = t.h[t.level[node]];
  const int loc[3] = {l & 7, (l >> 3) & 7, l >> 6};
  for (int d = 0; d < 3; ++d) x[d] = t.origin[d] + h * ((double)(8 * t.ijk[3 * node + d] + loc[d]) + 0.5);
}

// Block reductions in a fixed order (shared-memory tree over the 256 threads).
template <int OP>  // 0 sum, 1 max
__device__ double block_reduce(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kScfThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = OP == 0 ? sh[threadIdx.x] + sh[threadIdx.x + s]
                                                   : fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// 1. mass and first moments per leaf node
__global__ void __launch_bounds__(kScfThreads) k_scf_mass(ScfArgs a) {
  __shared__ double sh[kScfThreads];
  const int node = a.leaf_nodes[blockIdx.x];
  const int64_t lid = a.t.leaf_id[node];
  const double h3 = a.t.h3[a.t.level[node]];
  double m = 0, mx = 0, my = 0;
  for (int l = threadIdx.x; l < 512; l += kScfThreads) {
    double x[3];
    cell_centre(a.t, node, l, x);
    const double mc = a.rho[lid * 512 + l] * h3;
    m += mc;
    mx += mc * x[0];
    my += mc * x[1];
  }
  m = block_reduce<0>(m, sh);
  mx = block_reduce<0>(mx, sh);
  my = block_reduce<0>(my, sh);
  if (threadIdx.x == 0) {
    double* q = a.part + (int64_t)blockIdx.x * kScfPartials;
    q[0] = m, q[1] = mx, q[2] = my;
  }
}

// Sum (or max) of partial column k over the nodes, in node order per thread, then
// across the block.
template <int OP>
__device__ double column(const ScfArgs& a, int k, double* sh) {
  double v = OP == 0 ? 0.0 : -DBL_MAX;
  for (int i = threadIdx.x; i < a.n_leaf_nodes; i += kScfThreads) {
    const double q = a.part[(int64_t)i * kScfPartials + k];
    v = OP == 0 ? v + q : fmax(v, q);
  }
  return block_reduce<OP>(v, sh);
}

__device__ __forceinline__ double w2_of(const ScfArgs& a, const double x[3]) {
  const double dx = x[0] - a.c[1], dy = x[1] - a.c[2];
  return dx * dx + dy * dy;
}

// 2. centre of mass, Omega^2, C_1, C_2 (one block)
__global__ void __launch_bounds__(kScfThreads) k_scf_constants(ScfArgs a) {
  __shared__ double sh[kScfThreads];
  const double M = column<0>(a, 0, sh), MX = column<0>(a, 1, sh), MY = column<0>(a, 2, sh);
  if (threadIdx.x == 0) {
    a.c[0] = M;
    a.c[1] = MX / M;
    a.c[2] = MY / M;
    const int64_t cells[3] = {a.p.cell_a, a.p.cell_b, a.p.cell_c};
    double phi[3], w2[3];
    for (int i = 0; i < 3; ++i) {
      const int64_t lid = cells[i] / 512;
      const int l = (int)(cells[i] % 512);
      double x[3];
      cell_centre(a.t, a.node_of_lid[lid], l, x);
      phi[i] = a.phi[cells[i]];
      w2[i] = w2_of(a, x);
    }
    const double omega2 = 2.0 * (phi[0] - phi[1]) / (w2[0] - w2[1]);
    a.c[3] = omega2;
    a.c[4] = phi[0] - 0.5 * omega2 * w2[0];
    a.c[5] = phi[2] - 0.5 * omega2 * w2[2];
  }
}

__device__ __forceinline__ double enthalpy(const ScfArgs& a, const double x[3], double phi, bool star1) {
  return (star1 ? a.c[4] : a.c[5]) - phi + 0.5 * a.c[3] * w2_of(a, x);
}

// 3. largest enthalpy of each star per leaf node
__global__ void __launch_bounds__(kScfThreads) k_scf_hmax(ScfArgs a) {
  __shared__ double sh[kScfThreads];
  const int node = a.leaf_nodes[blockIdx.x];
  const int64_t lid = a.t.leaf_id[node];
  double h1 = -DBL_MAX, h2 = -DBL_MAX;
  for (int l = threadIdx.x; l < 512; l += kScfThreads) {
    double x[3];
    cell_centre(a.t, node, l, x);
    const bool s1 = x[0] < a.p.x_split;
    const double H = enthalpy(a, x, a.phi[lid * 512 + l], s1);
    if (s1)
      h1 = fmax(h1, H);
    else
      h2 = fmax(h2, H);
  }
  h1 = block_reduce<1>(h1, sh);
  h2 = block_reduce<1>(h2, sh);
  if (threadIdx.x == 0) {
    double* q = a.part + (int64_t)blockIdx.x * kScfPartials;
    q[3] = h1, q[4] = h2;
  }
}

__global__ void __launch_bounds__(kScfThreads) k_scf_hmax_all(ScfArgs a) {
  __shared__ double sh[kScfThreads];
  const double h1 = column<1>(a, 3, sh), h2 = column<1>(a, 4, sh);
  if (threadIdx.x == 0) a.c[6] = h1, a.c[7] = h2;
}

// 4./5. new density (in place: each thread reads its cell's old value first) and
// the per-node partials of the diagnostics
__global__ void __launch_bounds__(kScfThreads) k_scf_density(ScfArgs a) {
  __shared__ double sh[kScfThreads];
  const int node = a.leaf_nodes[blockIdx.x];
  const int64_t lid = a.t.leaf_id[node];
  const double h3 = a.t.h3[a.t.level[node]];
  const double n = a.p.n;
  double dmax = 0, W = 0, T = 0, Pi = 0;
  for (int l = threadIdx.x; l < 512; l += kScfThreads) {
    double x[3];
    cell_centre(a.t, node, l, x);
    const bool s1 = x[0] < a.p.x_split;
    const int64_t k = lid * 512 + l;
    const double phi = a.phi[k], rho = a.rho[k];
    const double H = enthalpy(a, x, phi, s1);
    const double hmax = s1 ? a.c[6] : a.c[7];
    const double rmax = s1 ? a.p.rho_max[0] : a.p.rho_max[1];
    const double rnew = H > 0.0 ? rmax * pow(H / hmax, n) + a.p.rho_floor : a.p.rho_floor;
    const double m = rho * h3;
    const double K = hmax / ((n + 1.0) * pow(rmax, 1.0 / n));
    dmax = fmax(dmax, fabs(rnew - rho));
    W += m * phi;
    T += m * w2_of(a, x);
    Pi += K * pow(rho, 1.0 + 1.0 / n) * h3;
    a.rho[k] = rnew;
  }
  dmax = block_reduce<1>(dmax, sh);
  W = block_reduce<0>(W, sh);
  T = block_reduce<0>(T, sh);
  Pi = block_reduce<0>(Pi, sh);
  if (threadIdx.x == 0) {
    double* q = a.part + (int64_t)blockIdx.x * kScfPartials;
    q[5] = dmax, q[6] = W, q[7] = T, q[8] = Pi;
  }
}

__global__ void __launch_bounds__(kScfThreads) k_scf_stats(ScfArgs a) {
  __shared__ double sh[kScfThreads];
  const double dmax = column<1>(a, 5, sh), W = 0.5 * column<0>(a, 6, sh);
  const double T = 0.5 * a.c[3] * column<0>(a, 7, sh), Pi = column<0>(a, 8, sh);
  if (threadIdx.x == 0) {
    double* st = a.c + 8;
    st[0] = a.c[3];
    st[1] = a.c[4];
    st[2] = a.c[5];
    st[3] = dmax / fmax(a.p.rho_max[0], a.p.rho_max[1]);
    st[4] = W;
    st[5] = T;
    st[6] = Pi;
    st[7] = fabs(2.0 * T + W + 3.0 * Pi) / fabs(W);
  }
}

int scf_fail(octo_fmm* h, int code, const std::string& msg) {
  h->err = msg;
  return code;
}

// Checks the parameters against the handle; allocates the SCF scratch (partials,
// constants, the leaf-to-node map) on first use.
int scf_prepare(octo_fmm* h, const octo_scf_params* p) {
  if (!p) return scf_fail(h, OCTO_EINVAL, "scf: params is null");
  const int64_t nl = (int64_t)h->plan.n_leaf * 512;
  if (!(p->n > 0.0) || !(p->rho_max[0] > 0.0) || !(p->rho_max[1] > 0.0) || !(p->rho_floor >= 0.0))
    return scf_fail(h, OCTO_EINVAL, "scf: need n > 0, rho_max > 0 and rho_floor >= 0");
  for (int64_t c : {p->cell_a, p->cell_b, p->cell_c})
    if (c < 0 || c >= nl) return scf_fail(h, OCTO_EINVAL, "scf: a surface cell index is outside the leaf cells");
  if (p->cell_a == p->cell_b) return scf_fail(h, OCTO_EINVAL, "scf: cells A and B must differ");
  if (h->d_scf) return OCTO_OK;
  const Plan& P = h->plan;
  std::vector<int> node_of_lid(P.n_leaf, -1);
  for (int k = 0; k < P.n_nodes; ++k)
    if (P.leaf_id[k] >= 0) node_of_lid[P.leaf_id[k]] = k;
  const size_t n_part = (size_t)P.leaf_nodes.size() * kScfPartials;
  cudaError_t e = cudaMalloc(&h->d_scf, sizeof(double) * (n_part + kScfConsts));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_scf_nodes, sizeof(int) * node_of_lid.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_scf_nodes, node_of_lid.data(), sizeof(int) * node_of_lid.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(h->d_scf);
    cudaFree(h->d_scf_nodes);
    h->d_scf = nullptr;
    h->d_scf_nodes = nullptr;
    return scf_fail(h, e == cudaErrorMemoryAllocation ? OCTO_ENOMEM : OCTO_ECUDA,
                    std::string("scf scratch: ") + cudaGetErrorString(e));
  }
  return OCTO_OK;
}

int scf_step(octo_fmm* h, const octo_scf_params* p, double* rho, const double* phi, double* stats, cudaStream_t s) {
  ScfArgs a;
  a.t = h->dt;
  a.leaf_nodes = h->d_leaf;
  a.n_leaf_nodes = (int)h->plan.leaf_nodes.size();
  a.node_of_lid = h->d_scf_nodes;
  a.rho = rho;
  a.phi = phi;
  a.part = h->d_scf;
  a.c = h->d_scf + (size_t)a.n_leaf_nodes * kScfPartials;
  a.p = *p;
  const int nb = a.n_leaf_nodes;
  k_scf_mass<<<nb, kScfThreads, 0, s>>>(a);
  k_scf_constants<<<1, kScfThreads, 0, s>>>(a);
  k_scf_hmax<<<nb, kScfThreads, 0, s>>>(a);
  k_scf_hmax_all<<<1, kScfThreads, 0, s>>>(a);
  k_scf_density<<<nb, kScfThreads, 0, s>>>(a);
  k_scf_stats<<<1, kScfThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  double st[8];
  if (e == cudaSuccess) e = cudaMemcpyAsync(st, a.c + 8, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return scf_fail(h, OCTO_ECUDA, std::string("scf step: ") + cudaGetErrorString(e));
  if (stats)
    for (int i = 0; i < 8; ++i) stats[i] = st[i];
  return OCTO_OK;
}

}  // namespace

}  // namespace octo

using namespace octo;

extern "C" int octo_fmm_scf_step(octo_fmm_t h, const octo_scf_params* p, double* rho_dev, const double* phi_dev,
                                 double* stats, void* stream) {
  if (!h || !rho_dev || !phi_dev) return h ? scf_fail(h, OCTO_EINVAL, "scf: null buffer") : OCTO_EINVAL;
  if (h->plan.leaf_nodes.empty()) return scf_fail(h, OCTO_EINVAL, "scf: the tree has no leaf cells");
  int rc = scf_prepare(h, p);
  if (rc != OCTO_OK) return rc;
  return scf_step(h, p, rho_dev, phi_dev, stats, (cudaStream_t)stream);
}

extern "C" int octo_fmm_scf_solve(octo_fmm_t h, const octo_scf_params* p, double* rho_dev, int max_iter, double tol,
                                  double* history, int* n_iter, void* stream) {
  if (!h || !rho_dev) return h ? scf_fail(h, OCTO_EINVAL, "scf: null buffer") : OCTO_EINVAL;
  if (max_iter < 1) return scf_fail(h, OCTO_EINVAL, "scf: max_iter must be >= 1");
  int rc = scf_prepare(h, p);
  if (rc != OCTO_OK) return rc;
  const int64_t n = h->n_leaf_cells();
  double* phi = h->d_io + n;   // the handle's own result buffers (as octo_fmm_forces_host)
  double* g = h->d_io + 2 * n;
  int it = 0;
  for (; it < max_iter; ++it) {
    rc = octo_fmm_forces(h, rho_dev, phi, g, stream);
    if (rc != OCTO_OK) break;
    double st[8];
    rc = scf_step(h, p, rho_dev, phi, st, (cudaStream_t)stream);
    if (rc != OCTO_OK) break;
    if (history)
      for (int i = 0; i < 8; ++i) history[(size_t)it * 8 + i] = st[i];
    if (st[3] < tol) {
      ++it;
      break;
    }
  }
  if (n_iter) *n_iter = it;
  return rc;
}
