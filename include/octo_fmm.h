/*
 * octo_fmm.h -- C ABI of the GB300 (sm_103a) fast-multipole self-gravity solver.
 *
 * The method is the gravity solver of Octo-Tiger as described in the paper's
 * Section IV-C ("Octo-Tiger"): an adaptive octree whose nodes are leaves or fully
 * refined, each node carrying an 8x8x8 subgrid of cells; a leaf cell is a single
 * monopole at the cell centre, interior cells carry monopole, quadrupole and
 * octupole moments about their centre of mass; a modification conserves angular
 * momentum.  The solve runs in the three phases of Section VII-C: a bottom-up
 * traversal (P2M, M2M), same-level cell-to-cell interactions on each level (M2L,
 * plus P2P between near leaf cells), and a top-down traversal (L2L, L2P).
 * Units: G = 1, phi = -sum m / r, g = -grad phi.
 *
 * Conventions for every call below
 *  - Pointers named *_dev are device pointers (cudaMalloc'd or torch CUDA memory)
 *    owned by the caller; they must stay valid until the stream work completes.
 *  - rho, phi: float64 [n_leaf * 512]; g: float64 [3][n_leaf * 512] (structure of
 *    arrays).  Leaves are ordered as they appear in the descriptor's node array;
 *    the 512 cells of a leaf are x-fastest (local = a + 8 b + 64 c).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Compute calls are
 *    asynchronous: they enqueue work and return.  Launch and argument errors are
 *    returned immediately.  Errors found on the device (a density that is not
 *    finite and positive, a bounded wait of a kernel for its own bulk copies that
 *    ran out, a failed index check of the adjoint) are recorded in a device word of
 *    the handle and reported, once, by the next octo_fmm_stats call or by
 *    octo_fmm_forces_host, which read it back.  No kernel of this library waits on
 *    another block, kernel or device.
 *  - Return value: OCTO_OK (0) or a negative OCTO_E* status; octo_fmm_last_error()
 *    gives a message.  No C++ exception crosses this interface.
 *  - One handle is not thread-safe; use one handle per host thread or serialise.
 */
#ifndef OCTO_FMM_H
#define OCTO_FMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct octo_fmm* octo_fmm_t; /* opaque, owned by the library */

/* Octree descriptor (host memory, owned by the caller, copied by create).
 * Section IV-C: every node is a leaf or has all 8 children.
 *  level[n]        level of node n, root = 0 (exactly one root)
 *  ijk[n][3]       integer position of node n within its level, 0 <= ijk < 2^level
 *  children[n][8]  child node by octant o = ox + 2 oy + 4 oz, or -1 (all -1 = leaf);
 *                  child ijk = 2 ijk + (ox, oy, oz)
 *  origin, extent  the cubic domain [origin, origin + extent)^3; cells of level l
 *                  have width h_l = extent / (8 * 2^l). */
typedef struct {
  int32_t n_nodes;
  const int32_t* level;
  const int32_t* ijk;
  const int32_t* children;
  double origin[3];
  double extent;
} octo_tree_desc;

enum {
  OCTO_OK = 0,
  OCTO_EINVAL = -1,   /* bad argument (null pointer, unsupported theta/order/precision) */
  OCTO_ETREE = -2,    /* inconsistent octree descriptor */
  OCTO_ENOMEM = -3,   /* device or host allocation failed */
  OCTO_ECUDA = -4,    /* a CUDA runtime call failed */
  OCTO_ETIMEOUT = -5, /* a kernel's bounded wait for its own asynchronous copies ran out */
  OCTO_ENONPOS = -6,  /* a leaf density was not finite and positive (NaN, <= 0, inf) */
  OCTO_ESTATE = -7    /* call out of order (e.g. backward before a forward solve) */
};

enum {
  OCTO_FP64 = 0, /* every phase in IEEE float64 */
  OCTO_MIXED = 1 /* far-field M2L in float32 with compensated sums; P2P, correction
                    accumulation, M2M and L2L/L2P in float64 */
};

/* Plans the solve and allocates the device workspace on the current device.
 * Allocation failures return OCTO_ENOMEM and free everything allocated so far.
 * (Test hook: with the environment variable OCTO_FMM_FAIL_ALLOC_AT=N set, the N-th
 * device allocation of this call fails as if the device were out of memory.)
 * theta: opening parameter; cells A, B interact through their expansions iff
 *   theta |c_A - c_B| >= (sqrt 3 / 2)(h_A + h_B) for geometric centres c (inclusive,
 *   evaluated exactly).  Supported: 0.433 <= theta <= 1 (near field within the 26
 *   neighbouring subgrids).
 * order: expansion order, must be 3 (monopole + quadrupole + octupole, Section IV-C).
 * precision: OCTO_FP64 or OCTO_MIXED.
 * On success *out receives a handle to release with octo_fmm_destroy. */
int octo_fmm_create(const octo_tree_desc* tree, double theta, int order, int precision, octo_fmm_t* out);

/* Bottom-up traversal (Section VII-C, first phase): P2M at leaf cells (m = rho h^3
 * at the cell centre) and M2M level by level up to the root (moments about the
 * centre of mass, Section IV-C).  rho_dev: float64 [n_leaf*512], every entry finite
 * and > 0 (centres of mass divide by the mass).  P2M checks this on the device: a
 * violation leaves NaN or inf in the results and makes the next octo_fmm_stats (or
 * octo_fmm_forces_host) return OCTO_ENONPOS.
 * Starts a new solve: octo_fmm_backward accepts the state only after the matching
 * octo_fmm_interact and octo_fmm_downward have followed. */
int octo_fmm_upward(octo_fmm_t h, const double* rho_dev, void* stream);

/* Same-level cell-to-cell interactions on every level (Section VII-C, second
 * phase; the "multipole kernel"): M2L over the fixed stencils with the
 * angular-momentum correction, cross-level pairs at refinement boundaries, and
 * P2P between near leaf cells.  Needs a preceding octo_fmm_upward. */
int octo_fmm_interact(octo_fmm_t h, void* stream);

/* Top-down traversal (Section VII-C, third phase): L2L down the tree and L2P at
 * leaf cells.  Writes phi_dev [n_leaf*512] and g_dev [3][n_leaf*512]. */
int octo_fmm_downward(octo_fmm_t h, double* phi_dev, double* g_dev, void* stream);

/* The whole solve (upward + interact + downward), replayed from a CUDA graph
 * captured on first use for this stream. */
int octo_fmm_forces(octo_fmm_t h, const double* rho_dev, double* phi_dev, double* g_dev, void* stream);

/* The same solve with HOST buffers (ordinary pageable memory is fine): copies rho
 * in and phi, g out on `stream` between the caller's buffers and device buffers
 * owned by the handle, and synchronises the stream before returning.
 * rho_host [n_leaf*512], phi_host [n_leaf*512], g_host [3][n_leaf*512].
 * Returns OCTO_ENONPOS (results written, but not meaningful) if a density was not
 * finite and positive. */
int octo_fmm_forces_host(octo_fmm_t h, const double* rho_host, double* phi_host, double* g_host, void* stream);

/* Vector-Jacobian product of the last forces/upward+interact+downward solve on this
 * handle: drho = (d phi / d rho)^T dphi + (d g / d rho)^T dg, through every phase
 * including the centre-of-mass dependence of the expansions.  dphi_dev
 * [n_leaf*512], dg_dev [3][n_leaf*512], drho_dev [n_leaf*512] (overwritten).
 * Returns OCTO_ESTATE if no forward solve has run. */
int octo_fmm_backward(octo_fmm_t h, const double* dphi_dev, const double* dg_dev, double* drho_dev, void* stream);

/* Ordered interaction counts of the plan: counts[0] same-level M2L, counts[1]
 * cross-level M2L, counts[2] same-level P2P, counts[3] cross-level P2P.
 * Synchronises the device and reports a pending device-side error, then clears it:
 * OCTO_ENONPOS for a density that was not finite and positive, OCTO_ETIMEOUT for a
 * bounded wait that ran out, OCTO_ECUDA for a failed index check of the adjoint
 * (counts are filled in either case). */
int octo_fmm_stats(octo_fmm_t h, int64_t counts[4]);

/* Host-only planning: validates the tree and returns the counts above without
 * touching a GPU. */
int octo_fmm_plan_counts(const octo_tree_desc* tree, double theta, int64_t counts[4]);

/* Copies internal state to HOST memory in descriptor node order, for tests:
 * which = 0: multipoles [20][n_nodes*512]: m, X(3), M2 {xx,xy,xz,yy,yz,zz},
 *            M3 {xxx,xxy,xxz,xyy,xyz,xzz,yyy,yyz,yzz,zzz};
 * which = 1: local expansions [23][n_nodes*512]: L0, L1(3), L2(6), L3(10), dg(3)
 *            (L2 and L3 of leaf cells are not computed and read as NaN).
 * Synchronises the device. */
int octo_fmm_read_state(octo_fmm_t h, int which, double* host_out);

/* Options:
 *  key 1: replay the whole solve from a captured CUDA graph (1, default) or launch
 *         the stages one by one (0);
 *  key 2: record per-stage timing events inside the graph (1/0, default 0);
 *  key 3: strategy of the batched interaction phase (Section VII-C's same-level
 *         interactions of every level in one phase): 0 = autotune on the first
 *         forces call (default; times the candidates on this tree and keeps the
 *         fastest), 1 = one launch per item kind over all levels, 2 = one
 *         persistent launch pulling interior and leaf items of every level from a
 *         work queue (in mixed precision the float64 near field of the leaf nodes
 *         is a separate item kind, interleaved with the float32 items so that
 *         both pipes of every SM work at once);
 *  key 4: register budget of the persistent launch: 1 or 2 resident blocks per SM,
 *         or 3 (mixed precision only);
 *  key 5: mixed precision only: precision of the angular-momentum correction terms
 *         (Section IV-C) inside the float32 far-field pairs: 0 = float32 (default),
 *         1 = float64, formed from the float64 multipoles and summed in float64
 *         (a measurement variant; it runs as per-kind launches, key 3 = 1);
 *  key 6: mixed precision: stencil entries per float32 partial sum of the interior
 *         M2L items before its compensated merge: 32 (default) or 64;
 *  key 7: mixed precision: interior items of half a node with one thread per target
 *         cell (1, default), or of a quarter node with two threads per target cell,
 *         each over one half of the stencil (2).
 *  key 8: mixed precision, persistent queue: 1 = paced queue (the float32-bound
 *         and the float64-bound items in two queues, at most one block per SM
 *         holding a float64 item at a time), 0 = one merged queue (default).
 *  Keys 6 and 7 fix the interior shape, key 8 the queue; otherwise the autotuner
 *  chooses them (the shape changes the float32 summation order, so results differ
 *  at float32 rounding; the queue changes no result).
 * Setting an option drops the captured graph.  Returns OCTO_EINVAL for an unknown
 * key or value. */
int octo_fmm_set_option(octo_fmm_t h, int key, int64_t value);

/* Reads an option (keys 1-8 above; key 3 reports the strategy in use after
 * autotuning) or an autotuner measurement: keys 10, 11, 12, 13 = mean interaction
 * time in microseconds of per-kind launches and of the persistent launch with the
 * 1, 2 and 3 blocks/SM budgets; 0 when not measured (before autotuning, and key 13
 * in float64 mode); keys 14, 15, 16 = mean interaction time in microseconds of the
 * autotuner's later candidates (chunk 64, quarter-node items, paced queue; 0 when
 * not measured).  Sizes of the handle (read-only): key 20 = leaf cells
 * (n_leaf*512, the length of rho and phi), 21 = CUDA device the handle was created
 * on, 22 = octree nodes, 23 = precision (OCTO_FP64 or OCTO_MIXED), 24 = algorithmic
 * float64 flops of one octo_fmm_backward over its interaction pairs (each pair
 * expression's reverse mode as written, a fused multiply-add counting two; the
 * tree passes are not counted). */
int octo_fmm_get_option(octo_fmm_t h, int key, int64_t* value);

/* Number of kernel launches one octo_fmm_forces call enqueues. */
int octo_fmm_launches_per_solve(octo_fmm_t h);

/* Stage introspection for measurement.  The solve is a fixed list of stages, one
 * kernel launch each (e.g. "p2m", "m2m_l3", "m2l_interior", "leaf", "cross_cells",
 * "l2l_l2").  octo_fmm_stage_count returns their number; octo_fmm_stage_info gives
 * stage i's name (owned by the handle), the interactions it processes (pairs), the
 * cells it writes, its algorithmic floating-point operations (the per-pair
 * expression as written, a fused multiply-add counting two), how many of those
 * run in float64, and its algorithmic HBM bytes (tree passes: every value read or
 * written once); any output pointer may be NULL.  The stage list can change when
 * the interaction strategy changes (option 3, autotuning on the first forces call).
 * With option key 2 set to 1, the captured graph records a
 * CUDA event before every stage and after the last one; after the stream has
 * completed a forces call, octo_fmm_stage_times writes each stage's elapsed time in
 * milliseconds into ms[0..count) and returns count (cap must be >= count). */
int octo_fmm_stage_count(octo_fmm_t h);
int octo_fmm_stage_info(octo_fmm_t h, int i, const char** name, int64_t* pairs, int64_t* cells, int64_t* flops,
                        int64_t* flops64, int64_t* bytes);
int octo_fmm_stage_times(octo_fmm_t h, float* ms, int cap);

/* Allocation-free solve for callers that cannot allocate device memory at the
 * point of the call: engines whose memory manager owns all device memory and
 * forbids libraries from allocating behind its back, and time-critical loops that
 * must not pay for, or fail on, an allocation mid-run (an allocation can stall on
 * synchronisation or run out of memory).  The paper has no counterpart; it is an
 * interface addition.
 *
 * Solves n_subgrids independent single-subgrid problems, each an 8x8x8 block of
 * cells of width h forming a tree of one leaf node (so every cell pair interacts
 * exactly as point masses; G = 1, phi = -sum m / r).  rho_dev, phi_dev: float64
 * [n_subgrids * 512]; g_dev: float64 [3][n_subgrids * 512]; cells x-fastest inside
 * a subgrid.  All three are caller-owned device buffers; results agree with
 * octo_fmm_forces on a one-node tree.
 *
 * No memory is allocated by this call: the only intermediate state (the cell
 * masses) lives in one fixed device array inside the library, sized for at most
 * 1024 subgrids (4 MiB), which every GPU that loads the library keeps until the
 * process exits.  With CUDA's lazy module loading (the default) the driver
 * reserves that array, and loads this code, at the first call on each device; so
 * make one call (n_subgrids = 1 is enough) during set-up, and every later call
 * allocates nothing.  n_subgrids outside [0, 1024] returns OCTO_EINVAL (message via
 * octo_fmm_last_error(NULL)) without launching anything.  The first call on a
 * device looks up that array's device address (once per device, with the device
 * current); make that first call before any stream capture.  Every call reuses
 * the same array and keeps nothing from earlier calls, so calls whose work
 * overlaps on the GPU (different streams, different host threads) race: order
 * them on one stream.  Asynchronous on `stream` like the other compute calls. */
int octo_fmm_subgrids_noalloc(int n_subgrids, const double* rho_dev, double h, double* phi_dev, double* g_dev,
                              void* stream);

/* Self-consistent-field (SCF) initial models of a synchronously rotating binary of
 * two polytropes (Section IV-C: the binary models are initialised by an iterative
 * SCF technique; the hydrostatic equilibrium equation in the rotating frame,
 * integrated, is an algebraic relation between the effective potential and the
 * enthalpy).  Inside star i: H + Phi - Omega^2 w^2 / 2 = C_i with the enthalpy
 * H = (n + 1) K rho^(1/n) and w the distance from the rotation axis (parallel to z,
 * through the centre of mass).  The constants Omega^2, C_1, C_2 follow from H = 0
 * at three surface cells. */
typedef struct {
  double n;                        /* polytropic index of both stars, > 0 */
  double rho_max[2];               /* the maximum density each star keeps, > 0 */
  double rho_floor;                /* density outside the stars, >= 0 */
  int64_t cell_a, cell_b, cell_c;  /* leaf cells (indices into rho, 0 <= i < n_leaf*512) on
                                      the surfaces: A and B of star 1 (at different distances
                                      from the axis), C of star 2 */
  double x_split;                  /* cells whose centre has x < x_split belong to star 1 */
} octo_scf_params;

/* One SCF step.  phi_dev: the potential of the density in rho_dev (e.g. from
 * octo_fmm_forces).  rho_dev is overwritten with the new density:
 * rho = rho_max_i (H / H_max_i)^n + rho_floor where H > 0, else rho_floor.  stats
 * (host, 8 doubles, may be NULL): Omega^2, C_1, C_2, max |rho_new - rho| /
 * max(rho_max), and of the state that produced phi: W = sum m phi / 2, T =
 * Omega^2 sum m w^2 / 2, Pi = sum P h^3 (P = K_i rho^(1 + 1/n), K_i from H_max_i),
 * and the virial error |2T + W + 3 Pi| / |W|.  Synchronises the stream.  The
 * first call allocates a small device scratch.  Errors: OCTO_EINVAL (bad
 * parameters, cell indices out of range), OCTO_ENOMEM, OCTO_ECUDA. */
int octo_fmm_scf_step(octo_fmm_t h, const octo_scf_params* p, double* rho_dev, const double* phi_dev, double* stats,
                      void* stream);

/* The SCF iteration: octo_fmm_forces on rho_dev, then octo_fmm_scf_step, repeated
 * until the largest density change (stats[3]) is below tol or max_iter steps ran.
 * rho_dev: initial guess in, equilibrium out.  history (host, may be NULL):
 * [max_iter][8] stats of every step; *n_iter (may be NULL) receives the number of
 * steps.  The potential uses the handle's own buffers. */
int octo_fmm_scf_solve(octo_fmm_t h, const octo_scf_params* p, double* rho_dev, int max_iter, double tol,
                       double* history, int* n_iter, void* stream);

/* Measured arithmetic peak of the current device, the denominator of the solver's
 * roofline fractions (the paper has no counterpart; the interaction kernels are
 * bound by the float64 and float32 fused multiply-add pipes, Section VII-C's
 * "multipole kernel").  Runs independent fused multiply-add chains in float64
 * (fp64 = 1) or float32 (fp64 = 0) on every SM, 3 timed launches of 20-50 ms after
 * a warm-up, on `stream`, synchronises, and writes the rate in flop/s (an FMA
 * counting 2) to *flops_per_s.  Allocates nothing.  Errors: OCTO_EINVAL, OCTO_ECUDA
 * (message via octo_fmm_last_error(NULL)). */
int octo_fmm_measure_peak(int fp64, double* flops_per_s, void* stream);

/* Message for the last failing call on h (or for create failures, h = NULL). */
const char* octo_fmm_last_error(octo_fmm_t h);

/* Frees the handle and its device workspace (synchronises the device first). */
void octo_fmm_destroy(octo_fmm_t h);

#ifdef __cplusplus
}
#endif

#endif /* OCTO_FMM_H */
