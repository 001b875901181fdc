/*
 * hmg.h -- C ABI of a matrix-free high-order h-/p-multigrid solver for
 *          -div(mu grad u) = f,  u = 0 on the boundary,
 * discretized with continuous Q_p elements (1 <= p <= 16) on Gauss-Lobatto-Legendre
 * nodes of a structured, smoothly mapped quadrilateral (2D) or hexahedral (3D) mesh,
 * after H. Sundar, G. Stadler, G. Biros, "Comparison of multigrid algorithms for
 * high-order continuous finite element discretizations" (arXiv:1402.5938).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - Every function returns hmg_status (0 = OK, < 0 = error). No C++ exception crosses
 *   the ABI. hmg_last_error() gives a message for the calling thread's last failure.
 * - A problem handle owns its multigrid hierarchy in device memory of the device that
 *   was current at hmg_setup(); later calls must run with that device current.
 *   Handles are not thread-safe: use one handle per host thread.
 * - "_dev" pointers are device pointers owned by the caller (for example PyTorch
 *   tensors): contiguous FP64 vectors of the level's length hmg_ndof(), global nodes
 *   numbered lexicographically with x fastest, Dirichlet (boundary) nodes included.
 *   Boundary entries are ignored on input and written as zero on output.
 * - `stream` is a cudaStream_t (NULL = legacy default stream). Work is queued on it in
 *   order; functions that return host results (hmg_solve, hmg_lambda_max) synchronize
 *   that stream before returning.
 * - Level 0 is the finest level; level nlevels-1 is the coarsest (exact solve).
 */
#ifndef HMG_H
#define HMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HMG_OK = 0,
  HMG_EINVAL = -1,   /* invalid argument or descriptor */
  HMG_ENOMEM = -2,   /* device or host allocation failed, or over the memory budget */
  HMG_ENOCONV = -3,  /* solver reached maxit; solution and history are still written */
  HMG_EDEVICE = -4,  /* a CUDA call failed */
  HMG_ETIMEOUT = -5, /* a bounded wait gave up */
  HMG_EBUSY = -6,    /* result not ready yet (serving) */
  HMG_ENAN = -7      /* a non-finite value was detected in the input or the iteration */
} hmg_status;

typedef enum { HMG_HIER_H = 0, HMG_HIER_P = 1 } hmg_hier;
typedef enum {
  HMG_SMOOTH_JACOBI = 0,
  HMG_SMOOTH_CHEB = 1,
  HMG_SMOOTH_L1JACOBI = 2,
  HMG_SMOOTH_BLOCKJACOBI = 3
} hmg_smoother;
typedef enum { HMG_MODE_MG = 0, HMG_MODE_PCG = 1 } hmg_mode;
typedef enum { HMG_PREC_FP64 = 0, HMG_PREC_FP32 = 1, HMG_PREC_FP16 = 2, HMG_PREC_BF16 = 3 } hmg_prec;
/* Arithmetic of the finest level's FP64 operator (hmg_desc.fp64_arith). */
typedef enum { HMG_ARITH_FP64 = 0, HMG_ARITH_DF64 = 1 } hmg_arith;

/*
 * Problem descriptor (paper Sec. 2 problem statement, Sec. 2.3 meshing, Sec. 4.3 settings).
 *   dim, nelem, order  : structured nelem[0] x nelem[1] (x nelem[2]) mesh of [0,1]^dim, Q_order.
 *   warp_amp           : the mesh is mapped by x_i += warp_amp * prod_j sin(pi X_j) applied to
 *                        the reference coordinates X (0 = unit square/cube). The map fixes the
 *                        boundary; |warp_amp| * pi < 1 keeps it a diffeomorphism.
 *   mu_a, mu_b, mu_k   : coefficient mu(x) = mu_a + mu_b * sum_i cos^2(mu_k * pi * x_i), evaluated
 *                        at each level's Gauss points (q = p+1 per direction); needs mu > 0.
 *   hier, n_hlevels    : h-multigrid (Sec. 3.1.1): n_hlevels meshes at fixed p, each halving the
 *                        elements per axis. p-multigrid (Sec. 3.1.2): p, p/2, ..., 1 on the fine
 *                        mesh, then n_hlevels-1 mesh halvings at p = 1.
 *   smoother, nu_pre, nu_post, omega : point-Jacobi x += omega D^-1 (b - A x), Chebyshev-
 *                        accelerated Jacobi of degree nu (Sec. 3.2.1), or l1-Jacobi (Sec. 4.4,
 *                        Table 7): the Jacobi step with D_l1 = diag(sum_j |a_ij|) over the interior
 *                        unknowns, computed at setup by probing A with (2p+1)^d color classes;
 *                        or element-block Jacobi (Sec. 3.2.3, Sec. 4.4, Table 7): the damped step
 *                        x += omega M^-1 (b - A x) with M block diagonal, the exact element
 *                        matrix on each element's (p-1)^d interior nodes (inverted at setup) and
 *                        the diagonal on the nodes elements share; FP64 only (smooth_prec
 *                        HMG_PREC_FP64) and (p-1)^d <= 1000 (E * (p-1)^(2d) doubles per level);
 *                        p = 1 levels have no interior nodes and take the point step.
 *                        omega for the Jacobi forms only.
 *   arnoldi_iters, cheb_lo_frac, cheb_safety : Chebyshev interval [lo_frac*s*lam, s*lam] with
 *                        lam the largest Ritz value of D^-1 A after arnoldi_iters Arnoldi steps
 *                        (Sec. 3.2.2: [lam/4, lam], 10 iterations).
 *   arnoldi_seed       : base seed of the SplitMix64 start vectors (level k uses seed + k);
 *                        0 selects 0x1402593800000000.
 *   smooth_prec        : HMG_PREC_FP64, or HMG_PREC_FP32 for the V-cycle's smoother, residual and
 *                        transfer work below the FP64 fine residual / PCG / coarsest solve.
 *                        HMG_PREC_FP16 / HMG_PREC_BF16: the same FP32 V-cycle whose operator
 *                        applies store the geometric factors in 16 bits (FP16 with a power-of-two
 *                        scale per element; BF16 unscaled), read in FP32 arithmetic on every
 *                        level; PCG then uses the flexible (Polak-Ribiere) beta, since such a
 *                        preconditioner is only nearly linear.
 *   node_xyz, mu_fn    : optional user geometry and coefficient (Sec. 2: a general domain Omega
 *                        and mu(x) >= mu_0 > 0); NULL keeps the warp map and the cos^2 formula.
 *                        The solve server takes built-in geometry and coefficients only.
 *   solve_graph        : 1 (default): hmg_solve runs each solve as one instantiated CUDA graph with
 *                        a device-side loop (no host round trip per iteration); 0: host-driven loop
 *                        that reads the residual norm back every iteration. Same results.
 *   fp64_arith         : HMG_ARITH_FP64 (default): the finest level's operator (hmg_apply, the PCG
 *                        and MG residuals, and with an FP64 V-cycle its finest smoothing) in FP64
 *                        arithmetic, in the fastest form timed at setup. HMG_ARITH_DF64: the same
 *                        operator (Sec. 2.3) with FP64 vectors and the FP64 factors split into float
 *                        pairs, computed in double-float arithmetic (pairs of FP32 numbers, about 48
 *                        significant bits; rounding errors a few 2^-46 relative to the magnitudes
 *                        summed instead of 2^-53), for GPUs whose FP64 rate is a small fraction of
 *                        their FP32 rate. Finest orders 1-8 (else FP64 as by default); one more
 *                        copy of the finest level's factors (8 bytes per value). Values (factors,
 *                        x, intermediates) must stay inside FP32's exponent range (magnitudes
 *                        below about 3e38; below about 1e-31 the low word loses bits, below 1e-38
 *                        the value itself). Not in the paper: an arithmetic choice of this
 *                        implementation.
 */
typedef struct hmg_desc {
  int dim;
  int nelem[3];
  int order;
  double warp_amp;
  double mu_a, mu_b, mu_k;
  int hier;
  int n_hlevels;
  int smoother;
  int nu_pre, nu_post;
  double omega;
  int arnoldi_iters;
  double cheb_lo_frac;
  double cheb_safety;
  unsigned long long arnoldi_seed;
  int smooth_prec;
  int solve_graph;
  /* Optional, read during hmg_setup only (host memory, owned by the caller): */
  const double* node_xyz; /* [dim][N] physical coordinates of the finest level's nodes (numbering
                             x fastest, boundary nodes included), replacing the warp map; the
                             mapped mesh must not fold (det J > 0, else HMG_EINVAL). Coarser levels
                             take the finest level's isoparametric map at their own nodes. */
  void (*mu_fn)(size_t n, const double* xyz, double* mu, void* user);
                          /* coefficient at n Gauss points xyz[dim][n] -> mu[n] (> 0 and finite,
                             else HMG_EINVAL), called on the setup thread once per level;
                             replaces mu_a + mu_b sum cos^2(mu_k pi x_i). */
  void* mu_user;          /* passed to mu_fn */
  int fp64_arith;         /* hmg_arith of the finest level's FP64 operator (above) */
} hmg_desc;

typedef struct hmg_problem hmg_problem;

/* Fill *d with the paper's defaults: 3D, 8^3 Q_4, unit cube, mu = 1, h-MG with 3 meshes,
 * Chebyshev(3,3), omega 2/3, 10 Arnoldi iterations, interval [lam/4, lam], FP64. */
hmg_status hmg_desc_default(hmg_desc* d);

/* Build the hierarchy on the current device: per level the geometric factors
 * G = mu w det(J) J^-1 J^-T at every Gauss point (Sec. 2.3), D^-1 (Sec. 3.2.1), the Chebyshev
 * bound (Sec. 3.2.2), the 1D transfer stencils (Sec. 2.2), and the inverse of the coarsest
 * operator. Work runs on `stream`; the call synchronizes it. Owns all memory it allocates.
 * Errors: HMG_EINVAL (bad descriptor), HMG_ENOMEM, HMG_EDEVICE. */
hmg_status hmg_setup(const hmg_desc* desc, void* stream, hmg_problem** out);
/* Release a hierarchy. Work the caller enqueued on it (hmg_apply, hmg_vcycle, ... on any
 * stream) must have completed: work on the legacy default stream is waited for, other streams
 * are the caller's to synchronize. Device memory returns to the stream-ordered pool and pinned
 * host buffers to the library's pool, without a device-wide synchronization. */
hmg_status hmg_destroy(hmg_problem* prob);

/* Node count N of the finest level a descriptor describes (0 if the descriptor is invalid). */
size_t hmg_desc_ndof(const hmg_desc* desc);

/* Device bytes hmg_setup will hold for this descriptor (resident) and its peak during setup
 * (resident plus setup temporaries), computed without touching the device. Used for
 * admission by memory budget. */
hmg_status hmg_estimate_bytes(const hmg_desc* desc, size_t* resident, size_t* peak);

/* Hierarchy introspection. level_info writes nelem[3], order and the node count. */
int hmg_nlevels(const hmg_problem* prob);
size_t hmg_ndof(const hmg_problem* prob, int level);
hmg_status hmg_level_info(const hmg_problem* prob, int level, int* nelem3, int* order, size_t* ndof);
size_t hmg_device_bytes(const hmg_problem* prob);
/* Apply variants the setup's autotuner chose on a level (no counterpart in the paper):
 * FP64 operator (0-2 point-parallel block shapes, 3 with TMA-staged factors, 4 stored dense element
 * matrices for orders 1-2, 5 and 6 the pencil form with even/odd line products at orders >= 7,
 * factors read at their use (5) or one phase ahead (6, orders 7-8)) and the mixed V-cycle's operator
 * (pencil form, when a thread loads its factors: 0 one phase before the pointwise product, 1 before
 * the first phase, 2 at their use; 3 the tensor-core form, 16-bit factors at 3D orders 1-4, built
 * when the environment sets HMG_TC16=1). FP64 variant 7 on the finest level: the double-float
 * operator that hmg_desc.fp64_arith = HMG_ARITH_DF64 asks for (never chosen by timing). */
hmg_status hmg_level_variants(const hmg_problem* prob, int level, int* v_fp64, int* v_vcycle);

/* Physical node coordinates of a level, written as xyz_dev[c * N + node], c < dim (the warp map,
 * or with node_xyz the given finest coordinates and the finest isoparametric map on coarser levels). */
hmg_status hmg_node_coords(hmg_problem* prob, int level, double* xyz_dev, void* stream);

/* Load vector b_j = (f_h, phi_j) for the nodal interpolant f_h of f (all N nodal values used),
 * by the same Gauss rule (Sec. 2.1 f_k); boundary entries of b are zero. */
hmg_status hmg_rhs(hmg_problem* prob, const double* f_nodal_dev, double* b_dev, void* stream);

/* y = A_k x on level k: the matrix-free sum-factorized stiffness apply (Sec. 2.3 matrix-free
 * discussion; (A_k)_ij = a(phi_i, phi_j), Sec. 2.1), Dirichlet nodes masked. */
hmg_status hmg_apply(hmg_problem* prob, int level, const double* x_dev, double* y_dev, void* stream);

/* FP32-vector variant of hmg_apply: the operator the mixed-precision V-cycle applies on level k
 * (FP32 vectors and arithmetic; geometric factors in FP32 for smooth_prec = HMG_PREC_FP32, in
 * 16 bits for HMG_PREC_FP16 / HMG_PREC_BF16). Needs a smooth_prec other than HMG_PREC_FP64 at
 * setup. */
hmg_status hmg_apply_f32(hmg_problem* prob, int level, const float* x_dev, float* y_dev, void* stream);

/* D^-1 of level k (inverse diagonal of A_k; 0 on boundary nodes), Sec. 3.2.1. */
hmg_status hmg_diag_inv(hmg_problem* prob, int level, double* dinv_dev, void* stream);

/* Chebyshev bound of level k (largest Ritz value of D^-1 A_k after the Arnoldi steps), Sec. 3.2.2. */
hmg_status hmg_lambda_max(const hmg_problem* prob, int level, double* lam);

/* Inter-grid transfer between level k (fine) and k+1 (coarse), Sec. 2.2 Eq. (Pstencil):
 * x_f = P x_c (overwrites x_f) and r_c = P^T r_f. */
hmg_status hmg_prolong(hmg_problem* prob, int level, const double* xc_dev, double* xf_dev, void* stream);
hmg_status hmg_restrict(hmg_problem* prob, int level, const double* rf_dev, double* rc_dev, void* stream);

/* r_c = P^T r_f without a problem handle and without allocating: for callers that cannot
 * allocate device memory (code where cudaMalloc is forbidden or unsafe -- an allocation-free
 * real-time loop, a plug-in that may only use memory its host hands in, a process whose
 * memory manager owns the device), and so cannot create an hmg_problem. The paper has no
 * counterpart; it is the same restriction as hmg_restrict, for a structured mesh described
 * by its sizes: fine level nelem_fine[dim] elements of order_fine; the coarse level halves
 * the elements per axis (halve_mesh != 0, counts must be even) and/or has order_coarse <=
 * order_fine. rf_dev / rc_dev: caller-owned FP64 node vectors of the fine / coarse level
 * (lexicographic, x fastest, boundary entries ignored / written as zero); rf_dev must hold at
 * least prod_a (nelem_fine[a] * order_fine + 1) doubles and rc_dev at least
 * prod_a (Ec[a] * order_coarse + 1), Ec[a] = nelem_fine[a] / 2 when halving, else nelem_fine[a]
 * (a < dim). The C ABI cannot check device buffer sizes: shorter buffers are read and written
 * out of bounds.
 * Limits (fixed device storage held by every device that loads the library, ~18.5 MiB):
 * at most 4097 fine nodes per axis, and the two intermediate passes together at most
 * 2^21 doubles (16 MiB) -- e.g. a 129^3-node fine level; larger sizes return HMG_EINVAL.
 * That storage is reserved when the CUDA module of the library is loaded on a device; with
 * lazy module loading (the CUDA default) that may happen during this entry point's first
 * call on the device, which also looks up the storage's device addresses. A caller that may
 * not allocate at all makes one warm-up call (or sets CUDA_MODULE_LOADING=EAGER) before it
 * enters its allocation-free region. Every call copies the 1D stencils from pageable host
 * memory, which synchronizes `stream` before each copy starts; no call can therefore be
 * recorded into a CUDA graph by stream capture. Every call reuses the same storage (stencils
 * and intermediates), so calls that overlap on the GPU (different streams, or without
 * ordering between them) race; calls on one stream are ordered. */
hmg_status hmg_restrict_noalloc(int dim, const int nelem_fine[3], int order_fine, int order_coarse,
                                int halve_mesh, const double* rf_dev, double* rc_dev, void* stream);

/* `steps` smoothing steps on level k for A_k x = b (Jacobi or Chebyshev per the descriptor);
 * zero_guess != 0 treats x as zero on input. */
hmg_status hmg_smooth(hmg_problem* prob, int level, const double* b_dev, double* x_dev, int steps,
                      int zero_guess, void* stream);

/* z = V-cycle(r) from a zero initial guess on the finest level (Sec. 3.2.2, 4.3). */
hmg_status hmg_vcycle(hmg_problem* prob, const double* r_dev, double* z_dev, void* stream);

/* Solve A u = b on the finest level to ||r||_2 <= rtol ||b||_2 (Sec. 4.3), from u = 0:
 * HMG_MODE_MG repeats V-cycles; HMG_MODE_PCG is Algorithm 1 (one V-cycle per iteration).
 * iters: V-cycles (MG) or CG iterations (PCG). res_hist: host array of >= maxit+1 doubles,
 * res_hist[i] = ||r_i||_2 (may be NULL). Returns HMG_ENOCONV (u and history written) if
 * maxit is reached, HMG_ENAN on a non-finite residual. Synchronizes `stream`. */
hmg_status hmg_solve(hmg_problem* prob, int mode, const double* b_dev, double* u_dev, double rtol,
                     int maxit, int* iters, double* res_hist, void* stream);

/* Host-buffer forms of hmg_apply and of hmg_rhs + hmg_solve, for callers whose data lives in host
 * memory: the call copies its input into library-owned device staging (two finest-level FP64
 * vectors, allocated from the stream-ordered pool on the first host-buffer call of a handle and
 * held until hmg_destroy), runs the device path on `stream`, copies the result back and
 * synchronizes `stream`. Page-locked host buffers give full copy bandwidth; pageable ones work.
 * hmg_apply_host: y_host = A_k x_host on level k (hmg_ndof(prob, k) doubles each; Sec. 2.1, 2.3).
 * hmg_solve_host: f_host is the nodal right-hand side f (hmg_ndof(prob, 0) doubles); the load
 * vector b = M f (Sec. 2.1) is formed on the device and A u = b solved as by hmg_solve (Sec. 4.3,
 * Algorithm 1; same mode, rtol, maxit, iters, res_hist and statuses); u_host receives u, also
 * when the status is HMG_ENOCONV or HMG_ENAN. */
hmg_status hmg_apply_host(hmg_problem* prob, int level, const double* x_host, double* y_host, void* stream);
hmg_status hmg_solve_host(hmg_problem* prob, int mode, const double* f_host, double* u_host, double rtol,
                          int maxit, int* iters, double* res_hist, void* stream);

/* PCG on prob's finest operator A_p (Algorithm 1's loop, from u = 0, to ||r|| <= rtol ||b||)
 * preconditioned by the low-order operator on the same nodes (Sec. 3.1.3; Sec. 4.2's
 * "low-order MG pCG" column): `low` is a problem of order 1 on the mesh of order * nelem
 * elements per axis whose node_xyz are prob's finest node coordinates (hmg_node_coords) and
 * whose coefficient is prob's, so that both share the node grid and its lexicographic
 * numbering; each M^-1 r is low's own multigrid-preconditioned CG solve to inner_rtol (the
 * paper factors the low-order matrix; a tight inner_rtol stands in for that exact solve).
 * iters: outer CG iterations; inner_iters (may be NULL): inner CG iterations in total;
 * res_hist as for hmg_solve. HMG_EINVAL if the node grids differ or low is not of order 1.
 * Synchronizes `stream`. */
hmg_status hmg_solve_low_order(hmg_problem* prob, hmg_problem* low, const double* b_dev, double* u_dev,
                               double rtol, int maxit, double inner_rtol, int* iters, long long* inner_iters,
                               double* res_hist, void* stream);

/* n independent solves (different meshes, orders and coefficients allowed) as one call: a batch
 * plan (hmg_batch_create, below) built for the call, solved once and destroyed; batches with an
 * element-block Jacobi problem instead launch every problem's own per-iteration graphs in lockstep
 * on a pool of streams forked from and joined back to `stream`, which is synchronized on return.
 * b[i], u[i]: problem i's vectors; iters[i], res_hist[i] (host, >= maxit+1 doubles) and
 * status[i] may be NULL. Returns HMG_OK if every solve converged, else the first failing
 * status. A handle may appear only once per call. (Batched form of Sec. 4.3 / Algorithm 1.) */
hmg_status hmg_solve_batched(hmg_problem* const* probs, int n, int mode, const double* const* b_dev,
                             double* const* u_dev, double rtol, int maxit, int* iters, double* const* res_hist,
                             int* status, void* stream);

/* A batch plan: n independent problems (different meshes, orders, coefficients) solved together
 * by one CUDA graph launch per solve (batched form of Sec. 4.3 / Algorithm 1). Problems whose
 * hierarchies share their structure (dimension, levels, order per level, smoother, nu_pre / nu_post,
 * smooth_prec) form a group; every operator apply, smoothing step, transfer, coarsest solve and PCG
 * vector step of a group is one kernel launch over all its members, the groups run as parallel
 * branches, and a device-side loop iterates until every member has converged, reached maxit or gone
 * non-finite -- each member stopping at the iteration it would stop at alone.
 * hmg_batch_create: builds the plan (device tables, super-vectors, the instantiated graph) for
 *   mode HMG_MODE_MG or HMG_MODE_PCG and iteration caps up to maxit_cap. The problems must outlive
 *   the plan and may appear once each; element-block Jacobi problems are refused (HMG_EINVAL).
 * hmg_batch_solve: b_dev[i] -> u_dev[i] for problem i (as hmg_solve, from u = 0, to
 *   ||r|| <= rtol ||b||); iters, res_hist[i] (>= maxit+1 doubles), status may be NULL. Returns
 *   HMG_OK if every solve converged, else the first failing status. Synchronizes `stream`.
 * hmg_batch_info: number of groups and kernels launched per loop iteration. */
typedef struct hmg_batch hmg_batch;
hmg_status hmg_batch_create(hmg_problem* const* probs, int n, int mode, int maxit_cap, hmg_batch** out);
hmg_status hmg_batch_solve(hmg_batch* plan, const double* const* b_dev, double* const* u_dev, double rtol, int maxit,
                           int* iters, double* const* res_hist, int* status, void* stream);
hmg_status hmg_batch_info(const hmg_batch* plan, int* groups, long long* kernels_per_iteration);
hmg_status hmg_batch_destroy(hmg_batch* plan);

/* Number of finest-level operator applies issued since setup (cost-model accounting,
 * Sec. 4.2/4.3: 7 per V(3,3) cycle). */
long long hmg_fine_applies(const hmg_problem* prob);

/* Number of CUDA kernels this library has launched in this process (all handles). */
long long hmg_launch_count(void);

/* ---- serving: continuous batching of independent solves (one GPU) ----
 * A server owns `max_slots` worker threads with one CUDA stream each. Submitted requests queue
 * in FIFO order; a worker starts the head request as soon as a slot is free and its peak device
 * memory (hmg_estimate_bytes plus its vectors) fits in `hbm_budget` beside what is resident.
 * Hierarchies stay resident after their solve, keyed by the descriptor, so a later request for
 * the same problem skips hmg_setup; idle ones are evicted least-recently-used when an admission
 * needs the memory. Each request is hmg_rhs + hmg_solve on the worker's stream; work of
 * different requests overlaps on the device. The server is thread-safe. */
typedef struct hmg_server hmg_server;
hmg_status hmg_server_create(int device, size_t hbm_budget, int max_slots, hmg_server** out);
/* f_host: nodal right-hand side (hmg_desc_ndof(desc) doubles, copied at submit). Returns
 * HMG_ENOMEM if the request could never fit the budget. */
hmg_status hmg_server_submit(hmg_server* srv, const hmg_desc* desc, const double* f_host, double rtol, int mode,
                             int maxit, unsigned long long* ticket);
/* HMG_EBUSY while the request is queued or running; otherwise its solve status, once (the ticket
 * is released). u_host (hmg_desc_ndof doubles), iters, res_final (final relative residual) and
 * latency_s (submit to completion) may be NULL. */
hmg_status hmg_server_poll(hmg_server* srv, unsigned long long ticket, double* u_host, int* iters,
                           double* res_final, double* latency_s);
/* As poll, blocking up to timeout_s seconds (HMG_ETIMEOUT if still running). */
hmg_status hmg_server_wait(hmg_server* srv, unsigned long long ticket, double timeout_s, double* u_host,
                           int* iters, double* res_final, double* latency_s);
hmg_status hmg_server_stats(hmg_server* srv, long long* completed, long long* cache_hits, size_t* resident_bytes,
                            int* queued);
/* Stops the workers after the running requests, frees every resident hierarchy. */
hmg_status hmg_server_destroy(hmg_server* srv);

const char* hmg_status_string(hmg_status s);
const char* hmg_last_error(void);

/* Measured arithmetic peak of the current device in TFLOP/s, the denominator of the operator's
 * FP64 roofline (no counterpart in the paper): what = 0 FP64 fused multiply-add on the CUDA cores,
 * 1 FP32 fused multiply-add, 2 FP64 tensor-core MMA (m8n8k4), 3 both FP64 forms at once (half of
 * each block's warps each: a combined rate no higher than either alone means they share the FP64
 * units). Independent FMA (MMA) chains in every thread of 8 blocks of 256 threads per SM, best of
 * three timed launches (CUDA events, legacy default stream, synchronized) after a warm-up launch;
 * tens of milliseconds per call. */
hmg_status hmg_measure_peak(int what, double* tflops);

/* Failure-detection self test: one device thread waits, with at most `polls` polls, on an
 * mbarrier that nothing completes (no copy in flight) -- the bounded wait every TMA-staged kernel
 * uses. *timed_out = 1 and HMG_ETIMEOUT when the wait gave up; the context stays usable. */
hmg_status hmg_selftest_bounded_wait(unsigned polls, int* timed_out);

/* ---- host-only helpers (no device needed): the library's own 1D tables and eigen step ---- */

/* GLL nodes r[p+1], Gauss points g[p+1] and weights w[p+1] on [0,1] (Sec. 2.3, Fig. 1). */
hmg_status hmg_host_basis(int order, double* gll, double* gauss_x, double* gauss_w);

/* Largest real part of the eigenvalues of an m x m upper Hessenberg matrix (row-major),
 * by the Francis double-shift QR algorithm: the Ritz-value step of the Chebyshev bound. */
hmg_status hmg_host_hessenberg_max_real_eig(const double* H, int m, double* out);

#ifdef __cplusplus
}
#endif

#endif /* HMG_H */
