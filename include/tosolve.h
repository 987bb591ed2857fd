/*
 * tosolve.h -- C ABI of the GB300 (sm_103a) multigrid-preconditioned CG
 * solver for the multiresolution SIMP elasticity problem of Vitorino & Gomes,
 * "An efficient topology optimization algorithm for large-scale
 * three-dimensional structures" (arXiv 2311.05595).
 *
 * The library computes, on one GPU, the hot path of one SLP iteration:
 *   design variables x  --(density filter / projection, Sec. 2.2 and 3.2)-->
 *   densities rho       --(SIMP weights, Eq. matrixK_mr)-->  K(rho)
 *   K(rho) u = f        --(MG-preconditioned CG, Alg. 1, Sec. 2.3, 7.2)-->  u
 *   c = f^T u and dc/dx --(Sec. 3.4)-->  back to the host optimizer.
 *
 * Mesh and numbering (shared by every call):
 *   * nx*ny*nz cubic displacement elements of edge 1 (Sec. 7.1);
 *   * Lagrange degree k (1, 2 or 3): node lattice (k*nx+1)*(k*ny+1)*(k*nz+1),
 *     node id = i + Lx*(j + Ly*l) (x fastest), DOF = 3*node + component;
 *   * each element holds n_mr^3 density cells (Sec. 3.1): the density grid
 *     is (n_mr*nx)*(n_mr*ny)*(n_mr*nz) cells, flattened x fastest; the
 *     design grid (x and dc/dx) is the same with d_mr in place of n_mr;
 *     d_mr < n_mr projects x onto the densities with the filter weights
 *     between cell centres of the two grids (Sec. 3.2, Eq. projdsgn);
 *   * the Dirichlet mask has one byte per DOF, 1 = fixed (u = 0 there).
 *
 * Conventions of every call:
 *   * pointers named *_dev are device pointers (any allocator) on the
 *     device that was current at tosolve_create; *_host are host pointers;
 *     the caller owns every buffer it passes and the library keeps no
 *     reference to it after the call returns;
 *   * the library owns its workspace (allocated in tosolve_create, freed in
 *     tosolve_destroy); no call other than create/destroy allocates device
 *     memory;
 *   * work is issued on the stream given to tosolve_create; calls that return
 *     host values (tosolve_solve's info, tosolve_compliance_grad's c_host,
 *     tosolve_step_host) synchronise that stream before returning, the others
 *     are asynchronous;
 *   * every call returns a tosolve_status; on failure tosolve_last_error
 *     gives a one-line reason.  No call aborts the process or traps on the
 *     GPU.
 */
#ifndef TOSOLVE_H_
#define TOSOLVE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tosolve_s* tosolve_t;

typedef enum {
  TOSOLVE_OK = 0,
  TOSOLVE_EINVAL = 1,      /* bad descriptor, size, pointer or argument      */
  TOSOLVE_ENOMEM = 2,      /* device allocation failed in tosolve_create     */
  TOSOLVE_ENOTCONV = 3,    /* tolerance not reached (maxit or restarts); info valid */
  TOSOLVE_EBREAKDOWN = 4,  /* NaN/Inf, p^T K p <= 0 or a non-positive pivot  */
  TOSOLVE_ECUDA = 5        /* a CUDA runtime call failed                     */
} tosolve_status;

/* Precision of the multigrid preconditioner (the outer CG, its dot
 * products, the true residual, the coarse inverse, the compliance and the
 * gradient are always FP64). */
typedef enum {
  TOSOLVE_PREC_FP64 = 0, /* plain FP64 MG-PCG                                */
  TOSOLVE_PREC_FP32 = 1, /* FP32 V-cycle operators and vectors, FP32 accum.  */
  TOSOLVE_PREC_TF32 = 2, /* as FP32, but the finest level's operator is the  */
                         /* stacked subcell contraction of Eq. matrixK_mr on */
                         /* the tcgen05 tensor cores (TF32 operands, FP32    */
                         /* accumulation in TMEM); degree 1 with n_mr <= 2,  */
                         /* or Lagrange degree 2 with n_mr <= 3, mixed       */
                         /* trilinear/triquadratic meshes included           */
  TOSOLVE_PREC_FP32X2 = 3, /* FP32 V-cycle operators (formed in FP64, then   */
                         /* rounded) and vectors held as float pairs: about */
                         /* 48-bit arithmetic on the FP32 pipes, for        */
                         /* high-contrast densities where FP32 vectors slow */
                         /* convergence                                     */
  TOSOLVE_PREC_BF16 = 4, /* as TF32 with BF16 operands (8-bit mantissas) and */
                         /* FP32 accumulation: Lagrange degree 2 with       */
                         /* n_mr <= 3, mixed meshes included                */
  TOSOLVE_PREC_BF16X3 = 5, /* degree 2 as BF16, each operand split into a   */
                         /* BF16 pair (hi + lo, about 16 bits) and three    */
                         /* products hi hi + lo hi + hi lo                  */
  TOSOLVE_PREC_F16X3 = 6 /* degree 2 as BF16X3 with FP16 pairs (about 22   */
                         /* bits; vectors scaled per element and the table  */
                         /* globally by powers of two into FP16's range):   */
                         /* FP32-class operator accuracy at the FP16 tensor */
                         /* rate                                            */
} tosolve_precision;

/* Problem and solver description (Sec. 2, 3.1, 7 intro). */
typedef struct {
  int nx, ny, nz;         /* displacement elements per axis, >= 1           */
  int degree;             /* degree k: 1, 2 or 3 (see family)               */
  int n_mr;               /* density cells per element edge, 1..8           */
  int d_mr;               /* design cells per element edge, 1..n_mr (0 =   */
                          /* n_mr); below n_mr rmin must be > 0            */
  double E0, Emin;        /* SIMP: E(rho) = Emin + rho^p (E0 - Emin), Eq.   */
  double nu;              /*   matrixK; Poisson ratio nu in (-1, 0.5)       */
  double penal;           /*   penalty p >= 1                               */
  double rmin;            /* filter radius in element units; 0 => rho = x  */
  int mg_levels;          /* multigrid levels >= 1 (each halves the mesh;   */
                          /*   nx, ny, nz divisible by 2^(levels-1))        */
  int precision;          /* tosolve_precision of the preconditioner        */
  double omega;           /* damped-Jacobi factor (0 => 0.5, Sec. 7 intro;  */
                          /*   0.4 for Lagrange degree 2 and 3, 0.3 for     */
                          /*   serendipity: below 2 / lambda_max(D^-1 A))  */
  int cycle_gamma;        /* cycles per level: 1 = V-cycle (0 => 1; the     */
                          /*   only value this build accepts)               */
  int max_rhs;            /* load cases per solve call, >= 1 (0 => 1)       */
  int family;             /* element family (Sec. 2.1): 0 Lagrange; 1 the   */
                          /*   20-node serendipity element (degree 2 only), */
                          /*   on the degree-2 lattice without the face and */
                          /*   element-centre nodes, which the library holds */
                          /*   at 0 with the supports; coarse levels are    */
                          /*   serendipity meshes with shape-function       */
                          /*   transfers (Sec. 2.3)                         */
  int prolongation;       /* degree-2 transfers: 0 the coarse shape         */
                          /*   functions (Sec. 2.3 for serendipity; nested  */
                          /*   spaces, so the re-discretised coarse         */
                          /*   operators are the Galerkin products), 1      */
                          /*   linear interpolation on the node lattices    */
                          /*   (the paper's choice for Lagrange elements;   */
                          /*   not for serendipity); degree 1: the two are  */
                          /*   the same trilinear interpolation             */
  int inner_its;          /* 0: each outer FP64 CG iteration is              */
                          /*   preconditioned by one V-cycle (Alg. 1);       */
                          /*   k in 1..64: by k iterations of CG in FP32 on  */
                          /*   the level-0 operator of the preconditioner    */
                          /*   (the tensor-core stacked contraction, or the  */
                          /*   FP32 element matrices), each preconditioned   */
                          /*   by one V-cycle; the outer CG is flexible, its */
                          /*   residual, dot products and operator stay FP64 */
                          /*   (degree 2, FP32-vector precisions only)       */
  int smoother;           /* 0: damped Jacobi (Sec. 7 intro; omega above);  */
                          /*   1: Chebyshev on D^-1 A (degree 2 and 3, not  */
                          /*   FP32X2): at each tosolve_set_densities a     */
                          /*   few Lanczos steps estimate lambda_max of     */
                          /*   every level's smoothing operator, and the    */
                          /*   smoother is the Chebyshev iteration over     */
                          /*   [0.3 b, b], b = 1.1 lambda_max (Saad, Alg.   */
                          /*   12.1); omega is then ignored                 */
  int cheb_degree;        /* Chebyshev steps before and after the coarse    */
                          /*   correction, 1..4 (0: 2)                      */
} tosolve_desc;

typedef struct {
  int iterations;       /* PCG iterations of the last right-hand side        */
  int total_iterations; /* summed over the right-hand sides of the call      */
  double rel_residual;  /* max over rhs of the FP64 true ||f - K u|| / ||f|| */
  double ms;            /* device time of the solve (CUDA events)            */
  int status;           /* tosolve_status of the call                        */
} tosolve_info;

/* Builds the solver for one mesh: validates the descriptor, allocates all
 * device memory, computes the stacked subcell stiffness table K^(e_i)
 * (Sec. 3.3, Eq. matrixK_mr: computed once for a regular mesh), the filter
 * stencil and the multigrid level descriptors, and records the CUDA graph of
 * the PCG loop.
 *   desc:        problem description (copied).
 *   mask_host:   3*(nx+1)*(ny+1)*(nz+1) bytes, 1 = fixed DOF (copied).
 *   cuda_stream: cudaStream_t to run on; NULL makes the library create
 *                (and own) a blocking stream, ordered with the legacy
 *                default stream.  Must not be the legacy stream handle
 *                itself when non-NULL (the PCG loop is graph-captured).
 *   out:         receives the handle.
 * Errors: EINVAL (checked before any CUDA call), ENOMEM, ECUDA. */
tosolve_status tosolve_create(const tosolve_desc* desc, const uint8_t* mask_host,
                              void* cuda_stream, tosolve_t* out);

/* A mesh that mixes trilinear and triquadratic elements on the degree-2
 * lattice (desc->degree = 2, family 0).  elem_q1_host: nx*ny*nz bytes (x
 * fastest), 1 = trilinear element.  A triquadratic element carries its
 * matrix of Eq. matrixK_mr, a trilinear element its trilinear 24 x 24
 * matrix on its 8 vertices; a lattice node that is not an element vertex
 * and touches a trilinear element is slaved to the linear interpolation of
 * the vertices of its edge, face or cell (the coupling is conforming; the
 * paper raises the degree of the whole mesh, Sec. 7.4, and does not spell a
 * mixed coupling out).  The solve is on u = T u_r with T^T K T u_r = T^T f;
 * u_dev returns the expanded field, loads f_dev are the degree-2 consistent
 * loads on the whole lattice, compliance and gradient use the expanded u.
 * Otherwise as tosolve_create, every precision included.  Errors: EINVAL,
 * ENOMEM, ECUDA. */
tosolve_status tosolve_create_mixed(const tosolve_desc* desc, const uint8_t* mask_host,
                                    const uint8_t* elem_q1_host, void* cuda_stream, tosolve_t* out);

/* Number of unknowns of the handle's system: lattice DOFs that are neither
 * supported, (mixed meshes) slaved, nor suppressed by
 * tosolve_fix_variables.  Errors: EINVAL. */
tosolve_status tosolve_free_dofs(tosolve_t h, long long* n);

/* Fixing variables and suppressing DOFs of void regions (Sec. 6.1).  From the
 * densities of the last tosolve_set_densities and an optional design
 * gradient:
 *   an element is void when all its densities are <= rho_lo and all its
 *   design-gradient components are >= -eps_grad, solid when all densities
 *   are >= rho_hi and all components are <= eps_grad (the paper uses
 *   rho_lo = 1e-6, rho_hi = 0.9, eps_grad = 1e-6); an element is fixed when
 *   every element sharing a node with it (inside the domain) is of its kind;
 *   a lattice node is suppressed when every element containing it is a fixed
 *   void element: its DOFs join the supports (u = 0, rows and columns out of
 *   K, loads ignored) and the multigrid setup is redone at once.
 *   dcdx_dev:  design grid FP64 (e.g. from tosolve_compliance_grad), or NULL
 *              to use the density conditions alone.
 *   fixed_dev: NULL, or one byte per design variable (device) receiving the
 *              class of its fixed element: 0 free, 1 void, 2 solid (an SLP
 *              loop gives these variables zero step bounds).
 *   suppressed_dofs: NULL or (host) the DOFs suppressed.
 * The selection replaces any earlier one and stays in force through later
 * tosolve_set_densities calls until tosolve_release_variables; while it is in
 * force tosolve_compliance_grad returns dc/dx = 0 for the variables of fixed
 * void elements.  Synchronises.  Errors: EINVAL (no densities set, bad
 * thresholds), ECUDA. */
tosolve_status tosolve_fix_variables(tosolve_t h, const double* dcdx_dev, double rho_lo, double rho_hi,
                                     double eps_grad, uint8_t* fixed_dev, long long* suppressed_dofs);

/* ---- Thresholding and the Heaviside projection (Sec. 5) -------------------
 * Device-side steps of the density projection strategy, on a density vector
 * of n equal-volume cells (rho_dev, n FP64 on the device, values in [0, 1]).
 * They are independent of any handle: each takes a caller-owned device
 * scratch buffer of at least tosolve_threshold_scratch_bytes(n) bytes and
 * runs on cuda_stream (NULL: the legacy default stream), synchronising it.
 * With n = 0 nothing is read or written and pointers may be NULL.
 * Errors (tosolve_last_error(NULL)): EINVAL (NULL pointer, n outside
 * 0..2^31-1, a parameter out of range, scratch too small), ECUDA. */
size_t tosolve_threshold_scratch_bytes(long long n);

/* Heaviside projection: out = h(rho, beta, eta) with h(rho, beta, eta) =
 * (tanh(beta eta) + tanh(beta (rho - eta))) / (tanh(beta eta) +
 * tanh(beta (1 - eta))) and eta the zero of sum h(rho_i, beta, eta) -
 * sum rho_i (the volume is kept), by Newton's method from eta = 1/2 (a step
 * that would leave (0, 1) is halved; stop when |f| <= 1e-12 n or the step
 * is below 1e-14).  beta > 0.  eta, newton_its: host, may be NULL. */
tosolve_status tosolve_heaviside(const double* rho_dev, long long n, double beta, double* out_dev, double* eta,
                                 int* newton_its, void* scratch_dev, size_t scratch_bytes, void* cuda_stream);

/* Strategy based on the density values: densities >= round_hi become 1 and
 * <= round_lo become 0 (the paper: 0.95, 0.05); then the floor(vfrac n)
 * largest become 1 and the others 0 (among equal densities the lower index
 * first).  accepted (host, may be NULL) = 1 when d = out - rho_rounded and
 * -gradL make an angle below theta_max_deg (Eq. angle; the paper: 89.9).
 * gradL_dev: n FP64, the gradient of the Lagrangian w.r.t. the densities. */
tosolve_status tosolve_threshold_density(const double* rho_dev, long long n, double vfrac, double round_lo,
                                         double round_hi, const double* gradL_dev, double theta_max_deg,
                                         double* out_dev, int* accepted, void* scratch_dev, size_t scratch_bytes,
                                         void* cuda_stream);

/* Strategy based on the gradient of the Lagrangian: the same rounding, then
 * out = clip(rho - alpha gradL, 0, 1) with alpha the largest of the steps at
 * which a component reaches its bound (0 where gradL > 0, 1 where < 0; ties
 * ordered by index) such that out satisfies the angle condition and no
 * component reached 1 from a density below vu_min or 0 from one above
 * vl_max (the paper: 0.3, 0.7); alpha = 0 if none qualifies.  alpha: host,
 * may be NULL. */
tosolve_status tosolve_threshold_gradient(const double* rho_dev, const double* gradL_dev, long long n,
                                          double round_lo, double round_hi, double vu_min, double vl_max,
                                          double theta_max_deg, double* out_dev, double* alpha, void* scratch_dev,
                                          size_t scratch_bytes, void* cuda_stream);

/* Drops the selection of tosolve_fix_variables: the supports alone again,
 * multigrid setup redone if densities are set.  Synchronises.  Errors:
 * EINVAL, ECUDA. */
tosolve_status tosolve_release_variables(tosolve_t h);

/* Device memory tosolve_create would allocate for desc, in bytes (host
 * only; used for HBM admission).  Errors: EINVAL. */
tosolve_status tosolve_footprint(const tosolve_desc* desc, size_t* bytes);

/* New design: x_dev (design grid, FP64) -> rho = H x (Sec. 2.2 Eq.
 * filter_weights, Sec. 3.2 Eq. projdsgn), SIMP weights w = Emin +
 * rho^p (E0 - Emin), and the multigrid refresh of Sec. 7.2: every level's
 * operator from the densities, the Jacobi diagonals and the explicit FP64
 * inverse of the coarsest operator (the direct coarse solve; formed by
 * blocked symmetric Gauss-Jordan sweeps, whose pivots are those of a
 * Cholesky factorisation).  Asynchronous.
 * Errors: EINVAL, ECUDA. */
tosolve_status tosolve_set_densities(tosolve_t h, const double* x_dev);

/* Solves K(rho) u = f for nrhs load cases by MG-preconditioned CG (Sec. 2.3,
 * 7.2) until the true FP64 residual ||f - K u||_2 / ||f||_2 <= rtol.
 *   f_dev: nrhs x ndof FP64 (rows contiguous); f at fixed DOFs is ignored.
 *   u_dev: nrhs x ndof FP64; in: initial guess (warm start, Sec. 7.2.1),
 *          out: solution, 0 at fixed DOFs.
 *   info:  may be NULL; always written when non-NULL.
 * maxit is in 1..100000 (bounds the device-side loop).
 * When the recursive residual meets rtol but the true one does not, the
 * loop restarts from the current iterate, at most three times.
 * Synchronises the stream.  Errors: EINVAL, ENOTCONV (maxit reached, or the
 * true residual still above rtol after the three restarts), EBREAKDOWN,
 * ECUDA. */
tosolve_status tosolve_solve(tosolve_t h, const double* f_dev, int nrhs, double* u_dev,
                             double rtol, int maxit, tosolve_info* info);

/* Compliance and sensitivities for nrhs solutions (Sec. 3.4):
 *   c_host[r]  = f_r^T u_r                                  (FP64, host)
 *   dcdrho_dev = sum_r -p rho^(p-1) (E0-Emin) u_e^T K^(e_i) u_e  (density
 *                grid, may be NULL)
 *   dcdx_dev   = H^T dcdrho (design grid, may be NULL).
 * Synchronises the stream (c_host).  Errors: EINVAL, ECUDA. */
tosolve_status tosolve_compliance_grad(tosolve_t h, const double* u_dev, const double* f_dev,
                                       int nrhs, double* c_host, double* dcdx_dev,
                                       double* dcdrho_dev);

/* One whole SLP-iteration step from host buffers: copies x and f from the
 * host, runs set_densities, solve and compliance_grad, and copies u, c and
 * dc/dx back.  warm != 0 starts the solve from this handle's previous
 * solution (zero at the first call; Sec. 7.2.1 reuses the last solution),
 * warm == 0 from zero.  Buffers as above but on the host (pinned memory
 * makes the copies asynchronous); u_host and dcdx_host may be NULL.
 * Synchronises.  Errors: as the calls it makes. */
tosolve_status tosolve_step_host(tosolve_t h, const double* x_host, const double* f_host,
                                 int nrhs, double rtol, int maxit, int warm, double* u_host,
                                 double* c_host, double* dcdx_host, tosolve_info* info);

/* ---- Batches: many independent instances in one graph launch ---------- */

typedef struct tosolve_batch_s* tosolve_batch_t;

/* Records one CUDA graph that solves every load case of every instance.
 * Each instance is one parallel branch of the graph; its load cases follow
 * one another inside that branch (they share the handle's workspace), each
 * a device-side while loop like tosolve_solve's.  Instances of uneven size
 * therefore run concurrently and the whole batch is a single launch.
 *   handles: count distinct handles (1 <= count <= 4096; each has its own
 *            workspace, so a handle appears at most once).  The operators
 *            used are whatever the last tosolve_set_densities on each handle
 *            produced.  Handles outlive the batch.
 *   nrhs:    load cases per instance (1 .. that handle's max_rhs).
 *   f_dev, u_dev: per instance, nrhs x ndof FP64 device buffers (layout as
 *            in tosolve_solve).  The graph is bound to these addresses: the
 *            caller keeps them alive until tosolve_batch_destroy.
 * Errors: EINVAL (NULL, duplicate handle, nrhs out of range, a handle
 * created with graphs disabled), ENOMEM, ECUDA. */
tosolve_status tosolve_batch_create(const tosolve_t* handles, int count, const int* nrhs,
                                    const double* const* f_dev, double* const* u_dev,
                                    tosolve_batch_t* out);

/* Runs the batch once from the current contents of u_dev (warm start) to
 * ||f - K u|| / ||f|| <= rtol for every load case (1 <= maxit <= 100000),
 * ordered after all work issued so far on the instances' streams; work
 * issued on them later waits for the batch.  A load case whose recursive
 * residual met rtol but whose true residual did not is finished by
 * tosolve_solve on its own handle.  infos: count entries (one per instance,
 * as tosolve_solve's info; ms is the whole batch's graph time), may be NULL.
 * Synchronises.  Errors: ENOTCONV if a load case reached maxit first,
 * EBREAKDOWN, EINVAL (rtol, maxit, densities not set), ECUDA. */
tosolve_status tosolve_batch_solve(tosolve_batch_t b, double rtol, int maxit, tosolve_info* infos);

/* Frees the batch (not the handles).  NULL is accepted. */
void tosolve_batch_destroy(tosolve_batch_t b);

/* ---- Autotuning (the batching pattern's variant choice) ---------------- */

/* Times candidate descriptors of one instance class.  For each candidate c
 * a handle is created on cuda_stream (mask_host and elem_q1_host as in
 * tosolve_create / tosolve_create_mixed; elem_q1_host may be NULL), its
 * densities are set from x_dev, one untimed solve runs from u = 0, then
 * `reps` timed solves from u = 0 of the nrhs load cases f_dev (layout as
 * in tosolve_solve) to rtol; ms_out[c * reps + r] receives the device time
 * of solve r (info.ms).  A candidate that cannot be created or does not
 * reach rtol records +infinity; the others still run.  The handles and the
 * solution buffer are freed before return.  Synchronises; allocates.
 * Errors: EINVAL (a NULL pointer, ncand or reps outside 1..64, nrhs < 1),
 * ECUDA. */
tosolve_status tosolve_tune(const tosolve_desc* cand, int ncand, const uint8_t* mask_host,
                            const uint8_t* elem_q1_host, const double* x_dev, const double* f_dev,
                            int nrhs, double rtol, int maxit, int reps, void* cuda_stream,
                            double* ms_out);

/* The choice from timings (host only; touches no device).
 * ms[(k * ncand + c) * reps + r] is repeat r of candidate c in class k.
 * Per class and candidate the median of the finite repeats is taken (it is
 * infinite when fewer than half are finite); the fastest candidate wins,
 * ties to the lower index, but candidate 0, the default, is kept unless the
 * winner is faster by more than the fraction min_gain of its time
 * (0 <= min_gain < 1).  choice[k] = -1 when no candidate of class k has a
 * finite median.  Errors: EINVAL (NULL, sizes outside 1..4096, 1..64,
 * 1..64, min_gain outside [0, 1)). */
tosolve_status tosolve_tune_pick(const double* ms, int nclass, int ncand, int reps, double min_gain,
                                 int* choice);

/* Device memory of handles and servers comes from one stream-ordered pool
 * per device.  Memory freed by tosolve_destroy (or a server eviction) stays
 * reserved in that pool for the next build; this returns the unused part
 * above keep_bytes to the driver (current device; synchronises it).
 * Errors: ECUDA. */
tosolve_status tosolve_trim_pool(size_t keep_bytes);

/* ---- Serving: SLP-iteration requests of many designs ------------------- */

/* The serving runtime keeps many independent designs (mesh, supports, load
 * cases) and runs their SLP iterations as requests arrive.  One request =
 * new design variables x -> tosolve_set_densities, a solve warm-started
 * from the design's previous displacements (Sec. 7.2.1), compliance and
 * gradient.  Requests of one design run in submission order, one at a time;
 * requests of different designs run concurrently on `slots` worker threads,
 * each on its design's own CUDA stream, so their kernels overlap on the
 * GPU.  A design's handle, buffers and warm start stay on the device while
 * the budget allows; when a request needs room, idle designs are evicted
 * least recently used first (their displacements move to the host and come
 * back as the warm start).  Results carry timestamps for latency figures. */
typedef struct tosolve_server_s* tosolve_server_t;

typedef struct {
  int slots;          /* requests running at once, 1..64                     */
  size_t hbm_budget;  /* device bytes for resident designs (handle + x, f,   */
                      /* u, gradient buffers; tosolve_footprint + those)     */
  double rtol;        /* per request, as tosolve_solve                      */
  int maxit;          /* per request, 1..100000                             */
} tosolve_server_desc;

typedef struct {
  long long request;   /* id from tosolve_server_submit                      */
  int design;
  int status;          /* tosolve_status of the request; ENOMEM if the       */
                       /* design alone exceeds hbm_budget                    */
  int iterations;      /* PCG iterations over all load cases                 */
  int cold;            /* 1 if the design was (re)built for this request     */
  double compliance;   /* sum over load cases of f^T u                       */
  double rel_residual; /* worst true relative residual                       */
  double t_submit, t_start, t_end;  /* seconds on the server's clock          */
} tosolve_request_result;

typedef struct {
  int designs, resident_designs, pending, running;
  size_t resident_bytes;
  long long builds, evictions;
  double now;          /* the server's clock, seconds                        */
} tosolve_server_info;

/* Starts the worker threads on the current device.  Errors: EINVAL, ENOMEM. */
tosolve_status tosolve_server_create(const tosolve_server_desc* desc, tosolve_server_t* out);

/* Registers design `design` (any int, unique): its descriptor, DOF mask
 * (host, as tosolve_create) and nrhs load cases f_host (nrhs x ndof, host),
 * all copied.  No device memory is used until its first request.
 * Errors: EINVAL (invalid descriptor, duplicate id). */
tosolve_status tosolve_server_add_design(tosolve_server_t s, int design, const tosolve_desc* desc,
                                         const uint8_t* mask_host, const double* f_host, int nrhs);

/* Queues one SLP iteration of `design` with design variables x_host (host,
 * copied now).  If dcdx_host is not NULL, dc/dx (summed over load cases) is
 * written there when the request completes; the caller keeps it valid until
 * the request's result has been polled.  request may be NULL.
 * Errors: EINVAL (unknown design, NULL x, server stopping). */
tosolve_status tosolve_server_submit(tosolve_server_t s, int design, const double* x_host,
                                     double* dcdx_host, long long* request);

/* Moves up to max finished results to out (completion order), waiting up
 * to timeout_ms for the first one.  Returns how many were written. */
int tosolve_server_poll(tosolve_server_t s, tosolve_request_result* out, int max, int timeout_ms);

/* Occupancy and counters.  Errors: EINVAL. */
tosolve_status tosolve_server_stats(tosolve_server_t s, tosolve_server_info* info);

/* Message of the last failed server call on this thread. */
const char* tosolve_server_last_error(void);

/* The k-th most recent failed request (k = 0: the newest; the server keeps
 * the last 64): request id, design, whether it was cold, status, iterations,
 * relative residual and the handle's error message.  NULL if k is out of
 * range.  The string stays valid until the next call on this server. */
const char* tosolve_server_failure(tosolve_server_t s, int k);

/* Drops queued requests, waits for the running ones, frees every design.
 * NULL is accepted. */
void tosolve_server_destroy(tosolve_server_t s);

/* ---- Compliance without device allocation ----------------------------- */

/* Most load cases handled per call, and the size in bytes of the one fixed
 * device array (per device) that holds the partial sums. */
#define TOSOLVE_NOALLOC_MAX_RHS 16
#define TOSOLVE_NOALLOC_SCRATCH_BYTES 77824

/* c_dev[r] = f_r^T u_r summed over the free DOFs, r < nrhs: the compliance
 * that tosolve_compliance_grad returns, for callers that may not allocate
 * device memory when they need it (code confined to buffers a host
 * application hands it, or a latency-critical loop that cannot afford the
 * device-wide synchronisation a cudaMalloc can cause).  The paper has no
 * counterpart: it is a service of this library.  It allocates nothing and
 * needs no handle.
 *   f_dev, u_dev: nrhs x ndof FP64 device arrays, rows contiguous.
 *   mask_dev:     ndof bytes on the device, 1 = fixed DOF (excluded).
 *   ndof:         1 .. 2^62.
 *   nrhs:         1 .. TOSOLVE_NOALLOC_MAX_RHS; more is rejected with EINVAL.
 *   c_dev:        nrhs FP64 results on the device (caller-owned).
 *   cuda_stream:  cudaStream_t to run on (NULL = legacy default stream).
 * The partial sums live in one fixed device array of
 * TOSOLVE_NOALLOC_SCRATCH_BYTES per device, shared by every call and keeping
 * what the last call wrote; each call overwrites every entry it reads.
 * Calls whose kernels may overlap on the GPU race on that array: order them
 * (one stream, or events).  A call made outside a stream capture looks up
 * the array's address on the current device with cudaGetSymbolAddress; a
 * call inside a capture reuses the address of the last call made outside
 * one on that device, so make one call before capturing (again after a
 * cudaDeviceReset, which moves the array).  Asynchronous (does not
 * synchronise).  Errors: EINVAL (NULL pointer, ndof or nrhs out of range;
 * checked before any CUDA call), ECUDA.  Message: tosolve_last_error(NULL). */
tosolve_status tosolve_compliance_noalloc(const double* f_dev, const double* u_dev,
                                          const uint8_t* mask_dev, size_t ndof, int nrhs,
                                          double* c_dev, void* cuda_stream);

/* ---- Single steps of the path, for verification ------------------------ */

/* Number of multigrid levels and, for level l, its node lattice (Lx, Ly, Lz)
 * into dims[0..2].  Host only.  Errors: EINVAL. */
tosolve_status tosolve_level_dims(tosolve_t h, int level, int* dims);

/* Copies the stacked subcell stiffness table of the finest level, m x d x d
 * FP64 (m = n_mr^3, d = 24, E = 1), into table_dev (Sec. 3.3). */
tosolve_status tosolve_subcell_table(tosolve_t h, double* table_dev);

/* Chebyshev smoothing: the Lanczos estimate of lambda_max(D^-1 A) of level
 * l's smoothing operator from the last tosolve_set_densities, into
 * *lmax_host (synchronises the handle's stream).  Errors: EINVAL (no
 * Chebyshev smoother, level out of range or the coarsest level). */
tosolve_status tosolve_smoother_lmax(tosolve_t h, int level, double* lmax_host);

/* Copies the densities rho and SIMP weights w of the last set_densities
 * (density grid, FP64) into rho_dev / w_dev (either may be NULL). */
tosolve_status tosolve_densities(tosolve_t h, double* rho_dev, double* w_dev);

/* y = A_l x for the level-l operator (fixed rows/columns replaced by
 * identity), computed in FP64 (precision 0), in the preconditioner's FP32
 * stencil or element form (precision 1), on level 0 of a tensor-core handle
 * as the stacked contraction plus node gather (precision 2, 4, 5 or 6: the
 * handle's own), or with the FP32 operator and float-pair arithmetic of
 * FP32X2 (precision 3); inputs and outputs are FP64.  x_dev, y_dev:
 * 3*nodes(l).
 * Level 0 FP64 is K(rho) of Eq. matrixK_mr; coarser levels are re-discretised
 * from the density field (Sec. 7.2: system matrices of each mesh level). */
tosolve_status tosolve_apply(tosolve_t h, int level, int precision, const double* x_dev,
                             double* y_dev);

/* Instrumentation of the level-0 tensor-core operator (preconditioner
 * precision TF32 on degree 2, BF16, BF16X3 or F16X3), so that a caller can
 * time its stacked subcell contraction (Sec. 3.2, Eq. 10: K_e u_e =
 * sum_i w_{e,i} K_i u_e) alone between its own events on the handle's
 * stream.  part 0 = the triquadratic elements (every element of a
 * single-degree mesh), 1 = the trilinear elements of a mixed mesh, whose
 * 24 x 24 vertex blocks are applied in FP32 on the CUDA cores (in a solve
 * they run in the same launch as the triquadratic rows' packing).  stages
 * bit 0: round x_dev (FP64, device, length 3*nodes(0)) to FP32 and, for
 * part 0, pack the operand rows (masked, deflated, split) into the handle's
 * scratch; bit 1: run the part's product (part 0: the contraction kernel on
 * the rows packed last; part 1: the FP32 products from the rounded x),
 * writing the per-element results to the handle's scratch (nothing is
 * returned: use tosolve_apply for K x).  x_dev is read only with bit 0 (may
 * be NULL otherwise).  Errors: TOSOLVE_EINVAL (no such operator, bad part
 * or stages). */
tosolve_status tosolve_tc_stage(tosolve_t h, int part, int stages, const double* x_dev);

/* z = B b: one multigrid cycle (Algorithm 1, recursive, zero initial guess)
 * of the preconditioner in its configured precision; b_dev, z_dev FP64,
 * length 3*nodes(0); b must be 0 at fixed DOFs. */
tosolve_status tosolve_precondition(tosolve_t h, const double* b_dev, double* z_dev);

/* Reason for the last failure on this handle (never NULL). */
const char* tosolve_last_error(tosolve_t h);

/* Frees everything owned by the handle (NULL is accepted). */
void tosolve_destroy(tosolve_t h);

#ifdef __cplusplus
}
#endif

#endif /* TOSOLVE_H_ */
